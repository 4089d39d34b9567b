"""FP64 CPU oracle for the extrinsic-likelihood hot path (test infrastructure).

This package is the correctness reference the CUDA library is compared against.
It is plain, slow and written from the paper's equations:

* Eq. (lnL), Eq. (overlap)            -> likelihood.lnL_bruteforce
* Eq. (def:lnL:Decomposed), Eq. (QUV) -> likelihood.lnL_factorised
* Eq. (strain_mode) harmonics          -> swsh
* detector response / arrival times    -> geometry (Sec. II.A, after Eq. strain_mode)
* Eq. (lnLmarg) Monte Carlo, n_eff     -> mc (Sec. II.A, Sec. II.C)
* learned proposal                     -> mdn

Everything is float64 numpy.  It shares no code with the CUDA path and imports
nothing from it.  Only the test-suite, the smoke check and the CPU-baseline leg
of the benchmark may import this package; the library itself never does.
"""
