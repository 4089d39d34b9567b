/*
 * rift_ile.h -- C ABI of the GB300 extrinsic-likelihood library.
 *
 * The library evaluates, for one or many intrinsic points lambda, the extrinsic
 * log-likelihood of Eq. (def:lnL:Decomposed) (Sec. II.A) from precomputed mode
 * inner products Q, U, V (Eq. QUV), and reduces it to the marginalised
 * likelihood of Eq. (lnLmarg) by importance-sampled Monte Carlo (Sec. II.A, II.C).
 *
 * Conventions shared by every entry point
 *  - No exception crosses the ABI.  Every call returns a rift_status; details of the
 *    last failure on a handle are in rift_ile_last_error().
 *  - "host" pointers are ordinary CPU memory; "device" pointers are CUDA global
 *    memory of the current device.  The caller keeps ownership of everything it
 *    passes; the library copies what it needs at create time.
 *  - Complex arrays are interleaved (re, im) float64.
 *  - Angles in radians, times in seconds, distances in Mpc.
 *  - Work is issued on the handle's stream (desc.cuda_stream, NULL = legacy default).
 *    Entry points that return host results synchronise that stream; rift_ile_lnL
 *    (device buffers) does not.
 *  - The likelihood is, with F_k = F_+ - i F_x and x = D_ref / D,
 *      lnL = x Re sum_k sum_lm F_k conj(Y_lm) Q_{k,lm}(t + delay_k)
 *            - x^2/4 sum_k [ |F_k|^2 conj(Y)^T U_k Y + Re( conj(F_k)^2 Y^T V_k Y ) ],
 *    Y_lm = -2Y_lm(incl, phi), delay_k = -(x_k . n)/c.  This is Eq. (def:lnL:Decomposed)
 *    with the conjugations that follow from h_k = Re(conj(F_k) h), h = h_+ - i h_x.
 */
#ifndef RIFT_ILE_H
#define RIFT_ILE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rift_ile rift_ile; /* opaque; owns all device buffers of one or many points */

typedef enum {
  RIFT_OK = 0,
  RIFT_EINVAL = 1,        /* bad argument (sizes, null pointers, non-Hermitian U, ...) */
  RIFT_EWINDOW = 2,       /* Q window does not cover t-range + time of flight + taps   */
  RIFT_ENOMEM = 3,        /* device or host allocation failed                          */
  RIFT_ECUDA = 4,         /* a CUDA runtime call failed                                */
  RIFT_ETIMEOUT = 5,      /* a bounded device wait expired                             */
  RIFT_ENONFINITE = 6,    /* a NaN/Inf likelihood was produced                         */
  RIFT_ENOTCONVERGED = 7, /* max_evals reached before n_eff_target (results are valid) */
  RIFT_EUNSUPPORTED = 8   /* valid request outside what this build implements          */
} rift_status;

/* Maximum sizes accepted by rift_ile_create. */
#define RIFT_MAX_DET 4
#define RIFT_MAX_MODES 21 /* all (l, m) with 2 <= l <= 4 */

/*
 * One intrinsic point: everything Eq. (def:lnL:Decomposed) needs that does not
 * depend on the extrinsic sample (Sec. II.A, "multidimensional arrays").
 * All pointers are host pointers, read during rift_ile_create only.
 */
typedef struct {
  int n_det;                /* K, 1..RIFT_MAX_DET                                          */
  const double *det_tensor; /* [K][3][3] response tensors (symmetric), Earth-fixed frame      */
  const double *det_pos;    /* [K][3] vertex positions, metres, Earth-fixed frame             */
  int n_modes;              /* M, 1..RIFT_MAX_MODES                                          */
  const int *lm;            /* [M][2] (l, m), 2 <= l <= 4, |m| <= l, no duplicates            */
  int n_t;                  /* T, samples of each Q_{k,lm} time series (>= 4)                */
  const double *Q;          /* [K][M][T] complex: Q_{k,lm}(tau_j), tau_j = q_t0_gps[k] + j/fs */
  const double *q_t0_gps;   /* [K] GPS time of Q[k][*][0]                                    */
  double fs;                /* Q sampling rate, Hz                                           */
  const double *U;          /* [K][M][M] complex, Hermitian: U_{k,lm,l'm'} = <h_lm|h_l'm'>   */
  const double *V;          /* [K][M][M] complex, symmetric: V_{k,lm,l'm'} = <h*_lm|h_l'm'>  */
  double t_ref_gps;         /* geocentre reference time; sample t is measured from it        */
  double d_ref_mpc;         /* D_ref of Eq. (strain_mode)                                    */
  double t_lo, t_hi;        /* time prior of the point, relative to t_ref (t_lo < t_hi)       */
  int interp;               /* Q interpolation: 0 nearest, 1 linear, 3 cubic Lagrange         */
  void *cuda_stream;        /* cudaStream_t, or NULL                                         */
} rift_ile_desc;

/*
 * Create a handle for one point (Sec. II.B: Q, U, V are shipped to the device once).
 * Validates sizes, U Hermitian and V symmetric (1e-10 relative), and that the Q
 * window of every detector covers [t_lo - |x_k|/c - taps/fs, t_hi + |x_k|/c + taps/fs]
 * (else RIFT_EWINDOW).  Computes GMST(t_ref) and all per-point constants in FP64 on
 * the host (the sidereal angle is held fixed over the window, Sec. II.A).
 * On failure *out is NULL.
 */
rift_status rift_ile_create(const rift_ile_desc *desc, rift_ile **out);

/* Many points in one handle (the batched workload).  descs[i] as above; all points
 * must share n_det and the stream of descs[0] is used. */
rift_status rift_ile_batch_create(const rift_ile_desc *descs, int n_points, rift_ile **out);

void rift_ile_destroy(rift_ile *h);
const char *rift_status_str(rift_status s);
const char *rift_ile_last_error(const rift_ile *h);
int rift_ile_n_points(const rift_ile *h);

/* Forms the kernels take for point `point` of the handle, as bits of the return value (0 for a
 * null handle or a point out of range): 1 the grouped quadratic form over the 21 canonical
 * modes (Eq. (def:lnL:Decomposed) regrouped by m_b - m_a), 2 with the pairs skipped that vanish
 * when each mode lives on one sign of frequency, 4 the positive form 2 beta^H U beta of a
 * point whose modes have the reflection symmetry conj(h_a(-f)) = sigma_a h_abar(f), 8 the half
 * rows of the time quadrature (Eq. (lnL:tmarg)): Q_abar(t) = sigma_a conj(Q_a(t)) holds at every
 * sample (real data), so only the modes with m >= 0 are read.  Every form gives the same
 * likelihood up to rounding; the flags only say which one runs. */
unsigned rift_ile_forms(const rift_ile *h, int point);

/*
 * Per-sample log-likelihood, Eq. (def:lnL:Decomposed), at caller-supplied samples
 * (point 0 of the handle).  Device pointers, float32, each of length n:
 * right ascension, declination, t (geocentre, relative to t_ref), polarisation psi,
 * reference phase phi, inclination, distance D (Mpc).  lnL_out: device, length n.
 * Asynchronous on the handle's stream.  A sample whose interpolation taps leave the
 * Q window is clamped, flagged, and reported as RIFT_EWINDOW by the next call of
 * rift_ile_check().
 */
rift_status rift_ile_lnL(rift_ile *h, size_t n, const float *ra, const float *dec, const float *t,
                         const float *psi, const float *phi, const float *incl, const float *dist,
                         float *lnL_out);

/* Same with host pointers: the library copies the samples to the device, evaluates,
 * copies lnL back and synchronises.  Staging buffers are owned by the handle. */
rift_status rift_ile_lnL_host(rift_ile *h, size_t n, const float *ra, const float *dec, const float *t,
                              const float *psi, const float *phi, const float *incl, const float *dist,
                              float *lnL_out);

/*
 * Time-marginalised log-likelihood, Eq. (lnL:tmarg) (Sec. II.C: the event time is integrated
 * numerically for every draw of the other extrinsic parameters), at caller draws of
 * point 0: ln L_margT = ln (1/J) sum_j exp(lnL(theta, t_j)), midpoint rule on the sampling
 * interval of Q, t_j = t_lo + (j + 1/2)/fs, j < J = floor((t_hi - t_lo) fs), with lnL of
 * rift_ile_lnL.  Device float32 arrays of length n: ra, dec, psi, phi, incl, D (Mpc); out:
 * device, length n.  Asynchronous on the handle's stream; window and non-finite flags as for
 * rift_ile_lnL.
 */
rift_status rift_ile_lnL_tmarg(rift_ile *h, size_t n, const float *ra, const float *dec, const float *psi,
                               const float *phi, const float *incl, const float *dist, float *out);

/*
 * Frequency-domain description of one point, for forming Q, U, V of Eq. (QUV) on the device.
 * Host arrays, FP64 unless noted, copied during the call (the caller keeps ownership).
 * Frequency grid: n_f bins, bin i at f_i = nu[i] * df with integer nu[i] (negative for f < 0);
 * mirror[i] is the bin of -f_i.  weight[k][i] = 1/S_k(|f_i|) inside the band, 0 outside
 * (Eq. overlap).  Q grid: n_t samples of detector k at q_t0_gps[k] + j/fs, with fs/df an integer
 * n >= n_t.  The remaining fields are those of rift_ile_desc.
 */
typedef struct {
  int n_det;                /* K                                                      */
  const double *det_tensor; /* [K][3][3]                                              */
  const double *det_pos;    /* [K][3] metres                                          */
  int n_modes;              /* M                                                      */
  const int *lm;            /* [M][2]                                                 */
  int n_f;                  /* frequency bins                                         */
  const int *nu;            /* [n_f] f_i / df (int32)                                 */
  double df;                /* Hz                                                     */
  const double *hlm;        /* [M][n_f] complex128 h_lm(f_i) (at D_ref)               */
  const double *data;       /* [K][n_f] complex128 d_k(f_i)                           */
  const double *weight;     /* [K][n_f] band / S_k(|f_i|)                             */
  const int *mirror;        /* [n_f] bin of -f_i (int32)                              */
  int n_t;                  /* Q samples per (detector, mode)                         */
  const double *q_t0_gps;   /* [K] GPS time of Q sample 0                             */
  double fs;                /* Q sampling rate, Hz                                    */
  double t_ref_gps, d_ref_mpc, t_lo, t_hi;
  int interp;
  void *cuda_stream;
} rift_ile_fd_desc;

/*
 * Eq. (QUV) on the device (direct sums over the bins with nonzero weight; FP32 terms summed in
 * blocks of 32 into double-float totals):
 *   Q[k][m][j] = 2 df sum_i exp(2 pi i f_i tau_j) conj(h_m(f_i)) d_k(f_i) w_k(f_i),
 *                tau_j = q_t0_gps[k] - t_ref_gps + j/fs,
 *   U[k][m][m'] = 2 df sum_i conj(h_m(f_i)) h_m'(f_i) w_k(f_i),
 *   V[k][m][m'] = 2 df sum_i h_m(-f_i) h_m'(f_i) w_k(f_i).
 * Outputs: host complex128 arrays in the layouts of rift_ile_desc (Q [K][M][n_t], U, V [K][M][M]).
 * Synchronous on d->cuda_stream.  RIFT_EINVAL for inconsistent grids; detail in
 * rift_quv_last_error() (per thread).
 */
rift_status rift_quv(const rift_ile_fd_desc *d, double *Q, double *U, double *V);
const char *rift_quv_last_error(void);
/* Device time (ms, CUDA events on the call's stream) of the two kernels of the last successful
 * rift_quv call of the calling thread: out[0] the Q sums, out[1] the U and V sums (host array of 2). */
void rift_quv_kernel_ms(double out[2]);

/* rift_quv followed by rift_ile_create on the result (U made exactly Hermitian and V exactly
 * symmetric by averaging each pair of transposed elements): a handle built from frequency-domain
 * inputs. */
rift_status rift_ile_create_fd(const rift_ile_fd_desc *d, rift_ile **out);

/* Reads and clears the device status word (out-of-window taps, non-finite lnL). */
rift_status rift_ile_check(rift_ile *h);

/* Proposal kinds for rift_mc_opts.proposal. */
#define RIFT_PROPOSAL_PRIOR 0
#define RIFT_PROPOSAL_ADAPTIVE 1
#define RIFT_PROPOSAL_LEARNED 2

/*
 * Monte Carlo options (Sec. II.C: fixed n_eff threshold; Sec. III.B: adaptive
 * sampling prior regenerated from the most recent chunk).
 * Prior: ra ~ U[0,2pi), sin dec ~ U[-1,1], t ~ U[t_lo,t_hi] of the point, psi ~ U[0,pi),
 * phi ~ U[0,2pi), cos incl ~ U[-1,1], p(D) ~ D^2 on [d_lo, d_hi].
 * Uniforms: Philox4x32-10, key = (seed lo32, seed hi32), counter = (sample index,
 * round, block, point id); block b gives uniforms 4b..4b+3; u = ((x >> 9) + 1/2) 2^-23.
 */
typedef struct {
  uint64_t seed;
  uint32_t point_id;     /* counter word 3 (single-point handles); batches use the point index */
  uint32_t n_per_round;  /* samples per round (chunk)                                   */
  uint64_t max_evals;    /* stop after this many samples                                 */
  double n_eff_target;   /* stop once sum w / max w reaches this                         */
  double d_lo, d_hi;     /* distance prior bounds, Mpc                                   */
  int proposal;          /* RIFT_PROPOSAL_*                                              */
  int n_bins;            /* adaptive: bins per adapted coordinate (ra, sin dec, t), <= 256 */
  double beta;           /* adaptive: tempering exponent on the weights                 */
  double floor_eps;      /* adaptive: mixture weight of the prior in the new proposal   */
  int adapt_rounds;      /* adaptive: rebuild tables after rounds 0..adapt_rounds-1 (<0: always) */
  const float *tables;   /* adaptive: host [3][n_bins+1] float32 CDF tables of round 0, or NULL = prior */
  const void *mdn;       /* learned proposal: a rift_mdn handle (RIFT_PROPOSAL_LEARNED)  */
  float *dbg_ell;        /* optional device [max_evals]: log weight of sample (round r, i) at r*n_per_round+i */
  float *dbg_tables;     /* optional device [rounds][3][n_bins+1]: tables used in each round */
  int max_rounds;        /* optional cap on rounds (0 = none)                            */
  int timing;            /* nonzero: time every likelihood-kernel launch with CUDA events */
  int strata[3];         /* stratification of each round in (ra, sin dec, t): powers of two;
                            {0,0,0} = chosen by the library; {1,1,1} = none.  A round of n samples
                            over C = product cells puts contiguous blocks of samples in each cell
                            (cells [0, n mod C) get one more), sample i of cell (c0,c1,c2) uses the
                            uniforms (c_d + u_d)/S_d, and its log weight gains ln(n / (C n_c)).
                            Rounds with n < C are not stratified.  C <= RIFT_MAX_CELLS.        */
  const void *resume;    /* optional host RIFT_MC_STATE_BYTES blob written through `save` by an earlier
                            call on the same point with the same options (seed, point_id,
                            n_per_round, proposal, n_bins, beta, floor_eps, d_lo, d_hi, strata):
                            the run continues from it (round index, compensated accumulator,
                            adapted tables), so a run stopped after r rounds and resumed gives
                            bit for bit the result of the uninterrupted run; max_evals and
                            max_rounds count the resumed rounds too.  RIFT_EINVAL if the blob does
                            not match the handle or the options.  Single-point calls only.       */
  void *save;            /* optional host buffer of RIFT_MC_STATE_BYTES: the sampler state at return  */
  int time_marg;         /* nonzero: each draw integrates the event time by quadrature, Eq. (lnL:tmarg)
                            (rift_ile_lnL_tmarg), instead of sampling it; the draws cover (ra, dec,
                            psi, phi, incl, D), strata and adaptive tables cover (ra, sin dec) only
                            (the time table stays uniform), n_evals counts draws.  All proposals,
                            single-point calls and the batched runner; with the learned proposal
                            the mixture's time coordinate is integrated out (dropped from each
                            diagonal component) and the weight is that of the other four.        */
  int tables_per_point;  /* adaptive, with `tables`: the tables are host [n_points][3][n_bins+1], one
                            set per point (0: one set for every point).  With `tables_out` this
                            warm-starts each intrinsic point from an earlier run's integrator
                            (Sec. II.C and III.B: the adaptive integrator is reused from one intrinsic
                            point to the next).                                                  */
  float *tables_out;     /* adaptive, optional host [n_points][3][n_bins+1]: each point's proposal at
                            return -- the tables rebuilt from its last round when that round adapted
                            (adapt_rounds), else the tables that round used: the proposal its next
                            round would draw from.  RIFT_EINVAL with other proposals.            */
  double fallback_neff;  /* learned proposal: fallback to the adaptive sampler.  After a learned round
                            whose own draws have n_eff = sum w / max w (over that round alone) below
                            this value -- importance weights dominated by a few draws -- the point
                            draws its remaining rounds from the adaptive proposal (n_bins, beta,
                            floor_eps; starting from the prior's tables, unstratified like learned
                            rounds) and rebuilds it from each of them.  Every round enters the
                            estimate with its own q, so the pooled estimate stays unbiased.
                            0 = no fallback; RIFT_EINVAL with other proposals or opts.tables.    */
  int refine;            /* nonzero: the heaviest samples of each sampled-time round from the prior or
                            the adaptive proposal are evaluated again in FP64 (draw, response,
                            harmonics, interpolation, Eq. (def:lnL:Decomposed) with U, V kept in
                            FP64; Q from its FP32 copy), and the estimate uses those values.  Per
                            round: the samples within B nats of the running maximum, B the largest of
                            1..24 that keeps them at RIFT_REFINE_CAP at most (none if more than that
                            lie within one nat), taken from the two largest log weights of every warp
                            of every work item.  This removes the FP32 floor of estimates that rest
                            on a few samples (n_eff ~ 1: the heaviest sample's FP32 error).  Rounds
                            of the learned proposal and time-marginalised rounds are not refined.
                            Single-point and batched calls; RIFT_EINVAL with resume, save or the
                            allocation-free entry point.                                        */
} rift_mc_opts;

/* Samples refined per point and round at most (rift_mc_opts.refine). */
#define RIFT_REFINE_CAP 64

/* Size of the sampler-state blob of rift_mc_opts.resume / save (same library build and byte order). */
#define RIFT_MC_STATE_BYTES 8192

#define RIFT_MAX_CELLS 32768

typedef struct {
  double lnL_marg;   /* log( sum_i w_i / N ), w = L p / q                                */
  double n_eff;      /* sum w / max w                                                    */
  double n_eff_kish; /* (sum w)^2 / sum w^2                                              */
  double sigma;      /* standard error of lnL_marg                                        */
  uint64_t n_evals;  /* likelihood evaluations used                                       */
  int rounds;
  int status;        /* rift_status of this point                                          */
  double acc_max, acc_s1, acc_s2; /* mergeable state: max l, sum e^{l-max}, sum e^{2(l-max)} */
  double kernel_ms;  /* with opts.timing: summed duration of the likelihood-kernel launches */
  int kernel_launches; /* likelihood + reduction + adaptive kernels launched by this call   */
  int strata[3];     /* strata used for rounds with n >= C                                     */
  int fallback_round; /* learned proposal with fallback_neff: the first round drawn from the adaptive
                         proposal, -1 if the point never fell back                                 */
  int n_refined;      /* opts.refine: samples evaluated again in FP64 over the call               */
} rift_mc_result;

/*
 * Marginalised likelihood of point 0, Eq. (lnLmarg), by rounds of n_per_round
 * samples drawn on the device, until n_eff >= n_eff_target or max_evals.
 * Returns RIFT_ENOTCONVERGED (with a valid *res) if max_evals was reached first.
 * Synchronises the handle's stream.
 */
rift_status rift_ile_marginalize(rift_ile *h, const rift_mc_opts *opts, rift_mc_result *res);

/*
 * Batched marginalisation of every point of a batch handle in one persistent launch
 * per round group, replayed as a CUDA graph.  res: host array of n_points.
 * Per point the same estimator and stopping rule as rift_ile_marginalize; the uniforms
 * of point i use counter word 3 = i.
 */
rift_status rift_ile_batch_marginalize(rift_ile *h, const rift_mc_opts *opts, rift_mc_result *res);

/*
 * Learned proposal (a mixture-density network over ra, sin dec, t, cos incl, ln D, conditioned
 * on a 64-feature summary of each point's Q time series; defensive mixture with the prior).
 * With opts.proposal = RIFT_PROPOSAL_LEARNED, rift_ile_marginalize and
 * rift_ile_batch_marginalize sample every point from its learned proposal: from opts.mdn (the
 * network is evaluated on the device on each point's summary) or, when opts.mdn is NULL, from
 * the network heads last given by rift_ile_set_proposal_head.  Learned rounds are not stratified.
 */
typedef struct rift_mdn rift_mdn;
#define RIFT_MDN_PARAMS 105048   /* W1[256][64] b1[256] W2[256][256] b2[256] W3[88][256] b3[88] */
#define RIFT_MDN_SUMMARY 64
#define RIFT_MDN_HEAD 88         /* 8 logits, 8x5 means, 8x5 log sigmas (clamped to [-8, 4])     */

/* New network: weights uniform(-1,1) sqrt(3/fan_in) from Philox4x32-10 (key = seed), zero biases. */
rift_status rift_mdn_create(uint64_t seed, rift_mdn **out);
void rift_mdn_destroy(rift_mdn *m);
const char *rift_mdn_last_error(const rift_mdn *m);
/* Parameters in the layout above: host float32 [RIFT_MDN_PARAMS]; set resets Adam's state.
 * get: which = 0 the float32 master copy, 1 the bfloat16 weights the kernels use. */
rift_status rift_mdn_set_params(rift_mdn *m, const float *host);
rift_status rift_mdn_get_params(rift_mdn *m, float *host, int which);
/* head_dev[n][88] = network(summ_dev[n][64]) (device pointers; the device's default stream).
 * The three layers run on the tensor cores (tcgen05 BF16 products, FP32 accumulators in tensor
 * memory), 128 points per CTA; each layer's FP32 input is split into two BF16 terms, so inputs
 * keep about 16 significant bits and the weights are exactly their BF16 values.  Synchronises the
 * device; RIFT_ETIMEOUT if a bounded wait for the tensor core expired. */
rift_status rift_mdn_forward(rift_mdn *m, int n, const float *summ_dev, float *head_dev);
/* Device time (ms, CUDA events around the kernel) of the last rift_mdn_forward of this thread. */
double rift_mdn_forward_ms(void);
/* Mean over the n points of the weighted negative log likelihood
 *   -sum_j w[p][j] ln q_MDN(theta[p][j] | summ[p]),
 * theta_dev [n][H][5] = (ra, sin dec, t, cos incl, ln D), w_dev [n][H], box_dev [n][2][5] the
 * lower and upper bounds of the five coordinates; *loss_out and the weight gradient (host
 * [RIFT_MDN_PARAMS], may be NULL). */
rift_status rift_mdn_loss_grad(rift_mdn *m, int n, const float *summ_dev, const float *theta_dev, const float *w_dev,
                               int H, const float *box_dev, double *loss_out, float *grad_host);
/* `steps` Adam steps (lr; beta1 0.9, beta2 0.999, eps 1e-8) of the same loss on minibatches of
 * `batch` consecutive points (cycling); loss_per_step: host [steps] or NULL. */
rift_status rift_mdn_train(rift_mdn *m, int n, const float *summ_dev, const float *theta_dev, const float *w_dev,
                           int H, const float *box_dev, int steps, int batch, double lr, double *loss_per_step);
/* Summary features of every point of the handle: out_dev [n_points][64] (device). */
rift_status rift_ile_batch_summary(rift_ile *h, float *out_dev);
/* Learned proposal of every point from given network heads (host [n_points][88]). */
rift_status rift_ile_set_proposal_head(rift_ile *h, const float *head_host);
/* Boxes of the five learned coordinates of every point for distance prior [d_lo, d_hi]:
 * host out [n_points][2][5]. */
rift_status rift_ile_boxes(rift_ile *h, double d_lo, double d_hi, float *out_host);
/* Training samples: runs rift_ile_batch_marginalize with opts, then draws H samples of each
 * point's last round by systematic resampling with probabilities ~ exp(beta (l - max l)),
 * writing theta_dev [n_points][H][5] (ra, sin dec, t, cos incl, ln D); res as the batch call. */
rift_status rift_ile_batch_harvest(rift_ile *h, const rift_mc_opts *opts, int H, double beta, float *theta_dev,
                                   rift_mc_result *res);

/*
 * Extrinsic posterior samples (Eq. (lnLmarg) read as a posterior: the importance-sampled draws
 * theta_i ~ q of a marginalisation, weighted by w_i = L_i p_i / q_i, are samples of the
 * extrinsic posterior at the intrinsic point; Sec. VI: the same integration yields the
 * extrinsic distributions).  Both calls run the marginalisation of rift_ile_batch_marginalize
 * with `opts` (every point of the handle; a single-point handle is a batch of one; res
 * [n_points] as there; RIFT_ENOTCONVERGED is returned with the samples written) and then read
 * the draws of each point's LAST round.  Every column is float32:
 *   0 ra (rad)   1 dec (rad)   2 t (s from t_ref, geocentre)   3 psi   4 phi   5 incl (rad)
 *   6 D (Mpc)    7 lnL (Eq. (def:lnL:Decomposed); with time_marg, as described per call)
 *   8 ln p - ln q (rift_ile_samples only; includes the stratification factor ln(n / (C n_c)))
 * so that the weight of an exported draw is exp(lnL + ln p - ln q).  lnL is the draw's log
 * weight minus ln p - ln q, both as the sampler computed them in FP32.
 * Errors: RIFT_EINVAL for NULL or inconsistent arguments, the statuses of the marginalisation.
 */
#define RIFT_SAMPLE_COLS 9
#define RIFT_POSTERIOR_COLS 8

/* Weighted export: out_dev [n_points][cap][RIFT_SAMPLE_COLS] (device, caller-owned) receives the
 * first min(n_p, cap) draws of point p's last round in draw order, NaN rows after them;
 * n_out [n_points] (host) receives n_p, the number of draws of that round.  cap may be 0 (counts
 * only; out_dev may then be NULL).  With time_marg, column 2 is NaN (the time was integrated
 * out) and column 7 is the time-marginalised lnL of Eq. (lnL:tmarg). */
rift_status rift_ile_samples(rift_ile *h, const rift_mc_opts *opts, size_t cap, float *out_dev, uint64_t *n_out,
                             rift_mc_result *res);

/* H equal-weight posterior samples per point: systematic resampling of the last round, slot h
 * taking the first draw i with C_i > (h + 1/2) C_{n-1} / H, C the cumulative sums (FP64) of
 * exp(l_i - max l).  out_dev [n_points][H][RIFT_POSTERIOR_COLS] (device); idx_dev [n_points][H]
 * (device, may be NULL) receives the resampled draw (its row in rift_ile_samples), -1 for a point
 * without draws (its rows are NaN).  With time_marg, each resampled draw then gets its event time
 * from the conditional on the quadrature grid of Eq. (lnL:tmarg), P(t_j | rest) proportional to
 * L(t_j), t_j = t_lo + (j + 1/2)/fs: the first j whose cumulative probability exceeds u, u the
 * uniform of Philox block 3 of counter (h, 0, point word: opts.point_id for a single-point handle,
 * the point index in a batch) (the sampler uses blocks 0-2); column 7 is
 * then lnL(t_j).  A non-finite likelihood there gives RIFT_ENONFINITE, taps outside the Q window
 * RIFT_EWINDOW. */
rift_status rift_ile_posterior(rift_ile *h, const rift_mc_opts *opts, int H, float *out_dev, int *idx_dev,
                               rift_mc_result *res);

/*
 * Device and pinned host buffers of handles are kept in a process-wide cache when a handle is
 * destroyed and reused by later handles of the same sizes (a handle per intrinsic point then costs
 * no device allocation).  rift_release_cached_memory gives every cached buffer back to CUDA (the
 * cache also does so by itself when an allocation fails for lack of memory).  Buffers in use by live
 * handles are not affected.  Call it before cudaDeviceReset (which invalidates cached buffers) and
 * before handing the memory to another allocator.
 */
void rift_release_cached_memory(void);

/*
 * Counters of the buffer cache since the library was loaded (host array of 4, written):
 * out[0] device-buffer requests, out[1] pinned-host-buffer requests (served from the cache or by
 * a new allocation), out[2] cudaMalloc calls, out[3] cudaMallocHost calls those requests needed.
 * Tracing only: a call that leaves all four unchanged made no handle allocation.
 */
void rift_cache_counters(unsigned long long out[4]);

/*
 * rift_ile_marginalize_static -- the same computation as rift_ile_marginalize (point 0,
 * prior or adaptive proposal, sampled or marginalised time; same kernels, same results) for callers that cannot
 * allocate device memory when they marginalise: programs that give (nearly) all device
 * memory to another allocator at start-up, or that forbid device allocation after
 * initialisation.  The paper has no counterpart; it is a deployment variant.
 *
 *  - Allocates nothing: no cudaMalloc/cudaFree, no library allocation.  Its scratch (block
 *    partials, accumulator, adaptive histograms, tables, one round of per-sample weights)
 *    is a file-scope device array of RIFT_STATIC_SCRATCH_BYTES that every device which
 *    loads the library holds until the process exits.
 *  - Every call looks that array's device address up (cudaGetSymbolAddress, with the
 *    caller's device current), so the address stays right after cudaDeviceReset.  The first
 *    call on a device is the set-up: the lookup may load the library's device code there;
 *    make this first call before any stream capture.
 *  - Limits: n_per_round <= RIFT_STATIC_MAX_PRIOR_ROUND (time-marginalised rounds, whose work
 *    items hold fewer draws: RIFT_STATIC_MAX_PRIOR_ROUND / 8), and with the adaptive proposal
 *    n_per_round <= RIFT_STATIC_MAX_ROUND; larger rounds are rejected with RIFT_EINVAL.
 *    The learned proposal (whose network buffers a handle allocates on first use) is rejected
 *    with RIFT_EINVAL.  opts->dbg_tables and opts->timing must be 0.
 *  - Every call on a device shares the array and resets what must start from zero; calls
 *    whose GPU work overlaps (different streams or host threads) race and must not be issued.
 * The handle itself is created (and allocated) beforehand with rift_ile_create.
 */
#define RIFT_STATIC_MAX_ROUND 131072
#define RIFT_STATIC_MAX_PRIOR_ROUND 67108864
#define RIFT_STATIC_SCRATCH_BYTES 3552512
rift_status rift_ile_marginalize_static(rift_ile *h, const rift_mc_opts *opts, rift_mc_result *res);

/*
 * Detector-frame description of sources, for building physical injections (Sec. II.A: the
 * response F_k = F_+ - i F_x of detector k to a source at (ra, dec, psi), its arrival time
 * t_k = t + delay_k, delay_k = -(x_k . n)/c, and the harmonics -2Y_lm(incl, phi)): for source s
 * and detector k
 *   coef[s][k][a] = (D_ref / D) conj(F_k) Y_{l_a m_a}(incl, phi),   tk[s][k] = t + delay_k,
 * so that the source's strain in detector k is Re sum_a coef[s][k][a] h_a(t - tk[s][k]) (times
 * relative to t_ref_gps, at which GMST is taken).  Evaluated on the device with the likelihood
 * kernels' own response, time-of-flight and harmonic arithmetic (FP32, times in double-float).
 * Host arrays: det_tensor [K][3][3], det_pos [K][3] (m), lm [M][2]; src [n][7] float64 rows
 * (ra, dec, t, psi, phi, incl, D in Mpc, D > 0); outputs coef [n][K][M] complex128 (modes in the
 * caller's order) and tk [n][K] float64.  Synchronous on the legacy default stream; temporary
 * device buffers are allocated and freed inside.  RIFT_EINVAL for bad sizes, modes or values.
 */
rift_status rift_source_frame(int n_det, const double *det_tensor, const double *det_pos, int n_modes,
                              const int *lm, double t_ref_gps, double d_ref_mpc, size_t n, const double *src,
                              double *coef, double *tk);

/*
 * Launch shape of the Monte Carlo kernels: samples per stratification cell (sets the strata
 * when opts.strata is {0,0,0}) and the shared-memory split (each cell-kernel CTA stages Q
 * windows in the SM's shared memory / smem_split, less its fixed part; how many CTAs are
 * resident is set by registers and shared memory).  rift_ile_autotune times every candidate
 * on the handle's own workload (opts as for the marginalisation; each candidate runs `reps`
 * rounds of n_per_round samples per point), keeps the fastest in the handle and returns it.
 * The choice changes which cells samples fall in (a different but equally valid
 * stratification), not how a sample is evaluated.
 */
typedef struct {
  int cell_samples;  /* target samples per cell, in [64, 65536] (default 640 -> cells of 512..1280) */
  int smem_split;    /* 1..8 (default 3)                                                            */
  double ms;         /* rift_ile_autotune: time of the chosen shape per round (output)              */
} rift_tune;
rift_status rift_ile_get_tune(const rift_ile *h, rift_tune *out);
rift_status rift_ile_set_tune(rift_ile *h, const rift_tune *t);
rift_status rift_ile_autotune(rift_ile *h, const rift_mc_opts *opts, int reps, rift_tune *best);

/*
 * Draw the samples of one round (prior or tables) without evaluating them: theta_out is
 * device [7][n] float32 rows (ra, sin dec, t, psi, phi, cos incl, D); lpq_out device [n]
 * (ln p - ln q), bins_out device [3][n] int32 or NULL.  tables: device [3][n_bins+1] or NULL.
 */
rift_status rift_ile_draw(rift_ile *h, const rift_mc_opts *opts, uint32_t round, const float *tables,
                          size_t n, float *theta_out, float *lpq_out, int *bins_out);

#ifdef __cplusplus
}
#endif
#endif /* RIFT_ILE_H */
