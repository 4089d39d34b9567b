"""The FP64 oracle over many samples of one workload point, on all host cores (test helper).

Worker processes are started with the spawn method (never forked from a process that holds a
CUDA context), each builds the point once from its workload spec and seed, and evaluates
chunks of one round's draws: the round's log-sum-exp state over a range of sample indices, or
per-sample log weights and template norms <h|h> at given indices.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

_PT = None


def _init(spec_name, point_seed):
    global _PT
    import workload as W
    _PT = W.make_point(getattr(W, spec_name)(), point_seed)


def _accum_range(args):
    a, b, seed, S, n = args
    from oracle import mc
    pr = mc.Prior(_PT["t_lo"], _PT["t_hi"])
    th, _, lq = mc.draw(seed, 0, 0, np.arange(a, b, dtype=np.uint64), pr, None, S, n)
    acc = mc.Accum.of(mc.lnL_samples(_PT, th) + lq)
    return acc.m, acc.s1, acc.s2, acc.n


def _samples(args):
    idx, seed, S, n = args
    from oracle import mc
    pr = mc.Prior(_PT["t_lo"], _PT["t_hi"])
    th, _, lq = mc.draw(seed, 0, 0, idx, pr, None, S, n)
    ell = mc.lnL_samples(_PT, th) + lq
    silent = dict(_PT, Q=np.zeros_like(_PT["Q"]))
    hh = -2.0 * mc.lnL_samples(silent, th)
    return ell, hh


class OraclePool:
    def __init__(self, spec_name, point_seed):
        self.cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_init, initargs=(spec_name, point_seed))

    def accum(self, seed, S, n):
        """Oracle log-sum-exp state (max, s1, s2, count) of a whole prior round of n samples."""
        from oracle import mc
        edges = np.linspace(0, n, 8 * self.cores + 1).astype(np.int64)
        parts = self.pool.map(_accum_range, [(int(edges[i]), int(edges[i + 1]), seed, tuple(S), n)
                                             for i in range(len(edges) - 1)])
        acc = mc.Accum()
        for m, s1, s2, c in parts:
            acc = acc.merge(mc.Accum(m, s1, s2, c))
        return acc

    def samples(self, idx, seed, S, n):
        """Oracle log weights and <h|h> at sample indices idx of a prior round of n samples."""
        chunks = np.array_split(np.asarray(idx, dtype=np.uint64), 8 * self.cores)
        out = self.pool.map(_samples, [(c, seed, tuple(S), n) for c in chunks if c.size])
        return np.concatenate([o[0] for o in out]), np.concatenate([o[1] for o in out])

    def close(self):
        self.pool.close()
        self.pool.join()
