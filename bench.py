"""Benchmark: extrinsic lnL evaluations per second and lnL_marg per second on one GB300.

Workload (N = 1): the full-size plain ILE point -- 3 detectors (H1/L1/V1), all 21
modes with 2 <= l <= 4, Q over +-0.1 s at 16384 Hz, SNR 30 -- marginalised over
1e7 prior samples drawn on the device.  One step = one rift_ile_marginalize call
(Philox draw, response, harmonics, Q gather/interpolation, quadratic forms,
log-sum-exp, FP64 refinement of the heaviest samples, stopping rule) with Q/U/V
already resident on the device.

Under torchrun (N > 1) every rank marginalises its own point (independent points:
weak scaling, no data-path collective); the barrier and the max over ranks use
torch.distributed.  --impl reference times the FP64 oracle on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

N_SAMPLES = 10_000_000
WORKLOAD = "plain ILE full size: K=3 (H1,L1,V1), M=21 (2<=l<=4), Q +-0.1 s @ 16384 Hz (T=3277), SNR 30, N=1e7"


def flops_per_sample(K: int, M: int, taps: int) -> int:
    """Algorithmic FP32 flops of one likelihood evaluation (FMA = 2), the count the roofline
    fraction is reported on: response and time of flight 60 + 36 K; the harmonics 14 M; the Q
    term K M (6 + 4 taps + 2) + 4 taps K (tap weights and gather, conj(F Y) Q); the U forms
    3 M(M+1)/2 (products conj(Y_a) Y_b shared by the detectors) + 4 K M(M+1)/2; the V forms
    3 M(M+1)/2 + 8 K M(M+1)/2; combine, log weight and log-sum-exp 40.  11,764 at K = 3, M = 21,
    4 taps."""
    npair = M * (M + 1) // 2
    return (60 + 36 * K) + 14 * M + (K * M * (6 + 4 * taps + 2) + 4 * taps * K) + (3 * npair + 4 * K * npair) \
        + (3 * npair + 8 * K * npair) + 40


def pair_form_flops_per_sample(K: int, M: int, taps: int) -> int:
    """A recount of the same arithmetic as the pair-form kernel code does it (FMA = 2): per pair
    a <= b the products conj(ya) yb and ya yb (12), per detector Re(P U) (4) and R V (8); the
    linear term per (k, lm) F conj(Y) (6) and per tap Re(c q) + weight (5); harmonics ~14 M;
    response + delay ~60 + 40 K; transforms, combine and log-sum-exp ~60."""
    npair = M * (M + 1) // 2
    quad = npair * (12 + 12 * K) + 10 * K
    lin = K * M * (6 + 5 * taps) + 8 * K
    return quad + lin + 14 * M + 60 + 40 * K + 60


def mirror_quad_flops(K: int) -> int:
    """Flops the cell kernel executes for the quadratic form of a mirror-symmetric point with all
    21 (l <= 4) modes (the positive form over the 78 pairs of modes with m >= 0): per pair the
    products p_a p_b, q_a q_b (2) and p_a q_b - q_a p_b (3, off-diagonal), per detector 2, 3 or 6
    FMAs (diagonal, same m, other); per group and detector the combination (5 for D = 0, else 13);
    p, q of the 12 modes (6 each) and |F| products (3 per detector)."""
    ms = [m for l in (2, 3, 4) for m in range(-l, l + 1)]
    P = [j for j in range(21) if ms[j] >= 0]
    fl, groups = 0, set()
    for ia, a in enumerate(P):
        for b in P[ia:]:
            D = ms[b] - ms[a]
            groups.add(D)
            fl += (2 + 4 * K) if a == b else ((5 + 6 * K) if D == 0 else (5 + 12 * K))
    return fl + K * (5 + 13 * (len(groups) - 1)) + 12 * 6 + 3 * K


def executed_flops_per_sample(K: int, M: int, taps: int) -> int:
    """pair_form_flops_per_sample with the pair-form quadratic forms replaced by the positive
    form the cell kernel runs for the benchmark's point."""
    npair = M * (M + 1) // 2
    return pair_form_flops_per_sample(K, M, taps) - (npair * (12 + 12 * K) + 10 * K) + mirror_quad_flops(K)


def mdn_forward_mma_flops(P: int) -> int:
    """Flops of the network's three matrix products for P points (FMA = 2)."""
    return P * 2 * (64 * 256 + 256 * 256 + 256 * 88)


def fp32_peak_tflops(sms: int, mhz: float) -> float:
    """FP32 FMA issue peak: 128 lanes per SM x 2 flop per FMA x SMs x SM clock."""
    return 2 * 128 * sms * mhz * 1e6 / 1e12


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        return json.loads(p.read_text())
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)   # first sample in hand: the sampler is running when timing starts
            self.lines.clear()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        import torch
        if torch.cuda.is_available():
            dist.barrier(device_ids=[torch.cuda.current_device()])
        else:
            dist.barrier()


def max_over_ranks(world, x: float) -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda") if (torch.cuda.is_available() and dist.get_backend() == "nccl") else torch.device("cpu")
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def recorded_traffic():
    """DRAM bytes per launch of the likelihood kernel from the committed ncu record, or None once
    the kernel sources no longer hash to the recorded value (the counters describe older code)."""
    import hashlib
    rec = ROOT / "profiles" / "cells_kernel_traffic.txt"
    src = ROOT / "paper_1902_04934_gb300" / "csrc"
    try:
        kv = dict(l.strip().split("=", 1) for l in rec.read_text().splitlines() if "=" in l and not l.startswith("#"))
        h = hashlib.sha256(b"".join((src / f).read_bytes() for f in ("mc.cu", "draw.cuh", "rift_device.cuh", "rift_internal.h")))
    except OSError:
        return None
    # the Q arena is read about once per launch whatever the sample count, so the figure is
    # only reported for the launch size it was measured on
    if h.hexdigest()[:16] != kv.get("source_sha256") or int(kv["samples_per_launch"]) != N_SAMPLES:
        return None
    return int(kv["dram_bytes_per_launch"])


def whole_job(world: int, local_ms: float, steps: int, units_per_rank: int):
    """Whole-job time per step (the slowest rank) and throughput over all ranks' units."""
    ms_per_step = max_over_ranks(world, local_ms) / steps
    return ms_per_step, units_per_rank * world / (ms_per_step * 1e-3)


def point_seed(rank: int) -> int:
    """Rank r marginalises its own independent point (weak scaling over points)."""
    return 2 + 1000 * rank


# ---------------------------------------------------------------- CPU oracle leg
_ORACLE_PT = None


def _oracle_init():
    global _ORACLE_PT
    import workload as W
    _ORACLE_PT = W.make_point(W.cfg_full(), 2)


def _oracle_chunk(args):
    """One chunk of the oracle's plain marginalisation: draw, FP64 lnL, log-sum-exp state."""
    seed, start, n = args
    import numpy as np
    from oracle import mc
    pt = _ORACLE_PT
    pr = mc.Prior(pt["t_lo"], pt["t_hi"])
    t0 = time.perf_counter()
    th, _, lpq = mc.draw(seed, 0, 0, np.arange(start, start + n, dtype=np.uint64), pr)
    ell = mc.lnL_samples(pt, th) + lpq
    acc = mc.Accum.of(ell)
    return time.perf_counter() - t0, n, (acc.m, acc.s1, acc.s2, acc.n)


class OraclePool:
    """The FP64 oracle on the host cores: one spawned worker process per core (single-threaded
    numerics), each holding the full-size point; timed on bounded samples of the same workload."""

    def __init__(self, cores=None):
        import multiprocessing as mp
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[var] = "1"
        all_cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
        self.cores = cores or all_cores
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_init)
        cal = self.pool.map(_oracle_chunk, [(31, i * 2000, 2000) for i in range(self.cores)])
        self.per_sample = max(c[0] / c[1] for c in cal)

    def run(self, target_s: float, start: int = 0):
        chunk = 20000 if target_s >= 2.0 else 5000
        n_chunks = max(self.cores, int(target_s / (self.per_sample * chunk)) * self.cores)
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_chunk, [(31, start + i * chunk, chunk) for i in range(n_chunks)])
        wall = time.perf_counter() - t0
        n = sum(r[1] for r in res)
        return n / wall, n, wall

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_oracle_throughput(target_s: float = 12.0, single_s: float = 4.0):
    """The oracle on every host core, then on one core (one worker process)."""
    op = OraclePool()
    v, n, wall = op.run(target_s)
    op.close()
    one = OraclePool(cores=1)
    v1, n1, wall1 = one.run(single_s)
    one.close()
    return {"value": v, "unit": "evals/s", "cores": op.cores, "kind": "oracle",
            "sample": f"{n} prior samples of the full-size point (indices 0..{n - 1}, seed 31)",
            "wall_s": round(wall, 2),
            "single_core": {"value": v1, "unit": "evals/s", "cores": 1,
                            "sample": f"{n1} prior samples of the same round (indices 0..{n1 - 1})",
                            "wall_s": round(wall1, 2)}}


def _oracle_round(args):
    """The oracle's log-sum-exp state over samples [a, b) of a stratified round of n samples."""
    seed, S, n, a, b = args
    import numpy as np
    from oracle import mc
    pt = _ORACLE_PT
    th, _, lq = mc.draw(seed, 0, 0, np.arange(a, b, dtype=np.uint64), mc.Prior(pt["t_lo"], pt["t_hi"]), None, S, n)
    acc = mc.Accum.of(mc.lnL_samples(pt, th) + lq)
    return acc.m, acc.s1, acc.s2, acc.n


def precision_check(rift, pt, opts, tune):
    """The benchmark's own launch (same point, seed and launch shape) against the FP64 oracle on the
    host: lnL_marg of the whole round (the oracle evaluates every sample, on all host cores), and
    per-sample lnL on 20000 random draws and the 1000 of highest weight with the tolerance of the
    parity tests, 1e-3 max(1, <h|h>/900)."""
    import numpy as np
    import torch
    from oracle import likelihood as OL
    from oracle import mc
    h = rift.rift_ile_create(pt)
    rift.rift_ile_set_tune(h, cell_samples=tune["cell_samples"], smem_split=tune["smem_split"])
    n = opts["n_per_round"]
    dbg = torch.empty(n, dtype=torch.float32, device="cuda")
    res = rift.rift_ile_marginalize(h, dbg_ell=dbg, **opts)
    plain = rift.rift_ile_marginalize(h, **dict(opts, refine=0))   # the same round, FP32 only
    rift.rift_ile_destroy(h)
    got = dbg.cpu().numpy().astype(np.float64)
    del dbg
    S = tuple(res["strata"])
    op = OraclePool()
    t0 = time.perf_counter()
    edges = np.linspace(0, n, 8 * op.cores + 1).astype(np.int64)
    parts = op.pool.map(_oracle_round, [(opts["seed"], S, n, int(edges[i]), int(edges[i + 1]))
                                        for i in range(len(edges) - 1)])
    op.close()
    acc = mc.Accum()
    for m, s1, s2, c in parts:
        acc = acc.merge(mc.Accum(m, s1, s2, c))
    ref = acc.result()
    t_full = time.perf_counter() - t0
    top = np.argsort(got)[-1000:]
    r = np.random.default_rng(7)
    idx = np.unique(np.concatenate([top, r.integers(0, n, 20000)])).astype(np.uint64)
    th, _, lq = mc.draw(opts["seed"], 0, 0, idx, mc.Prior(pt["t_lo"], pt["t_hi"]), None, S, n)
    want = mc.lnL_samples(pt, th) + lq
    th64 = dict(ra=th["ra"], dec=np.arcsin(th["sindec"]), t=th["t"], psi=th["psi"], phi=th["phi"],
                incl=np.arccos(th["cosi"]), dist=th["dist"])
    hh = -2.0 * OL.lnL_factorised(dict(pt, Q=np.zeros_like(pt["Q"])), **th64)
    tol = 1e-3 * np.maximum(1.0, hh / 900.0)
    err = np.abs(got[idx.astype(np.int64)] - want)
    le30 = hh <= 900.0
    return {"samples": int(idx.size), "max_err_over_tol": float((err / tol).max()),
            "mean_err_over_tol": float((err / tol).mean()),
            "max_abs_dlnL_template_snr_le_30": float(err[le30].max()) if le30.any() else None,
            "dlnL_marg": float(res["lnL_marg"] - ref[0]), "refined_samples": res["n_refined"],
            "dlnL_marg_fp32_only": float(plain["lnL_marg"] - ref[0]),
            "lnL_marg_oracle": ref[0], "n_eff_oracle": ref[1],
            "oracle_full_round_s": round(t_full, 2), "oracle_samples": int(acc.n),
            "tolerance": "per sample 1e-3 max(1, <h|h>/900) (1e-3 absolute at template SNR <= 30); lnL_marg "
                         "1e-4; FP64 oracle on the same draws"}


# ---------------------------------------------------------------- GPU leg
def run_gpu(args, world, rank, local):
    import numpy as np
    import torch

    import __graft_entry__ as g
    g.build()
    import paper_1902_04934_gb300 as rift
    import workload as W

    torch.cuda.set_device(local)
    pt = W.make_point(W.cfg_full(), point_seed(rank))
    K, M, T = pt["Q"].shape
    h = rift.rift_ile_create(pt)
    # refine: the heaviest samples of the round are evaluated again in FP64 (the round's estimate rests
    # on about one sample, whose FP32 error would otherwise be the estimate's)
    opts = dict(seed=1234 + rank, n_per_round=N_SAMPLES, max_evals=N_SAMPLES, refine=1)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # > 129 MB L2
    # launch shape from the autotuner (cached per device and workload shape; untimed)
    dev_name = torch.cuda.get_device_name(local).replace(" ", "_")
    if args.no_tune:
        tune = dict(rift.rift_ile_get_tune(h), cached=None)
    else:
        tune = rift.autotune_cached(h, f"{dev_name}|K{K}M{M}T{T}|n{N_SAMPLES}|prior", reps=1, **opts)

    for _ in range(args.warmup):
        rift.rift_ile_marginalize(h, **opts)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    step_ms, kern_ms, launches = [], [], 0
    results = []
    barrier(world)
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    for s in range(args.steps):
        flush.zero_()                      # L2 flushed between timed steps (not timed)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        r = rift.rift_ile_marginalize(h, timing=1, **opts)
        e1.record()
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        kern_ms.append(r["kernel_ms"])
        launches += r["kernel_launches"]
        results.append(r)
    torch.cuda.synchronize()
    barrier(world)
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()

    ms_per_step, value = whole_job(world, sum(step_ms), args.steps, N_SAMPLES)
    evals = N_SAMPLES * world

    # roofline of the likelihood kernel (FP32 ALU bound)
    taps = 4
    kmean = statistics.mean(kern_ms)
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    # the SM clock sampled under load; without a sample (a very short timed region) the maximum clock,
    # which gives the lower, conservative fraction
    mp_ = measured_peaks() or {}
    f_mhz = clk["sm_mhz"] or clk.get("sm_max_mhz") or mp_.get("sm_max_mhz") or 2070.0
    f_basis = "median SM clock sampled during the run" if clk["sm_mhz"] else "maximum SM clock (no clock sample)"
    peak = fp32_peak_tflops(sms, f_mhz)
    achieved = flops_per_sample(K, M, taps) * N_SAMPLES / (kmean * 1e-3) / 1e12

    # end to end through the public API with host buffers: create (host Q/U/V -> device)
    # + marginalise + result back, every step
    # the same step without the FP64 refinement of the heaviest samples (the bulk and those samples
    # both in FP32): its time is the cost of the refinement
    fp32_only = None
    if opts.get("refine"):
        pl = []
        for _ in range(5):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            rift.rift_ile_marginalize(h, **dict(opts, refine=0))
            e1.record()
            e1.synchronize()
            pl.append(e0.elapsed_time(e1))
        fp32_only = {"ms_per_step": statistics.median(pl), "value": N_SAMPLES / (statistics.median(pl) * 1e-3),
                     "unit": "evals/s", "note": "same step with refine=0 (no FP64 re-evaluation)"}

    e2e = None
    if not args.no_e2e:
        h2d = K * T * ((M + 1) // 2 * 2) * 8 + (M * (M + 1) // 2) * K * 16 + 2048
        rift.rift_ile_destroy(h)
        torch.cuda.synchronize()
        times = []
        rounds = 0
        for s in range(max(1, min(args.steps, 5))):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h2 = rift.rift_ile_create(pt)
            rift.rift_ile_set_tune(h2, tune["cell_samples"], tune["smem_split"])   # the cached launch shape
            r = rift.rift_ile_marginalize(h2, **opts)
            rift.rift_ile_destroy(h2)
            times.append(time.perf_counter() - t0)
            rounds = r["rounds"]
        e2e_s = max_over_ranks(world, statistics.mean(times))
        e2e = {"value": evals / e2e_s, "unit": "evals/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": 64 * rounds + 4,
               "includes": "rift_ile_create from host FP64 arrays + rift_ile_set_tune (cached launch shape) + "
                           "rift_ile_marginalize + result read + destroy"}

    cpu = None
    precision = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_oracle_throughput(args.cpu_seconds)
        precision = precision_check(rift, pt, opts, tune)

    extras = {}
    if rank == 0 and world == 1 and not args.no_extras:
        extras = run_extras(args, rift, W, peak)

    r0 = results[-1]
    out = {
        "metric": "extrinsic lnL evals/sec (and lnL_marg/sec) per GB300",
        "value": value,
        "unit": "evals/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 (double-float time index; f64 accumulators; the round's heaviest samples refined in f64)",
        "data": "synthetic: seeded chirp-like modes, analytic aLIGO PSD, Gaussian noise; samples drawn on device",
        "config": bench_config(world),
        "lnL_marg_per_s": world / (ms_per_step * 1e-3),
        "lnL_marg": r0["lnL_marg"], "n_eff": r0["n_eff"], "strata": list(r0["strata"]),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": recorded_traffic(),
                     "kernel": "cells_kernel_mp<3,4> (stratified cell: draw + staged Q window + likelihood with the "
                               "positive quadratic form of a mirror-symmetric point, coefficients in the parameter "
                               "bank + log-sum-exp)",
                     "kernel_ms": kmean, "flops_per_sample": flops_per_sample(K, M, taps),
                     "pair_form_flops_per_sample": pair_form_flops_per_sample(K, M, taps),
                     "pair_form_frac": pair_form_flops_per_sample(K, M, taps) * N_SAMPLES / (kmean * 1e-3) / 1e12 / peak,
                     "executed_flops_per_sample": executed_flops_per_sample(K, M, taps),
                     "executed_frac": executed_flops_per_sample(K, M, taps) * N_SAMPLES / (kmean * 1e-3) / 1e12 / peak,
                     "peak_basis": f"FP32 FMA: 128 lanes/SM x {sms} SMs x 2 flop x {f_basis} {f_mhz} MHz "
                                   "(no FP32 figure in the measured peaks)"},
        "gpu_launches": launches,
        "autotune": tune,
        "clocks": clk,
        "e2e": e2e,
        "fp32_only": fp32_only,
        "cpu_baseline": cpu,
        "precision": precision,
        "wall_s": t_wall,
    }
    out.update(extras)
    if rank == 0:
        print(json.dumps(out))
    rift.rift_ile_destroy(h)


def _make_point(args):
    import workload as W
    spec, seed, inj = args
    return W.make_point(spec, seed, injection=inj)


def make_points(specs, seed0, injections=None):
    """Generate many points on the host cores (spawned processes)."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    with mp.get_context("spawn").Pool(min(cores, 32)) as pool:
        return pool.map(_make_point, [(s, seed0 + i, None if injections is None else injections[i])
                                      for i, s in enumerate(specs)], chunksize=4)


def physical_injections(rift, W, specs, seed):
    """A physical source per point: seeded sky position, arrival time (inside the point's time
    prior), polarisation, phase and inclination, at 400 Mpc (make_point rescales the waveform to
    the point's SNR), turned into detector-frame coefficients and arrival times by the library's
    own response and harmonics (rift_source_frame)."""
    import numpy as np
    r = np.random.default_rng(np.random.SeedSequence([0x50485953, seed]))
    out = []
    for sp in specs:
        tens = np.stack([W.detector(d)[0] for d in sp.dets])
        pos = np.stack([W.detector(d)[1] for d in sp.dets])
        src = np.array([[r.uniform(0, 2 * np.pi), np.arcsin(r.uniform(-1, 1)), r.uniform(-0.3, 0.3) * sp.t_half,
                         r.uniform(0, np.pi), r.uniform(0, 2 * np.pi), np.arccos(r.uniform(-1, 1)), sp.d_inj]])
        coef, tk = rift.rift_source_frame(tens, pos, sp.modes, sp.t_ref_gps, sp.d_ref, src)
        out.append((coef[0], tk[0]))
    return out


def physical_batch(rift, W, n, seed, seed0):
    import time as _t
    t0 = _t.perf_counter()
    specs = W.batch_specs(n, seed=seed)
    for sp in specs:
        sp.seg_len = 2.0
    pts = make_points(specs, seed0, physical_injections(rift, W, specs, seed))
    return pts, _t.perf_counter() - t0


def _timed_batch(rift, h, **kw):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = rift.rift_ile_batch_marginalize(h, **kw)
    torch.cuda.synchronize()
    return res, time.perf_counter() - t0


def _sequential(rift, pts, **kw):
    """The same points marginalised one at a time (a handle each, created before timing)."""
    import torch
    hs = [rift.rift_ile_create(p) for p in pts]
    rift.rift_ile_marginalize(hs[0], point_id=0, **kw)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, hh in enumerate(hs):
        rift.rift_ile_marginalize(hh, point_id=i, **kw)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    for hh in hs:
        rift.rift_ile_destroy(hh)
    return len(pts) / dt


def run_extras(args, rift, W, peak):
    """The batched workload (physical injections into points with uneven mode counts and Q lengths,
    adaptive rounds, one graph-replayed launch sequence) against sequential per-point runs, with the
    event time sampled and marginalised; the learned proposal trained on those points and judged on
    held-out points against the adaptive sampler; the time quadrature, Q/U/V and network kernels."""
    import numpy as np
    import torch
    out = {}
    sel = set(args.extras.split(","))
    if "tmarg" in sel:
        out["time_marginalised"] = run_tmarg(rift, W, peak)
    if "quv" in sel:
        out["quv"] = run_quv(rift, W, peak)
    if "mdn" in sel:
        out["mdn"] = run_mdn(rift, peak)
    if "config45" in sel:
        out["config45"] = run_config45(args, rift, W)
    if "converge" in sel:
        out["converge"] = run_converge(args, rift, W)
    if "batched" not in sel:
        return out
    pts, gen_s = physical_batch(rift, W, args.batch_points, 5, 1000)
    hb = rift.rift_ile_batch_create(pts)
    wl = (f"{len(pts)} physical injections (seeded sky, time, polarisation, phase, inclination), 3 detectors, "
          "M U{5..21}, Q U[800,3300] @ 16384 Hz, SNR U[8,30]")
    # configured estimator: the event time sampled, adaptive (ra, sin dec, t), 1e5-sample rounds
    kw = dict(seed=3, n_per_round=100000, max_evals=args.batch_evals, n_eff_target=1000.0, proposal="adaptive",
              n_bins=100)
    rift.rift_ile_batch_marginalize(hb, **kw)          # warm-up (graph instantiation, scratch)
    res, bt = _timed_batch(rift, hb, **kw)
    seq = _sequential(rift, pts[:32], **kw)
    out["batched"] = {
        "workload": wl + f"; adaptive 1e5-sample rounds until n_eff >= 1000 or {args.batch_evals} evaluations per point",
        "points_per_s": len(pts) / bt, "evals_per_s": sum(r["n_evals"] for r in res) / bt, "seconds": bt,
        "sequential_points_per_s": seq, "speedup_vs_sequential": (len(pts) / bt) / seq,
        "points_reaching_neff_1000": int(sum(r["n_eff"] >= 1000 for r in res)),
        "median_n_eff": float(np.median([r["n_eff"] for r in res])), "generation_s": gen_s}
    # the paper's estimator: the event time integrated by quadrature, adaptive (ra, sin dec)
    kt = dict(seed=4, n_per_round=20000, max_evals=args.tmarg_draws, n_eff_target=1000.0, proposal="adaptive",
              n_bins=100, time_marg=1)
    rift.rift_ile_batch_marginalize(hb, **dict(kt, max_evals=20000))
    rt, tt = _timed_batch(rift, hb, **kt)
    seq_t = _sequential(rift, pts[:16], **kt)
    conv = [r for r in rt if r["n_eff"] >= 1000]
    out["batched_time_marginalised"] = {
        "workload": wl + f"; event time integrated by quadrature, adaptive (ra, sin dec), 2e4-draw rounds until "
                         f"n_eff >= 1000 or {args.tmarg_draws} draws per point",
        "points_per_s": len(pts) / tt, "draws_per_s": sum(r["n_evals"] for r in rt) / tt, "seconds": tt,
        "sequential_points_per_s": seq_t, "speedup_vs_sequential": (len(pts) / tt) / seq_t,
        "points_reaching_neff_1000": len(conv),
        "median_draws_to_neff_1000": float(np.median([r["n_evals"] for r in conv])) if conv else None,
        "median_n_eff": float(np.median([r["n_eff"] for r in rt]))}
    if "learned" in sel:
        out["learned"] = run_learned(args, rift, W, hb, pts, rt)
    return out


def run_converge(args, rift, W):
    """Points of the batched workload run to the stopping rule (Sec. II.C, n_eff >= 1000): the
    event time integrated by quadrature, adaptive (ra, sin dec), 1e5-draw rounds, in one batched
    launch sequence, up to --converge-draws draws per point.  Reports which points converge, the
    draws they needed, and the batch's wall time to the rule (or the cap)."""
    import numpy as np
    pts, gen_s = physical_batch(rift, W, args.converge_points, 7, 3000)
    hb = rift.rift_ile_batch_create(pts)
    kt = dict(seed=11, n_per_round=100000, max_evals=args.converge_draws, n_eff_target=1000.0,
              proposal="adaptive", n_bins=100, time_marg=1)
    rift.rift_ile_batch_marginalize(hb, **dict(kt, max_evals=100000))   # warm-up (graph, scratch)
    res, secs = _timed_batch(rift, hb, **kt)
    rift.rift_ile_destroy(hb)
    snr = [float(p["snr"]) for p in pts]
    conv = [i for i, r in enumerate(res) if r["n_eff"] >= 1000]
    return {"workload": f"{len(pts)} physical injections of the batched workload (SNR U[8,30]); event time "
                        f"integrated by quadrature, adaptive (ra, sin dec), 1e5-draw rounds until n_eff >= 1000 "
                        f"or {args.converge_draws:.0e} draws per point",
            "seconds": secs, "points_per_s_to_rule_or_cap": len(pts) / secs,
            "draws_per_s": sum(r["n_evals"] for r in res) / secs,
            "points_reaching_neff_1000": len(conv),
            "median_draws_to_neff_1000": float(np.median([res[i]["n_evals"] for i in conv])) if conv else None,
            "points": [{"snr": round(snr[i], 2), "n_eff": round(float(r["n_eff"]), 1), "draws": int(r["n_evals"]),
                        "lnL_marg": round(float(r["lnL_marg"]), 4), "sigma_lnL": round(float(r["sigma"]), 4)}
                       for i, r in enumerate(res)],
            "generation_s": gen_s}


def run_config45(args, rift, W):
    """The learned proposal at production scale (opt-in: point generation takes about a minute):
    trained on samples harvested from 4096 physical injections (SNR U[8,40]), judged on 512 held-out
    ones against the adaptive sampler, and the 4096-point sweep itself within 1e8 draws in total
    (time integrated, 2e4-draw rounds), adaptive against learned with the fallback."""
    import numpy as np
    import torch
    t0 = time.perf_counter()
    specs = W.batch_specs(4096, seed=45, snr_range=(8.0, 40.0))
    for sp in specs:
        sp.seg_len = 2.0
    pts = make_points(specs, 200000, physical_injections(rift, W, specs, 45))
    gen_s = time.perf_counter() - t0
    hb = rift.rift_ile_batch_create(pts)
    t0 = time.perf_counter()
    S = rift.rift_ile_batch_summary(hb)
    box = torch.as_tensor(rift.rift_ile_boxes(hb), device="cuda")
    H = 64
    w = torch.full((len(pts), H), 1.0 / H, device="cuda")
    m = rift.rift_mdn_create(3)
    for stage in range(3):
        hk = dict(seed=50 + stage, n_per_round=65536, max_evals=262144)
        if stage == 0:
            theta, _ = rift.rift_ile_batch_harvest(hb, H, beta=0.5, proposal="adaptive", n_bins=32, **hk)
        else:
            theta, _ = rift.rift_ile_batch_harvest(hb, H, beta=0.5, proposal="learned", mdn=m, **hk)
        rift.rift_mdn_train(m, S, theta, w, box, steps=2000, batch=256, lr=1e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    cap = int(1e8) // len(pts) // 20000 * 20000 or 20000
    kt = dict(seed=8, n_per_round=20000, max_evals=cap, n_eff_target=1000.0, n_bins=100, time_marg=1)
    ad, t_ad = _timed_batch(rift, hb, proposal="adaptive", **kt)
    le, t_le = _timed_batch(rift, hb, proposal="learned", mdn=m, fallback_neff=args.fallback_neff, **kt)
    rift.rift_ile_destroy(hb)
    held, _ = physical_batch(rift, W, 512, 46, 300000)
    hh = rift.rift_ile_batch_create(held)
    kh = dict(kt, max_evals=args.tmarg_draws)
    had, _ = _timed_batch(rift, hh, proposal="adaptive", **kh)
    hle, _ = _timed_batch(rift, hh, proposal="learned", mdn=m, fallback_neff=args.fallback_neff, **kh)
    hln, _ = _timed_batch(rift, hh, proposal="learned", mdn=m, **kh)
    rift.rift_ile_destroy(hh)
    rift.rift_mdn_destroy(m)

    def stats(rs):
        return {"median_n_eff": float(np.median([r["n_eff"] for r in rs])),
                "points_reaching_neff_1000": int(sum(r["n_eff"] >= 1000 for r in rs)),
                "points_fallen_back": int(sum(r.get("fallback_round", -1) >= 0 for r in rs))}
    return {"workload": f"4096 physical injections, SNR U[8,40], M U{{5..21}}, Q U[800,3300] @ 16384 Hz; network "
                        f"trained in {train_s:.1f} s on them (generation {gen_s:.0f} s); sweep: time integrated, "
                        f"2e4-draw rounds, at most {cap} draws per point ({cap * len(pts):.2e} in all); "
                        f"held-out: 512 injections, at most {args.tmarg_draws} draws per point",
            "sweep_adaptive": dict(stats(ad), points_per_s=len(pts) / t_ad, draws_per_s=sum(r["n_evals"] for r in ad) / t_ad),
            "sweep_learned_with_fallback": dict(stats(le), points_per_s=len(pts) / t_le,
                                                draws_per_s=sum(r["n_evals"] for r in le) / t_le),
            "heldout_adaptive": stats(had), "heldout_learned_with_fallback": stats(hle),
            "heldout_learned_without_fallback": stats(hln)}


def run_learned(args, rift, W, hb, pts, ad_train):
    """The learned proposal: trained on samples harvested from the batch's points (the adaptive
    sampler first, then its own proposal), then run on held-out physical points with the event time
    integrated, against the adaptive sampler (its fallback and judge) at the same budget."""
    import numpy as np
    import torch
    t0 = time.perf_counter()
    S = rift.rift_ile_batch_summary(hb)
    box = torch.as_tensor(rift.rift_ile_boxes(hb), device="cuda")
    H = 64
    w = torch.full((len(pts), H), 1.0 / H, device="cuda")
    m = rift.rift_mdn_create(3)
    for stage in range(3):
        hk = dict(seed=50 + stage, n_per_round=65536, max_evals=262144)
        if stage == 0:
            theta, _ = rift.rift_ile_batch_harvest(hb, H, beta=0.5, proposal="adaptive", n_bins=32, **hk)
        else:
            theta, _ = rift.rift_ile_batch_harvest(hb, H, beta=0.5, proposal="learned", mdn=m, **hk)
        rift.rift_mdn_train(m, S, theta, w, box, steps=800, batch=min(256, len(pts)), lr=1e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    held, _ = physical_batch(rift, W, args.heldout_points, 6, 90000)
    hh = rift.rift_ile_batch_create(held)
    kt = dict(seed=8, n_per_round=20000, max_evals=args.tmarg_draws, n_eff_target=1000.0, n_bins=100, time_marg=1)
    ad, t_ad = _timed_batch(rift, hh, proposal="adaptive", **kt)
    le, t_le = _timed_batch(rift, hh, proposal="learned", mdn=m, fallback_neff=args.fallback_neff, **kt)
    ln, _ = _timed_batch(rift, hh, proposal="learned", mdn=m, **kt)
    rift.rift_ile_destroy(hh)
    rift.rift_mdn_destroy(m)

    def stats(rs):
        return {"median_n_eff": float(np.median([r["n_eff"] for r in rs])),
                "points_reaching_neff_1000": int(sum(r["n_eff"] >= 1000 for r in rs)),
                "median_draws_per_point": float(np.median([r["n_evals"] for r in rs]))}
    good = [i for i in range(len(held)) if ad[i]["n_eff"] >= 100 and le[i]["n_eff"] >= 100]
    dl = np.array([abs(le[i]["lnL_marg"] - ad[i]["lnL_marg"]) for i in good])
    return {
        "workload": f"network trained in {train_s:.1f} s on samples harvested from the {len(pts)} batch points "
                    f"(adaptive, then its own proposal, 3 stages); judged on {len(held)} held-out physical points, "
                    "event time integrated, 2e4-draw rounds until n_eff >= 1000 or "
                    f"{args.tmarg_draws} draws, against the adaptive (ra, sin dec) sampler",
        "adaptive": stats(ad), "learned_with_fallback": stats(le), "learned_without_fallback": stats(ln),
        "fallback_neff": args.fallback_neff,
        "points_fallen_back": int(sum(r["fallback_round"] >= 0 for r in le)),
        "points_compared": len(good),
        "median_abs_dlnL_marg_vs_adaptive": float(np.median(dl)) if len(dl) else None,
        "frac_within_0.05_of_adaptive": float(np.mean(dl <= 0.05)) if len(dl) else None,
        "seconds_adaptive": t_ad, "seconds_learned_with_fallback": t_le}


def run_quv(rift, W, peak):
    """Eq. (QUV) on the device for the full-size point (direct sums over the band: no FFT): the wall
    time of the C call (host preparation, uploads, kernels, downloads) and each kernel's CUDA-event
    time, after one warm call."""
    pt = W.make_point(W.cfg_full(), point_seed(0))
    rift.rift_quv(pt)
    times, qms, uvms = [], [], []
    for _ in range(3):
        t0 = time.perf_counter()
        rift.rift_quv(pt)
        times.append(time.perf_counter() - t0)
        a, b = rift.rift_quv_kernel_ms()
        qms.append(a)
        uvms.append(b)
    K, M, T = pt["Q"].shape
    nb = int((pt["weight"] != 0).any(axis=0).sum())
    q_flops = 8 * K * M * T * nb          # one complex multiply-add (4 FMA) per (k, mode, time, bin)
    uv_flops = 2 * 8 * K * M * M * nb     # U and V: one complex multiply-add each per (k, a, b, bin)
    q_ms, uv_ms = statistics.median(qms), statistics.median(uvms)
    return {"workload": f"K={K}, M={M}, n_t={T}, {nb} band bins of {len(pt['freqs'])}",
            "ms_per_point": 1e3 * statistics.median(times), "q_kernel_ms": q_ms, "uv_kernel_ms": uv_ms,
            "complex_macs": K * M * T * nb + 2 * K * M * M * nb,
            "roofline_q": {"bound": "alu", "kernel": "quv_q_kernel", "achieved": q_flops / (q_ms * 1e-3) / 1e12,
                           "peak": peak, "unit": "TFLOP/s", "frac": q_flops / (q_ms * 1e-3) / 1e12 / peak,
                           "flops": q_flops, "traffic": None},
            "roofline_uv": {"bound": "alu", "kernel": "quv_uv_kernel", "achieved": uv_flops / (uv_ms * 1e-3) / 1e12,
                            "peak": peak, "unit": "TFLOP/s", "frac": uv_flops / (uv_ms * 1e-3) / 1e12 / peak,
                            "flops": uv_flops, "traffic": None}}


def run_mdn(rift, peak):
    """The network's forward kernel on 4096 points (tensor cores; CUDA events around the kernel on
    the stream it runs on, the default stream), and one training step on 256 points with 64
    samples each (forward, loss, backward, Adam)."""
    import numpy as np
    import torch
    m = rift.rift_mdn_create(11)
    P = 4096
    g = torch.Generator(device="cuda").manual_seed(5)
    S = torch.randn((P, 64), device="cuda", generator=g)
    for _ in range(3):
        rift.rift_mdn_forward(m, S)
    torch.cuda.synchronize()
    fw = []
    for _ in range(5):
        rift.rift_mdn_forward(m, S)
        fw.append(rift.rift_mdn_forward_ms())
    B, H = 256, 64
    th = torch.rand((B, H, 5), device="cuda", generator=g) * 0.8 + 0.1
    w = torch.full((B, H), 1.0 / H, device="cuda")
    box = torch.as_tensor(np.tile(np.array([[0, 0, 0, 0, 0], [1, 1, 1, 1, 1]], dtype=np.float32), (B, 1, 1)),
                          device="cuda")
    rift.rift_mdn_train(m, S[:B], th, w, box, steps=3, batch=B, lr=1e-4)
    torch.cuda.synchronize()
    steps = 20
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    rift.rift_mdn_train(m, S[:B], th, w, box, steps=steps, batch=B, lr=1e-4)
    e1.record()
    e1.synchronize()
    tr = e0.elapsed_time(e1) / steps
    rift.rift_mdn_destroy(m)
    ms = statistics.median(fw)
    fl = mdn_forward_mma_flops(P)
    mp = measured_peaks() or {}
    tpeak = mp.get("bf16_tflops") or 1900.0
    return {"workload": f"forward on {P} points; training steps of {B} points x {H} samples",
            "forward_ms": ms, "train_step_ms": tr,
            "roofline_forward": {"bound": "tensor", "kernel": "mdn_forward_tc_kernel", "achieved": fl / (ms * 1e-3) / 1e12,
                                 "peak": tpeak, "unit": "TFLOP/s", "frac": fl / (ms * 1e-3) / 1e12 / tpeak,
                                 "flops": fl, "traffic": None,
                                 "peak_basis": "measured cuBLAS bf16 burst" if mp.get("bf16_tflops") else
                                               "fallback bf16 burst (no measured peaks)",
                                 "note": "tcgen05 BF16 products with FP32 accumulators in tensor memory, 128 points "
                                         "per CTA; flops are the network's (the kernel issues twice as many: each "
                                         "layer input is split into two BF16 terms); GELU on the CUDA cores"},
            "train_step_note": "the step's time includes the per-step loss read back to the host"}


def run_tmarg(rift, W, peak):
    """Eq. (lnL:tmarg): the event time integrated by quadrature for each draw.  Throughput on the
    full-size point (draws/s and likelihood points/s, CUDA events around the kernel launch)."""
    import numpy as np
    import torch
    pt = W.make_point(W.cfg_full(), point_seed(0))
    J = int(np.floor((pt["t_hi"] - pt["t_lo"]) * pt["fs"] + 1e-9))
    h = rift.rift_ile_create(pt)
    n = 200_000
    kw = dict(seed=5, n_per_round=n, max_evals=n, time_marg=1)
    for _ in range(3):
        rift.rift_ile_marginalize(h, **kw)
    torch.cuda.synchronize()
    kms = [rift.rift_ile_marginalize(h, timing=1, **kw)["kernel_ms"] for _ in range(5)]
    rift.rift_ile_destroy(h)
    ms = statistics.median(kms)
    # per (draw, t): per detector 8 M (conj(Y) Q row) + 4 taps x 4 (interpolation) + 4 (Re F Z); 12 for the
    # log-sum-exp step; per draw the quadratic forms and geometry of one sample
    K, M = pt["Q"].shape[0], pt["Q"].shape[1]
    flops = n * (J * (K * (8 * M + 4 * 4 + 4) + 12) + flops_per_sample(3, 21, 4))
    # executed by the merged-row GEMM form: per detector 4 flops per merged slot (Re(gamma q), 12 slots
    # for the 21 modes) and 2 per interpolation tap, no redundant rows counted
    mh = sum(1 for _, m in np.asarray(pt["lm"]).tolist() if m >= 0)
    exe = n * (J * (K * (4 * mh + 2 * 4) + 12) + flops_per_sample(3, 21, 4))
    return {
        "workload": f"full-size point, {n} draws per launch, each integrating J={J} times (midpoint rule on the "
                    "Q sampling interval)",
        "kernel_ms": ms, "draws_per_s": n / (ms * 1e-3), "lnL_points_per_s": n * J / (ms * 1e-3),
        "tflops": flops / (ms * 1e-3) / 1e12, "flops_per_draw": flops / n,
        "executed_flops_per_draw": exe / n, "executed_frac": exe / (ms * 1e-3) / 1e12 / peak,
        "roofline": {"bound": "alu", "kernel": "cells_kernel<3,4,0,2> (time-quadrature GEMM over merged rows)",
                     "achieved": flops / (ms * 1e-3) / 1e12,
                     "peak": peak, "unit": "TFLOP/s", "frac": flops / (ms * 1e-3) / 1e12 / peak, "traffic": None}}


def run_reference(args, world, rank):
    """The FP64 oracle timed as the reference arm on the host cores (rank 0 only): each step draws
    and evaluates a bounded sample of the same prior round (as many samples as the step's time
    budget allows), and the line reports the samples it ran and the time it took."""
    if rank != 0:
        return
    op = OraclePool()
    per_step = max(1.0, min(args.ref_seconds, 120.0 / max(1, args.steps + args.warmup)))
    walls, ns, start = [], [], 0
    for s in range(args.warmup + args.steps):
        v, n, wall = op.run(per_step, start=start)
        start += n
        if s >= args.warmup:
            walls.append(wall)
            ns.append(n)
    op.close()
    v = sum(ns) / sum(walls)
    desc = (f"{statistics.mean(ns):.0f} prior samples of the full-size point per step (seed 31, consecutive "
            f"indices), {op.cores} worker processes, about {per_step:.1f} s per step")
    out = {
        "impl": "reference",
        "metric": "extrinsic lnL evals/sec (and lnL_marg/sec) per GB300",
        "value": v, "unit": "evals/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.mean(walls), "samples_per_step": statistics.mean(ns),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic: seeded chirp-like modes, analytic aLIGO PSD, Gaussian noise",
        "config": bench_config(1),
        "cpu_baseline": {"value": v, "unit": "evals/s", "cores": op.cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def bench_config(world):
    """The workload the benchmark line is quoted on."""
    return {"workload": WORKLOAD, "global_batch": N_SAMPLES * world, "samples_per_point": N_SAMPLES,
            "points": world, "parallelism": f"independent points x{world}", "l2": "flushed between steps"}


def main():
    global N_SAMPLES
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=6.0)
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--extras", default="batched,learned,tmarg,quv,mdn",
                    help="comma-separated extras to run after the timed steps (profiling captures select one)")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch shape (profiling captures)")
    ap.add_argument("--batch-points", type=int, default=512)
    ap.add_argument("--batch-evals", type=int, default=2_000_000)
    ap.add_argument("--tmarg-draws", type=int, default=1_000_000,
                    help="draws per point at most in the time-marginalised batched runs")
    ap.add_argument("--heldout-points", type=int, default=128)
    ap.add_argument("--converge-points", type=int, default=16, help="points of the opt-in 'converge' extra")
    ap.add_argument("--converge-draws", type=int, default=200_000_000, help="draw cap per point of 'converge'")
    ap.add_argument("--fallback-neff", type=float, default=10.0)
    ap.add_argument("--samples", type=int, default=N_SAMPLES,
                    help="samples per step (profiling captures use a smaller count of the same workload)")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    N_SAMPLES = args.samples
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_gpu(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
