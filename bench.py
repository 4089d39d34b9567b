"""Benchmark: extrinsic lnL evaluations per second and lnL_marg per second on one GB300.

Workload (N = 1): the full-size plain ILE point -- 3 detectors (H1/L1/V1), all 21
modes with 2 <= l <= 4, Q over +-0.1 s at 16384 Hz, SNR 30 -- marginalised over
1e7 prior samples drawn on the device.  One step = one rift_ile_marginalize call
(Philox draw, response, harmonics, Q gather/interpolation, quadratic forms,
log-sum-exp, stopping rule) with Q/U/V already resident on the device.

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
    """Algorithmic FP32 flops of one likelihood evaluation (FMA = 2).

    quadratic forms over pairs a <= b: products conj(ya) yb and ya yb (12), then per
    detector Re(P U) (4) and R V (8); linear term per (k, lm): F conj(Y) (6) and per tap
    Re(c q) + weight (5); harmonics ~14 M; response + delay ~60 + 40 K; transforms,
    combine and log-sum-exp ~60."""
    npair = M * (M + 1) // 2
    quad = npair * (12 + 12 * K) + 10 * K
    lin = K * M * (6 + 5 * taps) + 8 * K
    return quad + lin + 14 * M + 60 + 40 * K + 60


def grouped_quad_flops(K: int, sparse: bool) -> int:
    """Flops the cell kernel executes for the quadratic forms of a point with all 21 (l <= 4) modes
    (grouped form): per pair one product d_a d_b and per detector two FMAs per part (one for the
    |m_b - m_a| = 0 group of the U part), one rotation per group and part, the F combination;
    with `sparse` the pairs that vanish for one-sign modes are skipped."""
    ms = [m for l in (2, 3, 4) for m in range(-l, l + 1)]
    pairs = [(a, b) for a in range(21) for b in range(a, 21)]
    u = [(a, b) for a, b in pairs if not (sparse and ms[a] * ms[b] < 0)]
    v = [(a, b) for a, b in pairs if not (sparse and ms[a] * ms[b] > 0)]
    fl = sum(1 + K * (2 if ms[a] == ms[b] else 4) for a, b in u) + sum(1 + 4 * K for _ in v)
    fl += len({abs(ms[b] - ms[a]) for a, b in u}) * 4 * K + len({ms[a] + ms[b] for a, b in v}) * 8 * K
    return fl + 8 * K


def executed_flops_per_sample(K: int, M: int, taps: int, sparse: bool) -> int:
    """flops_per_sample with the pair-form quadratic forms replaced by the grouped form the
    kernel runs for a full 21-mode point."""
    npair = M * (M + 1) // 2
    return flops_per_sample(K, M, taps) - (npair * (12 + 12 * K) + 10 * K) + grouped_quad_flops(K, sparse)


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
    """The FP64 oracle on the host cores: one spawned worker process per core, each holding the
    full-size point; timed on bounded samples of the same workload."""

    def __init__(self):
        import multiprocessing as mp
        self.cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_init)
        cal = self.pool.map(_oracle_chunk, [(31, i * 2000, 2000) for i in range(self.cores)])
        self.per_sample = max(c[0] / c[1] for c in cal)

    def run(self, target_s: float, start: int = 0):
        chunk = 20000
        n_chunks = max(self.cores, int(target_s / (self.per_sample * chunk)) * self.cores)
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_chunk, [(31, start + i * chunk, chunk) for i in range(n_chunks)])
        wall = time.perf_counter() - t0
        n = sum(r[1] for r in res)
        return n / wall, n, wall

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_oracle_throughput(target_s: float = 12.0):
    op = OraclePool()
    v, n, wall = op.run(target_s)
    op.close()
    return v, op.cores, f"{n} prior samples of the full-size point (indices 0..{n - 1}, seed 31)", wall


def precision_check(rift, pt, opts, tune):
    """Per-sample lnL of the benchmark's own launch (same point, seed and launch shape) against the
    FP64 oracle on the host: 2000 random draws and the 300 of highest weight, with the tolerance of
    the parity tests, 1e-3 max(1, <h|h>/900); and lnL_marg restricted to the top 300 on both sides."""
    import numpy as np
    import torch
    from oracle import likelihood as OL
    from oracle import mc
    h = rift.rift_ile_create(pt)
    rift.rift_ile_set_tune(h, cell_samples=tune["cell_samples"], smem_split=tune["smem_split"])
    n = opts["n_per_round"]
    dbg = torch.empty(n, dtype=torch.float32, device="cuda")
    res = rift.rift_ile_marginalize(h, dbg_ell=dbg, **opts)
    rift.rift_ile_destroy(h)
    got = dbg.cpu().numpy().astype(np.float64)
    del dbg
    top = np.argsort(got)[-300:]
    r = np.random.default_rng(7)
    idx = np.unique(np.concatenate([top, r.integers(0, n, 2000)])).astype(np.uint64)
    th, _, lq = mc.draw(opts["seed"], 0, 0, idx, mc.Prior(pt["t_lo"], pt["t_hi"]), None, tuple(res["strata"]), n)
    want = mc.lnL_samples(pt, th) + lq
    th64 = dict(ra=th["ra"], dec=np.arcsin(th["sindec"]), t=th["t"], psi=th["psi"], phi=th["phi"],
                incl=np.arccos(th["cosi"]), dist=th["dist"])
    hh = -2.0 * OL.lnL_factorised(dict(pt, Q=np.zeros_like(pt["Q"])), **th64)
    tol = 1e-3 * np.maximum(1.0, hh / 900.0)
    err = np.abs(got[idx.astype(np.int64)] - want)
    sel = np.isin(idx.astype(np.int64), top)
    a, b = mc.Accum.of(got[idx.astype(np.int64)][sel]).result()[0], mc.Accum.of(want[sel]).result()[0]
    return {"samples": int(idx.size), "max_abs_dlnL": float(err.max()), "max_err_over_tol": float((err / tol).max()),
            "mean_err_over_tol": float((err / tol).mean()), "dlnL_marg_top300": float(abs(a - b)),
            "tolerance": "1e-3 max(1, <h|h>/900) per sample (FP64 oracle, same draws)"}


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
    opts = dict(seed=1234 + rank, n_per_round=N_SAMPLES, max_evals=N_SAMPLES)
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
    fl = flops_per_sample(K, M, taps) * N_SAMPLES
    kmean = statistics.mean(kern_ms)
    achieved = fl / (kmean * 1e-3) / 1e12
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    f_mhz = clk["sm_mhz"] or 1455.0
    peak = 2 * 128 * sms * f_mhz * 1e6 / 1e12

    # end to end through the public API with host buffers: create (host Q/U/V -> device)
    # + marginalise + result back, every step
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
            r = rift.rift_ile_marginalize(h2, **opts)
            rift.rift_ile_destroy(h2)
            times.append(time.perf_counter() - t0)
            rounds = r["rounds"]
        e2e_s = max_over_ranks(world, statistics.mean(times))
        e2e = {"value": evals / e2e_s, "unit": "evals/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": 64 * rounds + 4,
               "includes": "rift_ile_create from host FP64 arrays + rift_ile_marginalize + result read + destroy"}

    cpu = None
    precision = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, cores, sample, wall = cpu_oracle_throughput(args.cpu_seconds)
        cpu = {"value": v, "unit": "evals/s", "cores": cores, "kind": "oracle", "sample": sample,
               "wall_s": round(wall, 2)}
        precision = precision_check(rift, pt, opts, tune)

    extras = {}
    if rank == 0 and world == 1 and not args.no_extras:
        extras = run_extras(args, rift, W)

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
        "dtype": "f32 (double-float time index; f64 accumulators)",
        "data": "synthetic: seeded chirp-like modes, analytic aLIGO PSD, Gaussian noise; samples drawn on device",
        "config": {"workload": WORKLOAD, "global_batch": N_SAMPLES * world, "samples_per_point": N_SAMPLES,
                   "points": world, "parallelism": f"independent points x{world}", "l2": "flushed between steps"},
        "lnL_marg_per_s": world / (ms_per_step * 1e-3),
        "lnL_marg": r0["lnL_marg"], "n_eff": r0["n_eff"], "strata": list(r0["strata"]),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": recorded_traffic(),
                     "kernel": "cells_kernel_cp<3,4,1> (stratified cell: draw + staged Q window + likelihood with the "
                               "grouped quadratic form, coefficients in the parameter bank + log-sum-exp)",
                     "kernel_ms": kmean, "flops_per_sample": flops_per_sample(K, M, taps),
                     "executed_flops_per_sample": executed_flops_per_sample(K, M, taps, True),
                     "executed_frac": executed_flops_per_sample(K, M, taps, True) * N_SAMPLES / (kmean * 1e-3) / 1e12
                     / peak,
                     "peak_basis": f"FP32 FMA: 128 lanes/SM x {sms} SMs x 2 flop x median SM clock {f_mhz} MHz "
                                   "sampled during the run"},
        "gpu_launches": launches,
        "autotune": tune,
        "clocks": clk,
        "e2e": e2e,
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
    spec, seed = args
    return W.make_point(spec, seed)


def make_points(specs, seed0):
    """Generate many points on the host cores (spawned processes, before heavy GPU work)."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    with mp.get_context("spawn").Pool(min(cores, 32)) as pool:
        return pool.map(_make_point, [(s, seed0 + i) for i, s in enumerate(specs)], chunksize=4)


def run_extras(args, rift, W):
    """The batched workload (many points, uneven mode counts and Q lengths, adaptive rounds,
    one graph-replayed launch sequence) against sequential per-point runs, and the learned
    proposal against the prior at equal evaluations."""
    import numpy as np
    import torch
    out = {}
    t0 = time.perf_counter()
    specs = W.batch_specs(args.batch_points, seed=5)
    for sp in specs:
        sp.seg_len = 2.0
    pts = make_points(specs, 1000)
    gen_s = time.perf_counter() - t0
    hb = rift.rift_ile_batch_create(pts)
    kw = dict(seed=3, n_per_round=100000, max_evals=args.batch_evals, n_eff_target=1000.0, proposal="adaptive",
              n_bins=100)
    rift.rift_ile_batch_marginalize(hb, **kw)          # warm-up (graph instantiation, scratch)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = rift.rift_ile_batch_marginalize(hb, **kw)
    torch.cuda.synchronize()
    bt = time.perf_counter() - t0
    nseq = min(32, len(pts))
    hs = [rift.rift_ile_create(p) for p in pts[:nseq]]
    rift.rift_ile_marginalize(hs[0], point_id=0, **kw)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, hh in enumerate(hs):
        rift.rift_ile_marginalize(hh, point_id=i, **kw)
    torch.cuda.synchronize()
    st = time.perf_counter() - t0
    ev = sum(r["n_evals"] for r in res)
    out["batched"] = {
        "workload": f"{len(pts)} points, 3 detectors, M U{{5..21}}, Q U[800,3300] @ 16384 Hz, SNR U[8,30]; adaptive "
                    f"1e5-sample rounds until n_eff >= 1000 or {args.batch_evals} evaluations per point",
        "points_per_s": len(pts) / bt, "evals_per_s": ev / bt, "seconds": bt,
        "sequential_points_per_s": nseq / st, "speedup_vs_sequential": (len(pts) / bt) / (nseq / st),
        "points_reaching_neff_1000": int(sum(r["n_eff"] >= 1000 for r in res)),
        "median_n_eff": float(np.median([r["n_eff"] for r in res])), "generation_s": gen_s}
    # learned proposal: train on harvested samples of the batch, compare with the prior
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
    ek = dict(seed=9, n_per_round=262144, max_evals=262144 * 4)
    prior = rift.rift_ile_batch_marginalize(hb, **ek)
    learned = rift.rift_ile_batch_marginalize(hb, proposal="learned", mdn=m, **ek)
    gains = np.array([l["n_eff"] / p["n_eff"] for l, p in zip(learned, prior)])
    dl = np.array([abs(l["lnL_marg"] - p["lnL_marg"]) for l, p in zip(learned, prior)])
    out["learned"] = {
        "workload": f"MDN trained in {train_s:.1f} s on samples harvested from the same {len(pts)} points "
                    "(adaptive, then its own proposal, 3 stages); both proposals 1.05e6 evaluations per point",
        "median_n_eff_gain": float(np.median(gains)), "mean_n_eff_gain": float(gains.mean()),
        "median_n_eff_prior": float(np.median([p["n_eff"] for p in prior])),
        "median_n_eff_learned": float(np.median([l["n_eff"] for l in learned])),
        "median_abs_dlnL_marg": float(np.median(dl)), "frac_within_0.05": float(np.mean(dl <= 0.05))}
    out["time_marginalised"] = run_tmarg(rift, W, pts[:16])
    out["quv"] = run_quv(rift, W)
    return out


def run_quv(rift, W):
    """Eq. (QUV) on the device for the full-size point (direct sums over the band: no FFT), the
    wall time of the C call including its uploads and downloads, after one warm call."""
    pt = W.make_point(W.cfg_full(), point_seed(0))
    rift.rift_quv(pt)
    times = []
    for _ in range(3):
        t0 = time.perf_counter()
        rift.rift_quv(pt)
        times.append(time.perf_counter() - t0)
    K, M, T = pt["Q"].shape
    nb = int((pt["weight"] != 0).any(axis=0).sum())
    return {"workload": f"K={K}, M={M}, n_t={T}, {nb} band bins of {len(pt['freqs'])}",
            "ms_per_point": 1e3 * statistics.median(times),
            "complex_macs": K * M * T * nb + 2 * K * M * M * nb}


def run_tmarg(rift, W, pts):
    """Eq. (lnL:tmarg): the event time integrated by quadrature for each draw.  Throughput on the
    full-size point (draws/s and likelihood points/s, CUDA events around the kernel launch) and,
    on batched points, n_eff and lnL_marg against the sampled-time estimator at equal time."""
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
    flops = n * (J * (pt["Q"].shape[0] * (8 * pt["Q"].shape[1] + 4 * 4 + 4) + 12) + flops_per_sample(3, 21, 4))
    ns, nt, dl = [], [], []
    for i, p in enumerate(pts):
        hh = rift.rift_ile_create(p)
        a = rift.rift_ile_marginalize(hh, seed=3, point_id=i, n_per_round=100000, max_evals=2_000_000,
                                      proposal="adaptive", n_bins=100)
        b = rift.rift_ile_marginalize(hh, seed=3, point_id=i, n_per_round=20000, max_evals=400_000,
                                      proposal="adaptive", n_bins=100, time_marg=1)
        ns.append(a["n_eff"]); nt.append(b["n_eff"]); dl.append(b["lnL_marg"] - a["lnL_marg"])
        rift.rift_ile_destroy(hh)
    return {
        "workload": f"full-size point, {n} draws per launch, each integrating J={J} times (midpoint rule on the "
                    f"Q sampling interval); {len(pts)} batched points, adaptive (ra, sin dec), 4e5 draws vs 2e6 "
                    "sampled-time evaluations per point",
        "kernel_ms": ms, "draws_per_s": n / (ms * 1e-3), "lnL_points_per_s": n * J / (ms * 1e-3),
        "tflops": flops / (ms * 1e-3) / 1e12, "flops_per_draw": flops / n,
        "median_n_eff_tmarg": float(np.median(nt)), "median_n_eff_sampled_t": float(np.median(ns)),
        "median_lnL_marg_tmarg_minus_sampled": float(np.median(dl))}


def run_reference(args, world, rank):
    """The FP64 oracle timed as the reference arm on the host cores (rank 0 only)."""
    if rank != 0:
        return
    op = OraclePool()
    per_step, desc = [], None
    for s in range(args.warmup + args.steps):
        v, n, wall = op.run(args.ref_seconds)
        if s >= args.warmup:
            per_step.append(v)
            desc = f"{n} prior samples of the full-size point per step (seed 31), {op.cores} worker processes"
    op.close()
    v = statistics.mean(per_step)
    out = {
        "impl": "reference",
        "metric": "extrinsic lnL evals/sec (and lnL_marg/sec) per GB300",
        "value": v, "unit": "evals/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": N_SAMPLES / v * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (same workload generator)",
        "config": {"workload": WORKLOAD, "global_batch": N_SAMPLES, "points": 1,
                   "parallelism": "host cores (spawned processes)"},
        "cpu_baseline": {"value": v, "unit": "evals/s", "cores": op.cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


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
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch shape (profiling captures)")
    ap.add_argument("--batch-points", type=int, default=512)
    ap.add_argument("--batch-evals", type=int, default=2_000_000)
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
