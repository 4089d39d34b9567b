"""Learned proposal on the GPU against the oracle: summary features, network forward,
loss and gradient, the proposal's sampler and density, a marginalisation with a given
proposal, and what training buys over the prior."""
from __future__ import annotations

import math

import numpy as np
import pytest

import workload as W
from oracle import mc
from oracle import mdn
from oracle import philox as P

pytestmark = pytest.mark.gpu


def _params(seed, scale=0.5):
    r = np.random.default_rng(seed)
    W_ = {k: r.normal(0.0, scale / math.sqrt(max(1, s[-1])), s) for k, s in mdn.SHAPES.items()}
    return mdn.flatten(W_).astype(np.float32)


@pytest.fixture(scope="module")
def pts():
    specs = W.batch_specs(5, seed=8, snr_range=(10.0, 20.0), fs=4096.0, t_range=(300, 600), m_range=(5, 21))
    for s in specs:
        s.seg_len = 2.0
    return [W.make_point(s, 300 + i) for i, s in enumerate(specs)]


def test_summary_matches_oracle(lib, cuda, pts):
    h = lib.rift_ile_batch_create(pts)
    got = lib.rift_ile_batch_summary(h).cpu().numpy().astype(np.float64)
    for p, pt in enumerate(pts):
        want = mdn.summary(pt)
        assert np.allclose(got[p], want, rtol=2e-4, atol=2e-5), (p, np.max(np.abs(got[p] - want)))


@pytest.mark.parametrize("n,scale", [(1, 1.0), (37, 1.0), (128, 3.0), (300, 1.0)])
def test_forward_matches_oracle(lib, cuda, n, scale):
    """The tensor-core forward pass (128 points per CTA: one point, a partial CTA, one full CTA,
    three CTAs with a ragged last one) against the oracle's FP64 network on the BF16 weights."""
    import torch
    m = lib.rift_mdn_create(1)
    prm = _params(2)
    lib.rift_mdn_set_params(m, prm)
    bfw = lib.rift_mdn_get_params(m, 1).astype(np.float64)
    assert np.array_equal(bfw, mdn.bf16_round(prm))              # round-to-nearest-even, bit for bit
    S = np.random.default_rng(3 + n).normal(0, scale, (n, 64)).astype(np.float32)
    got = lib.rift_mdn_forward(m, torch.as_tensor(S, device="cuda")).cpu().numpy().astype(np.float64)
    want = mdn.forward(mdn.unflatten(bfw), S.astype(np.float64))
    assert np.allclose(got, want, rtol=1e-4, atol=1e-4), float(np.max(np.abs(got - want)))


def test_loss_and_gradient_match_oracle(lib, cuda):
    import torch
    m = lib.rift_mdn_create(1)
    prm = _params(4, scale=0.3)
    lib.rift_mdn_set_params(m, prm)
    Wb = mdn.unflatten(mdn.bf16_round(prm))
    n, H = 6, 50
    r = np.random.default_rng(5)
    S = r.normal(0, 1, (n, 64))
    a, b = mdn.bounds(-0.04, 0.04, 1.0, 1000.0)
    th = a + (b - a) * r.uniform(0.03, 0.97, (n, H, 5))
    w = r.uniform(0.1, 1.0, (n, H))
    box = np.stack([np.stack([a, b])] * n)
    dev = lambda x: torch.as_tensor(np.ascontiguousarray(x, dtype=np.float32), device="cuda")
    loss, g = lib.rift_mdn_loss_grad(m, dev(S), dev(th), dev(w), dev(box))
    wl, wg = mdn.loss_and_grad(Wb, S.astype(np.float32).astype(np.float64),
                               [(th[i].astype(np.float32).astype(np.float64), w[i].astype(np.float32)) for i in range(n)],
                               [a] * n, [b] * n)
    wg = mdn.flatten(wg)
    assert abs(loss - wl) < 1e-4 * abs(wl) + 1e-4
    assert np.max(np.abs(g - wg)) < 2e-3 * np.max(np.abs(wg)) + 1e-6


def test_adam_step_on_device(lib, cuda):
    import torch
    m = lib.rift_mdn_create(1)
    prm = _params(6, scale=0.3)
    lib.rift_mdn_set_params(m, prm)
    n, H = 4, 30
    r = np.random.default_rng(7)
    a, b = mdn.bounds(-0.04, 0.04, 1.0, 1000.0)
    dev = lambda x: torch.as_tensor(np.ascontiguousarray(x, dtype=np.float32), device="cuda")
    S, th, w = dev(r.normal(0, 1, (n, 64))), dev(a + (b - a) * r.uniform(0.05, 0.95, (n, H, 5))), dev(np.ones((n, H)))
    box = dev(np.stack([np.stack([a, b])] * n))
    _, g = lib.rift_mdn_loss_grad(m, S, th, w, box)
    lib.rift_mdn_train(m, S, th, w, box, steps=1, batch=n, lr=1e-3)
    new = lib.rift_mdn_get_params(m, 0).astype(np.float64)
    want = prm.astype(np.float64) - 1e-3 * g / (np.abs(g) + 1e-8)     # Adam's first step
    # the gradient is summed with atomics, so its order varies between the two evaluations: a
    # component within rounding of zero can change sign, which flips its first step (+-lr)
    sure = np.abs(g) > 1e-5 * np.abs(g).max()
    assert sure.mean() > 0.5
    assert np.allclose(new[sure], want[sure], atol=2e-6)
    assert np.all(np.abs(new - prm) <= 1e-3 + 2e-6)


def _head(seed, pt):
    """A proposal head concentrated around the best of a few thousand prior draws."""
    pr = mc.Prior(pt["t_lo"], pt["t_hi"])
    u = P.uniforms(seed, 0, 0, np.arange(20000, dtype=np.uint64), 8)
    th = mc.prior_transform(u, pr)
    ell = mc.lnL_samples(pt, th)
    top = np.argsort(ell)[-8:]
    a, b = mdn.bounds(pr.t_lo, pr.t_hi, pr.d_lo, pr.d_hi)
    th5 = np.stack([th["ra"], th["sindec"], th["t"], th["cosi"], np.log(th["dist"])], axis=-1)[top]
    x = (th5 - a) / (b - a)
    z = np.log(x) - np.log1p(-x)
    head = np.zeros(mdn.N_OUT)
    head[mdn.N_COMP:mdn.N_COMP + 40] = z.ravel()
    head[mdn.N_COMP + 40:] = np.tile([-1.0, -1.0, -3.0, -0.5, -0.5], 8)
    return head.astype(np.float32)


def test_learned_sampler_matches_oracle(lib, cuda, pts):
    pt = pts[0]
    h = lib.rift_ile_create(pt)
    head = _head(11, pt)
    lib.rift_ile_set_proposal_head(h, head[None])
    n = 20000
    theta, lpq, _ = lib.rift_ile_draw(h, 2, n, seed=13, proposal="learned")
    g = theta.cpu().numpy().astype(np.float64)
    pr = mc.Prior(pt["t_lo"], pt["t_hi"])
    u = P.uniforms(13, 0, 2, np.arange(n, dtype=np.uint64), 10)
    th, lq = mdn.sample(u, head.astype(np.float64)[None], pr)
    assert np.allclose(g[0], th["ra"], atol=2e-5)
    assert np.allclose(g[1], th["sindec"], atol=2e-6)
    assert np.allclose(g[2], th["t"], atol=5e-8)
    assert np.allclose(g[5], th["cosi"], atol=2e-6)
    assert np.allclose(g[6], th["dist"], rtol=1e-5)
    assert np.allclose(lpq.cpu().numpy(), lq, atol=2e-4)


def test_learned_marginalisation_matches_oracle(lib, cuda, pts):
    pt = pts[1]
    h = lib.rift_ile_create(pt)
    head = _head(12, pt)
    lib.rift_ile_set_proposal_head(h, head[None])
    n = 40000
    res = lib.rift_ile_marginalize(h, seed=17, n_per_round=n, max_evals=2 * n, proposal="learned")
    pr = mc.Prior(pt["t_lo"], pt["t_hi"])
    acc = mc.Accum()
    for rnd in range(2):
        u = P.uniforms(17, 0, rnd, np.arange(n, dtype=np.uint64), 10)
        th, lq = mdn.sample(u, head.astype(np.float64)[None], pr)
        acc = acc.merge(mc.Accum.of(mc.lnL_samples(pt, th) + lq))
    want = acc.result()
    assert res["n_evals"] == 2 * n
    assert abs(res["lnL_marg"] - want[0]) < 1e-4, (res["lnL_marg"], want[0], res["n_eff"])
    assert abs(res["n_eff"] - want[1]) < 1e-3 * want[1] + 1e-3


def test_learned_estimator_is_unbiased(lib, cuda):
    """A given learned proposal (not trained) keeps the estimator unbiased: on weak signals
    (SNR 4-5) its lnL_marg agrees with a long plain run within the Monte Carlo errors."""
    specs = W.batch_specs(4, seed=31, snr_range=(4.0, 5.0), fs=4096.0, t_range=(300, 500), m_range=(5, 7))
    for s in specs:
        s.seg_len = 2.0
    pts_ = [W.make_point(s, 700 + i) for i, s in enumerate(specs)]
    h = lib.rift_ile_batch_create(pts_)
    heads = np.stack([_head(40 + i, p) for i, p in enumerate(pts_)])
    lib.rift_ile_set_proposal_head(h, heads)
    plain = lib.rift_ile_batch_marginalize(h, seed=1, n_per_round=1 << 24, max_evals=1 << 27)
    learned = lib.rift_ile_batch_marginalize(h, seed=2, n_per_round=1 << 20, max_evals=1 << 23, proposal="learned")
    for l, p in zip(learned, plain):
        assert p["n_eff"] > 30, p
        s = math.hypot(l["sigma"], p["sigma"])
        assert abs(l["lnL_marg"] - p["lnL_marg"]) < 5 * s + 0.02, (l, p)


def test_training_improves_on_the_prior(lib, cuda):
    """What the trained network gains: harvest tempered posterior samples of training points
    (first from the adaptive histogram sampler, then from the network's own proposal), train,
    and compare n_eff per evaluation of the learned proposal with the prior on those points."""
    import torch
    specs = W.batch_specs(64, seed=21, snr_range=(8.0, 15.0), fs=4096.0, t_range=(300, 500), m_range=(5, 9))
    for s in specs:
        s.seg_len = 2.0
    train = [W.make_point(s, 500 + i) for i, s in enumerate(specs)]
    ht = lib.rift_ile_batch_create(train)
    S = lib.rift_ile_batch_summary(ht)
    box = torch.as_tensor(lib.rift_ile_boxes(ht), device="cuda")
    H = 64
    w = torch.full((len(train), H), 1.0 / H, device="cuda")
    m = lib.rift_mdn_create(3)
    first = None
    for stage in range(3):
        kw = dict(seed=5 + stage, n_per_round=65536, max_evals=262144)
        if stage == 0:
            theta, _ = lib.rift_ile_batch_harvest(ht, H, beta=0.5, proposal="adaptive", n_bins=32, **kw)
        else:
            theta, _ = lib.rift_ile_batch_harvest(ht, H, beta=0.5, proposal="learned", mdn=m, **kw)
        assert not torch.isnan(theta).any()
        losses = lib.rift_mdn_train(m, S, theta, w, box, steps=800, batch=64, lr=1e-3)
        first = losses[:10].mean() if first is None else first
    assert losses[-10:].mean() < first
    kw = dict(seed=9, n_per_round=65536, max_evals=65536 * 4)
    prior = lib.rift_ile_batch_marginalize(ht, **kw)
    learned = lib.rift_ile_batch_marginalize(ht, proposal="learned", mdn=m, **kw)
    gain = np.median([l["n_eff"] / p["n_eff"] for l, p in zip(learned, prior)])
    assert gain > 2.0, gain


def _far_head():
    """Every mixture component at the corner of the box with narrow widths: only the defensive prior
    component of the proposal covers the likelihood, so the learned rounds' weights degenerate."""
    head = np.zeros(mdn.N_OUT, dtype=np.float32)
    head[mdn.N_COMP:mdn.N_COMP + 40] = 4.0
    head[mdn.N_COMP + 40:] = -3.0
    return head


@pytest.mark.parametrize("path", ["single", "batched"])
def test_learned_fallback_matches_oracle(lib, cuda, pts, path):
    """The fallback to the adaptive sampler: a learned round whose own n_eff is below fallback_neff
    hands the point to the adaptive proposal.  With the threshold just above the oracle's round-0
    value the device falls back at round 1, as the oracle does, and the pooled lnL_marg (a learned
    round, then an adaptive round from the prior's tables) agrees at 1e-4; with the threshold below
    every learned round's n_eff the point stays learned."""
    pt = pts[2]
    pr = mc.Prior(pt["t_lo"], pt["t_hi"])
    head = _far_head()
    n = 20000
    ref0 = mc.marginalize_learned(pt, 61, 0, pr, head.astype(np.float64), n, 2 * n, 1e300)
    rn = ref0["round_neff"]
    h = lib.rift_ile_create(pt) if path == "single" else lib.rift_ile_batch_create([pt])
    lib.rift_ile_set_proposal_head(h, head[None])
    run = lib.rift_ile_marginalize if path == "single" else (lambda hh, **kw: lib.rift_ile_batch_marginalize(hh, **kw)[0])
    kw = dict(seed=61, n_per_round=n, max_evals=2 * n, proposal="learned", n_bins=32)
    stay = run(h, fallback_neff=0.5 * min(rn), **kw)
    assert stay["fallback_round"] == -1
    assert abs(stay["lnL_marg"] - ref0["lnL_marg"]) < 1e-4
    ref = mc.marginalize_learned(pt, 61, 0, pr, head.astype(np.float64), n, 2 * n, 1e300,
                                 fallback_neff=1.01 * rn[0], n_bins=32)
    assert ref["fallback_round"] == 1
    got = run(h, fallback_neff=1.01 * rn[0], **kw)
    assert got["fallback_round"] == 1 and got["n_evals"] == 2 * n and got["rounds"] == 2
    assert abs(got["lnL_marg"] - ref["lnL_marg"]) < 1e-4, (got["lnL_marg"], ref["lnL_marg"])
    assert abs(got["n_eff"] - ref["n_eff"]) <= 1e-3 * ref["n_eff"] + 1e-3
    with pytest.raises(lib.RiftError):
        lib.rift_ile_marginalize(lib.rift_ile_create(pt), seed=1, n_per_round=n, max_evals=n, fallback_neff=5.0)


def test_training_is_deterministic(lib, cuda, pts):
    """Weight gradients are sums over the batch's points in a fixed order (no float atomics): two
    trainings from the same initial parameters on the same data give the same parameters, bit for
    bit (the device gradient against the oracle is test_loss_and_gradient_match_oracle)."""
    import torch
    h = lib.rift_ile_batch_create(pts)
    S = lib.rift_ile_batch_summary(h)
    box = torch.as_tensor(lib.rift_ile_boxes(h), device="cuda")
    g = torch.Generator(device="cuda").manual_seed(4)
    H = 32
    theta = box[:, 0:1, :] + (box[:, 1:2, :] - box[:, 0:1, :]) * (0.05 + 0.9 * torch.rand((len(pts), H, 5), device="cuda",
                                                                                         generator=g))
    w = torch.full((len(pts), H), 1.0 / H, device="cuda")
    out = []
    for _ in range(2):
        m = lib.rift_mdn_create(21)
        lib.rift_mdn_train(m, S, theta, w, box, steps=50, batch=len(pts), lr=1e-3)
        out.append(lib.rift_mdn_get_params(m))
        lib.rift_mdn_destroy(m)
    assert np.array_equal(out[0], out[1])
