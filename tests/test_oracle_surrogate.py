"""Pins of the oracle's surrogate pieces against independent computations:
features by brute force from the pick set, bf16 rounding against torch,
the MLP forward against torch float64 layers, its backward against torch
autograd and finite differences, Adam against torch.optim.Adam."""
import numpy as np
import torch

import oracle
import wh_gen


def brute_features(lay, locs):
    A, L = lay.n_aisles, lay.slots_per_side
    per = {}
    for loc in locs:
        a, k = loc // (2 * L), loc % L
        lo, hi = per.get(a, (k, k))
        per[a] = (min(lo, k), max(hi, k))
    f = np.zeros(192, np.float32)
    for a, (lo, hi) in per.items():
        f[hi * 64 // L] += 1
        f[64 + lo * 64 // L] += 1
        f[132 + a * 60 // A] += 1
    inv = np.float32(1.0 / A)
    if per:
        f[128] = np.float32(min(per)) * inv
        f[129] = np.float32(max(per)) * inv
    f[130] = np.float32(len(per)) * inv
    f[131] = np.float32(len(locs)) * np.float32(1 / 64)
    return f


def test_features_match_brute_force():
    rng = np.random.default_rng(1)
    for lay in (wh_gen.Layout(10, 30), wh_gen.Layout(500, 200), wh_gen.Layout(7, 13, 2, 3, 4), wh_gen.Layout(1, 5)):
        for _ in range(200):
            locs = rng.integers(0, lay.n_loc, size=int(rng.integers(0, 70)))
            assert np.array_equal(oracle.features(lay, locs), brute_features(lay, locs))


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.normal(size=5000).astype(np.float32) * 10.0 ** rng.integers(-5, 5, size=5000),
                        np.float32([0, -0.0, 1, 255, 257, 1e-30, 3.3895314e38])]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(oracle.bf16(x), want)


def rand_params(seed, scale=0.08):
    rng = np.random.default_rng(seed)
    p = {"w1": rng.normal(size=(192, 256)) * scale, "b1": rng.normal(size=256) * 0.05,
         "w2": rng.normal(size=(256, 256)) * scale, "b2": rng.normal(size=256) * 0.05,
         "w3": rng.normal(size=256) * scale, "b3": rng.normal(size=1) * 0.05}
    return {k: oracle.bf16(v.astype(np.float32)) for k, v in p.items()}


def rand_x(seed, n):
    rng = np.random.default_rng(seed)
    x = np.abs(rng.normal(size=(n, 192))).astype(np.float32) * 2
    return oracle.bf16(np.floor(x * 4) / 4)


def torch_forward(p, X, ste=False):
    t = {k: torch.tensor(v, dtype=torch.float64, requires_grad=ste) for k, v in p.items()}
    x = torch.tensor(X, dtype=torch.float64)

    def rnd(h):
        r = h.detach().to(torch.float32).to(torch.bfloat16).to(torch.float64)
        return h + (r - h).detach() if ste else r

    g = lambda z: 0.5 * z * (1 + torch.erf(z / np.sqrt(2.0)))
    h1 = rnd(g(x @ t["w1"] + t["b1"]))
    h2 = rnd(g(h1 @ t["w2"] + t["b2"]))
    return h2 @ t["w3"] + t["b3"], t


def test_forward_matches_torch_float64():
    p, X = rand_params(3), rand_x(4, 64)
    y = oracle.mlp_forward(p, X)
    want, _ = torch_forward(p, X)
    np.testing.assert_allclose(y, want.detach().numpy(), rtol=1e-9, atol=1e-9)


def test_backward_matches_autograd_and_finite_differences():
    p, X = rand_params(5), rand_x(6, 32)
    tgt = np.random.default_rng(7).normal(size=32)
    loss, g = oracle.mlp_backward(p, X, tgt)
    y, t = torch_forward(p, X, ste=True)
    tl = 0.5 * ((y - torch.tensor(tgt)) ** 2).mean()
    tl.backward()
    assert abs(loss - tl.item()) < 1e-9
    for k in p:
        np.testing.assert_allclose(g[k].reshape(-1), t[k].grad.numpy().reshape(-1), rtol=1e-6, atol=1e-10)
    # finite differences on the output layer, where no rounding sits between
    # the parameter and the loss
    eps = 1e-3
    for k, idx in (("w3", 7), ("b3", 0), ("w3", 100)):
        q = {kk: vv.copy() for kk, vv in p.items()}
        q[k] = q[k].astype(np.float64)
        q[k].reshape(-1)[idx] += eps
        up = 0.5 * np.mean((torch_forward(q, X)[0].detach().numpy() - tgt) ** 2)
        q[k].reshape(-1)[idx] -= 2 * eps
        dn = 0.5 * np.mean((torch_forward(q, X)[0].detach().numpy() - tgt) ** 2)
        assert abs((up - dn) / (2 * eps) - g[k].reshape(-1)[idx]) < 1e-6


def test_train_trace_matches_autograd_with_rounded_gradients():
    """The training trace against torch float64 autograd in which the forward
    rounds h1, h2 to bf16 (straight through) and gradient hooks round
    dL/dz2 and dL/dz1 to bf16: the same rounding points, computed
    independently.  With the roundings made identity the gradients reduce
    to or_mlp_backward's."""
    p, X = rand_params(9), rand_x(10, 48)
    tgt = np.random.default_rng(11).normal(size=48) * 0.1
    loss, tr, g = oracle.mlp_train_trace(p, X, tgt)
    t = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in p.items()}
    x = torch.tensor(X, dtype=torch.float64)
    rnd = lambda v: v.detach().to(torch.float32).to(torch.bfloat16).to(torch.float64)
    ste = lambda h: h + (rnd(h) - h).detach()
    gel = lambda z: 0.5 * z * (1 + torch.erf(z / np.sqrt(2.0)))
    seen = {}

    def hook(name):
        def f(grad):
            seen[name + "pre"] = grad.detach().clone()
            seen[name] = rnd(grad)
            return seen[name]
        return f

    z1 = x @ t["w1"] + t["b1"]
    z1.register_hook(hook("d1"))
    h1 = ste(gel(z1))
    z2 = h1 @ t["w2"] + t["b2"]
    z2.register_hook(hook("d2"))
    h2 = ste(gel(z2))
    y = h2 @ t["w3"] + t["b3"]
    tl = 0.5 * ((y - torch.tensor(tgt)) ** 2).mean()
    tl.backward()
    assert abs(loss - tl.item()) < 1e-12
    for k, v in (("z1", z1), ("h1", h1), ("z2", z2), ("h2", h2)):
        np.testing.assert_allclose(tr[k], v.detach().numpy(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(tr["y"], y.detach().numpy(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(tr["dy"], (y.detach().numpy() - tgt) / 48, rtol=1e-12, atol=1e-15)
    for k in ("d2pre", "d2", "d1pre", "d1"):
        np.testing.assert_allclose(tr[k], seen[k].numpy(), rtol=1e-9, atol=1e-18)
    # the rounded gradients are bf16 values; about half their entries moved
    assert np.array_equal(tr["d2"], oracle.bf16(tr["d2"]).astype(np.float64))
    assert (tr["d1"] != tr["d1pre"]).mean() > 0.5
    for k in p:
        np.testing.assert_allclose(g[k].reshape(-1), t[k].grad.numpy().reshape(-1), rtol=1e-9, atol=1e-15)
    # without the gradient roundings: the plain backward
    _, g0 = oracle.mlp_backward(p, X, tgt)
    for k in ("w3", "b3"):
        np.testing.assert_allclose(g[k], g0[k], rtol=1e-12, atol=1e-18)
    assert not np.allclose(g["w1"], g0["w1"], rtol=1e-6, atol=0)


def test_adam_matches_torch():
    rng = np.random.default_rng(8)
    p0 = rng.normal(size=50)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    tp = torch.tensor(p0, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    for step in range(1, 6):
        g = rng.normal(size=50)
        oracle.adam(p, m, v, g, 1e-2, step)
        opt.zero_grad()
        tp.grad = torch.tensor(g)
        opt.step()
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-12, atol=1e-12)


def test_inference_erf_approximation_bound():
    """The tensor-core inference evaluates erf by Abramowitz & Stegun 7.1.28
    (after Hastings); its published bound |error| <= 3e-7 holds for the
    formula with these coefficients (float64, dense grid; odd extension)."""
    from scipy.special import erf
    a = (0.0705230784, 0.0422820123, 0.0092705272, 0.0001520143, 0.0002765672, 0.0000430638)
    x = np.linspace(-8.0, 8.0, 400001)
    ax = np.abs(x)
    poly = 1.0 + ax * (a[0] + ax * (a[1] + ax * (a[2] + ax * (a[3] + ax * (a[4] + ax * a[5])))))
    approx = np.sign(x) * (1.0 - poly ** -16.0)
    assert np.abs(approx - erf(x)).max() <= 3e-7
