"""The element-wise bounds of tests/mlp_chain.py on the CPU: a float32
emulation of the device's training step (bf16 operands, fp32 sums, the same
rounding points) passes them, and planted mistakes in it (a gradient entry of
the wrong sign, two gradient rows exchanged, a dropped term of GELU', a
dropped bias) fail them.  This shows the bounds are tight enough to catch
the mistakes a wrong kernel would make."""
import numpy as np
import pytest
import torch

import mlp_chain
import oracle


def params(seed, scale=0.06):
    rng = np.random.default_rng(seed)
    d = {"w1": rng.normal(size=(192, 256)) * scale, "b1": rng.normal(size=256) * 0.05,
         "w2": rng.normal(size=(256, 256)) * scale, "b2": rng.normal(size=256) * 0.05,
         "w3": rng.normal(size=256) * scale, "b3": rng.normal(size=1) * 0.05}
    return {k: oracle.bf16(v.astype(np.float32)) for k, v in d.items()}


def features(seed, n):
    rng = np.random.default_rng(seed)
    x = rng.poisson(0.4, size=(n, 192)).astype(np.float32)
    x[:, 128:132] = rng.random((n, 4))
    return oracle.bf16(x)


def emulate(p, X, t, plant=None):
    """fp32 training step with bf16 rounding points (the device's contract)."""
    f = lambda a: torch.as_tensor(np.asarray(a, np.float32))
    b16 = lambda v: v.to(torch.bfloat16).to(torch.float32)
    x, w1, b1, w2, b2, w3, b3 = (f(v) for v in (X, p["w1"], p["b1"], p["w2"], p["b2"], p["w3"], p["b3"]))
    gel = lambda z: 0.5 * z * (1 + torch.erf(z * 0.7071067811865476))
    gp = lambda z: 0.5 * (1 + torch.erf(z * 0.7071067811865476)) + (
        0.0 if plant == "gelu_grad" else z * torch.exp(-0.5 * z * z) * 0.3989422804014327)
    n = x.shape[0]
    z1 = x @ w1 + (0.0 if plant == "bias" else b1)
    h1 = b16(gel(z1))
    z2 = h1 @ w2 + b2
    h2 = b16(gel(z2))
    y = h2 @ w3 + b3
    e = y - f(t)
    dy = e / n
    loss = float((0.5 * e * e).sum() / n)
    dz2 = b16(dy[:, None] * w3 * gp(z2))
    dz1 = b16((dz2 @ w2.T) * gp(z1))
    g = {"b3": dy.sum().reshape(1), "w3": dy @ h2, "b2": dz2.sum(0), "w2": h1.T @ dz2, "b1": dz1.sum(0),
         "w1": x.T @ dz1}
    g = {k: v.double().numpy() for k, v in g.items()}
    dev = {"z1": z1, "h1": h1, "z2": z2, "h2": h2, "y": y, "dy": dy, "dz2": dz2, "dz1": dz1}
    return dev, g, loss


def run(p, X, t, dev, g, loss):
    want_loss, orc, want_g = oracle.mlp_train_trace(p, X, t)
    d = mlp_chain.check_forward(p, X, dev, orc)
    mlp_chain.check_backward(p, X, t, dev, orc, d, loss, g, want_g, want_loss)


@pytest.fixture(scope="module")
def case():
    p, X = params(1), features(2, 512)
    t = (np.random.default_rng(3).random(512) * 0.5).astype(np.float32).astype(np.float64)
    return p, X, t


def test_emulated_step_passes(case):
    p, X, t = case
    run(p, X, t, *emulate(p, X, t))


@pytest.mark.parametrize("plant", ["sign", "rows", "gelu_grad", "bias"])
def test_planted_mistakes_fail(case, plant):
    p, X, t = case
    dev, g, loss = emulate(p, X, t, plant if plant in ("gelu_grad", "bias") else None)
    if plant == "sign":
        # flip the sign of one entry of w1's gradient (one of the larger ones)
        i, j = np.unravel_index(np.argsort(np.abs(g["w1"]).ravel())[-200], g["w1"].shape)
        g["w1"][i, j] = -g["w1"][i, j]
    elif plant == "rows":
        g["w2"][[10, 11]] = g["w2"][[11, 10]]
    with pytest.raises(AssertionError):
        run(p, X, t, dev, g, loss)
