"""Element-wise comparison of the device's MLP training step with the
oracle's, layer by layer, with per-element tolerances derived from the
arithmetic (no tolerance is a tuned constant).

The contract (bf16 weights and activations on the tensor cores, fp32
accumulation; the learned prescreen of config 5): every product operand is a
bf16 value, every sum is accumulated in fp32.  The oracle (``mlp_train_trace``)
computes the same step in float64 with the same bf16 rounding points
(activations h1, h2; back-propagated gradients d2 = dL/dz2, d1 = dL/dz1).  The
two can differ only through

* fp32 accumulation: a sum of k terms carries at most ``acc(k) * M`` of error,
  M the sum of the terms' magnitudes (2u per addition, u = 2^-24: a rounding
  adder gives u, a truncating tensor-core adder at most 2u);
* the device's elementary functions: GELU with erf by Abramowitz & Stegun
  7.1.28 (|error| <= 3e-7) evaluated in fp32 (its 16th power and reciprocal
  add at most ~120u), GELU' with fp32 erff and the fast exponential;
* a bf16 rounding point where the device's and the oracle's values before
  rounding straddle a rounding boundary: the rounded values then differ by
  one bf16 step.  Rounding is monotone, so the device's bf16 value must lie
  between the roundings of (oracle value - D) and (oracle value + D), D the
  bound on the pre-rounding difference; anywhere else it must be equal.

Each layer is checked on the device's own inputs to it, and the tolerance of
the next layer carries the actual differences of those inputs forward exactly
(their effect computed in float64) plus the accumulation bound.  The final
tolerance of every gradient entry is therefore
``|G(device operands) - G(oracle operands)| + acc(k) * M`` with both G's exact
sums, the first term bounded by the (checked) per-operand differences.
"""
import numpy as np
import torch

U = 2.0 ** -24          # fp32 unit roundoff
GELU_D1 = 1.13          # max |gelu'(z)|
GELU_D2 = 0.8           # max |gelu''(z)| = 2 phi(0)


def acc(k):
    return 2.0 * k * U


def eps_gelu(z):
    """Device GELU vs exact: the device evaluates relu(z) - |z| Q(|z|)^-16
    (Abramowitz & Stegun 7.1.28 folded into one expression): the
    approximation itself is off by at most 1.5e-7 |z|, and its fp32
    evaluation by at most 66u |z| (7u on Q from the Horner chain over
    positive terms and the rounded coefficients, 127u after the four
    squarings, 129u after the reciprocal, 130u after the product with |z|
    on a term of at most |z|/2, u |z| for the final fma)."""
    return np.abs(z) * (2e-7 + 68.0 * U)


def eps_gelu_grad(z):
    return 32.0 * U * np.ones_like(z)


def bf16_round(v):
    """float64 -> float32 (nearest) -> bf16 (nearest even): monotone."""
    return torch.from_numpy(np.asarray(v, np.float64)).to(torch.float32).to(torch.bfloat16).to(
        torch.float64).numpy()


def f64(t):
    return t.detach().to(torch.float64).cpu().numpy()


def check_rounded(name, dev, pre_oracle, D):
    """dev (bf16 values) within the roundings of pre_oracle -/+ D."""
    lo, hi = bf16_round(pre_oracle - D), bf16_round(pre_oracle + D)
    bad = np.nonzero((dev < lo) | (dev > hi))
    assert bad[0].size == 0, (f"{name}: {bad[0].size} entries outside their rounding interval, first "
                              f"{[tuple(int(i) for i in b[:3]) for b in bad]}: dev {dev[bad][:3]}, "
                              f"oracle pre-rounding {pre_oracle[bad][:3]}, bound {D[bad][:3]}")


def check_close(name, dev, want, tol):
    err = np.abs(dev - want)
    bad = np.nonzero(err > tol * (1 + 1e-9) + 1e-300)
    assert bad[0].size == 0, (f"{name}: {bad[0].size} entries beyond their bound, first "
                              f"{[tuple(int(i) for i in b[:3]) for b in bad]}: dev {dev[bad][:3]}, "
                              f"oracle {want[bad][:3]}, bound {tol[bad][:3]}")


def check_forward(p, X, dev, orc):
    """z1, h1, z2, h2, y of the device (dict of tensors) against the oracle's
    trace; returns the float64 device values and the differences for the
    backward check."""
    w1, b1, w2, b2 = (np.asarray(p[k], np.float64) for k in ("w1", "b1", "w2", "b2"))
    w3, b3 = np.asarray(p["w3"], np.float64), float(np.asarray(p["b3"]).reshape(-1)[0])
    X = np.asarray(X, np.float64)
    d = {k: f64(dev[k]) for k in ("z1", "h1", "z2", "h2", "y")}
    # layer 1: K = 192 exact bf16 products plus the bias
    M1 = np.abs(b1) + np.abs(X) @ np.abs(w1)
    check_close("z1", d["z1"], orc["z1"], acc(193) * M1)
    from scipy.special import erf
    gel = lambda z: 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))
    dz1 = np.abs(d["z1"] - orc["z1"])
    check_rounded("h1", d["h1"], gel(orc["z1"]), GELU_D1 * dz1 + eps_gelu(orc["z1"]))
    # layer 2 on the device's h1: the h1 differences carried exactly
    M2 = np.abs(b2) + np.abs(d["h1"]) @ np.abs(w2)
    tol_z2 = np.abs((d["h1"] - orc["h1"]) @ w2) + acc(257) * M2
    check_close("z2", d["z2"], orc["z2"], tol_z2)
    dz2 = np.abs(d["z2"] - orc["z2"])
    check_rounded("h2", d["h2"], gel(orc["z2"]), GELU_D1 * dz2 + eps_gelu(orc["z2"]))
    # output
    M3 = abs(b3) + np.abs(d["h2"]) @ np.abs(w3)
    tol_y = np.abs((d["h2"] - orc["h2"]) @ w3) + acc(258) * M3
    check_close("y", d["y"], orc["y"], tol_y)
    return d


def check_backward(p, X, t, dev, orc, d, loss_dev, g_dev, g_orc, loss_orc):
    """dy, dZ2, dZ1, the loss and every gradient entry."""
    n = X.shape[0]
    w2, w3 = np.asarray(p["w2"], np.float64), np.asarray(p["w3"], np.float64)
    X = np.asarray(X, np.float64)
    t = np.asarray(t, np.float64)
    dy, dz2, dz1 = f64(dev["dy"]), f64(dev["dz2"]), f64(dev["dz1"])
    dyo = orc["dy"]
    # dy = (y - t) / n in fp32 (one subtraction, one fast division: 2 ulp)
    ey = np.abs(d["y"] - orc["y"])
    check_close("dy", dy, dyo, ey / n + 6 * U * (np.abs(dyo) + ey / n))
    # loss = sum 0.5 e^2 / n (fp32, any order)
    e_d, e_o = d["y"] - t, orc["y"] - t
    tol_loss = np.sum(0.5 * np.abs(e_d - e_o) * np.abs(e_d + e_o)) / n + acc(n + 8) * np.sum(0.5 * e_d ** 2) / n
    check_close("loss", np.array([loss_dev]), np.array([loss_orc]), np.array([tol_loss]))
    # dZ2 = bf16(dy * w3 * gelu'(z2)) on the device's dy and z2
    from scipy.special import erf
    gprime = lambda z: 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)
    dzz2 = np.abs(d["z2"] - orc["z2"])
    D2 = (np.abs(dy - dyo)[:, None] * np.abs(w3 * gprime(orc["z2"]))
          + np.abs(dy[:, None] * w3) * (GELU_D2 * dzz2 + eps_gelu_grad(orc["z2"]))
          + 4 * U * np.abs(orc["d2pre"]))
    check_rounded("dZ2", dz2, orc["d2pre"], D2)
    # dZ1 = bf16((dZ2 W2^T) * gelu'(z1)) on the device's dZ2 and z1
    s1_dev_exact = dz2 @ w2.T
    Ms = np.abs(dz2) @ np.abs(w2.T)
    ds1 = np.abs(s1_dev_exact - orc["s1"]) + acc(257) * Ms
    dzz1 = np.abs(d["z1"] - orc["z1"])
    D1 = (ds1 * GELU_D1 + (np.abs(orc["s1"]) + ds1) * (GELU_D2 * dzz1 + eps_gelu_grad(orc["z1"]))
          + 4 * U * np.abs(orc["d1pre"]))
    check_rounded("dZ1", dz1, orc["d1pre"], D1)
    # gradients: exact sums over the device's (checked) operands against the
    # oracle's, plus fp32 accumulation over the batch (and its split reduction)
    k = n + 64
    H1o, H2o = orc["h1"], orc["h2"]
    tol = {
        "b3": np.abs(np.array([dy.sum() - dyo.sum()])) + acc(k) * np.abs(dy).sum(),
        "w3": np.abs(dy @ d["h2"] - dyo @ H2o) + acc(k) * (np.abs(dy) @ np.abs(d["h2"])),
        "b2": np.abs(dz2.sum(0) - orc["d2"].sum(0)) + acc(k) * np.abs(dz2).sum(0),
        "w2": np.abs(d["h1"].T @ dz2 - H1o.T @ orc["d2"]) + acc(k) * (np.abs(d["h1"]).T @ np.abs(dz2)),
        "b1": np.abs(dz1.sum(0) - orc["d1"].sum(0)) + acc(k) * np.abs(dz1).sum(0),
        "w1": np.abs(X.T @ (dz1 - orc["d1"])) + acc(k) * (np.abs(X).T @ np.abs(dz1)),
    }
    for name in ("b3", "w3", "b2", "w2", "b1", "w1"):
        got = np.asarray(g_dev[name], np.float64).reshape(tol[name].shape)
        check_close("grad " + name, got, np.asarray(g_orc[name]).reshape(tol[name].shape), tol[name])
