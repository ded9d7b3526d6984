"""Surrogate on the GPU against the oracle: features bit-exact; the forward
and one training step (every intermediate, the loss, every gradient entry,
the Adam update) element by element within bounds derived from the
arithmetic (tests/mlp_chain.py); training that actually reduces the error."""
import numpy as np
import pytest

import mlp_chain
import oracle
import wh_gen

pytestmark = pytest.mark.gpu


def tour_locs(inst, t, smap):
    locs = []
    for o in inst.order_seq[inst.tour_off[t]:inst.tour_off[t + 1]]:
        locs.extend(smap[inst.line_sku[inst.order_off[o]:inst.order_off[o + 1]]].tolist())
    return locs


def gpu_features(wh, inst, maps=None):
    import torch
    lay = wh.Layout.of(inst.layout)
    prob = wh.to_device(inst, slot_map=None if maps is None else maps.ravel(),
                        slot_map_stride=0 if maps is None else inst.n_sku)
    X = wh.features(lay, prob)
    torch.cuda.synchronize()
    assert lay.status() == 0
    lay.close()
    return X


@pytest.mark.parametrize("which", ["tiny", "midsize", "paperscale", "paperscale_maps"])
def test_features_bit_exact(gpu_lib, which):
    import torch
    if which == "tiny":
        inst, maps = wh_gen.tiny(seed=1, n_plans=6), None
    elif which == "midsize":
        inst, maps = wh_gen.midsize(seed=2, n_plans=6), None
    else:
        inst = wh_gen.paperscale(seed=3, n_plans=2)
        rng = np.random.default_rng(0)
        maps = None if which == "paperscale" else np.stack(
            [rng.permutation(inst.layout.n_loc)[: inst.n_sku] for _ in range(2)]).astype(np.int32)
    X = gpu_features(gpu_lib, inst, maps).view(torch.int16).cpu().numpy()
    for t in range(inst.n_tours):
        plan = int(np.searchsorted(inst.plan_tour_off, t, side="right") - 1)
        smap = inst.slot_map if maps is None else maps[plan]
        want = oracle.bf16(oracle.features(inst.layout, tour_locs(inst, t, smap)))
        want_bits = torch.from_numpy(want).to(torch.bfloat16).view(torch.int16).numpy()
        assert np.array_equal(X[t], want_bits), f"tour {t}"


def bf16_params(seed, scale=0.06):
    rng = np.random.default_rng(seed)
    d = {"w1": rng.normal(size=(192, 256)) * scale, "b1": rng.normal(size=256) * 0.05,
         "w2": rng.normal(size=(256, 256)) * scale, "b2": rng.normal(size=256) * 0.05,
         "w3": rng.normal(size=256) * scale, "b3": rng.normal(size=1) * 0.05}
    return {k: oracle.bf16(v.astype(np.float32)) for k, v in d.items()}


def batch(wh, n_plans=12):
    """Features (bf16, device) and normalised optimal costs of mid-size tours."""
    import torch
    inst = wh_gen.midsize(seed=4, n_plans=n_plans)
    X = gpu_features(wh, inst)
    _, tr, _, _ = oracle.eval_plans(inst)
    lay = inst.layout
    norm = 2 * (lay.n_aisles - 1) * lay.aisle_pitch + lay.n_aisles * (
        lay.cross_aisle_width + (lay.slots_per_side - 1) * lay.slot_pitch)
    return X, torch.as_tensor(tr / norm, dtype=torch.float32).cuda()


def forward_checked(wh, p, X, y_pred=None):
    """Run one training step of a fresh surrogate with parameters p on rows X
    (device bf16), read back its forward intermediates and check them layer
    by layer, element by element, against the oracle's trace (tests/mlp_chain:
    tolerances derived from fp32 accumulation, the device's elementary
    functions and the bf16 rounding points).  When the prediction y_pred of
    the same rows is given it must equal the training forward's outputs bit
    for bit: prediction and the training forward run the same tensor-core
    kernel arithmetic, row by row."""
    import torch
    s = wh.Surrogate(0)
    s.set_params(wh.pack_params(p))
    n = int(X.shape[0])
    t = torch.zeros(n, dtype=torch.float32, device=X.device)
    s.train_step(X, t, 1e-3)
    dev = s.trace(n)
    torch.cuda.synchronize()
    Xh = X.float().cpu().numpy()
    _, orc, _ = oracle.mlp_train_trace(p, Xh, np.zeros(n))
    mlp_chain.check_forward(p, Xh, dev, orc)
    if y_pred is not None:
        np.testing.assert_array_equal(y_pred.cpu().numpy(), dev["y"].cpu().numpy())
    assert s.status() == 0
    s.close()


def test_predict_matches_oracle(gpu_lib):
    wh = gpu_lib
    X, _ = batch(wh)
    p = bf16_params(1)
    s = wh.Surrogate(0)
    s.set_params(wh.pack_params(p))
    y = s.predict(X)
    assert s.status() == 0
    s.close()
    forward_checked(wh, p, X, y)


def rand_features(seed, n):
    """bf16 rows with the value ranges of tour features: small histogram
    counts and four scalars in [0, 1]."""
    rng = np.random.default_rng(seed)
    x = rng.poisson(0.4, size=(n, 192)).astype(np.float32)
    x[:, 128:132] = rng.random((n, 4))
    return oracle.bf16(x)


# one tile, a ragged tail, several tiles per CTA (phases wrap on every
# barrier), more tiles than SMs with a tail
@pytest.mark.parametrize("n", [1, 127, 128, 129, 1000, 152 * 128 * 3 + 77])
def test_tensor_core_predict_ragged(gpu_lib, n):
    import torch
    wh = gpu_lib
    Xh = rand_features(n, n)
    X = torch.from_numpy(Xh).to(torch.bfloat16).cuda()
    p = bf16_params(3)
    s = wh.Surrogate(0)
    s.set_params(wh.pack_params(p))
    y = s.predict(X)
    idx = np.arange(n) if n <= 1000 else np.unique(np.concatenate(
        [np.arange(200), np.arange(n - 200, n), np.random.default_rng(n).integers(0, n, 600)]))
    # a row-offset view (16-byte aligned) predicts the same rows
    if n > 8:
        y5 = s.predict(X[5:]).cpu().numpy()
        np.testing.assert_array_equal(y5, y[5:].cpu().numpy())
    assert s.status() == 0
    s.close()
    it = torch.as_tensor(idx).cuda()
    forward_checked(wh, p, X[it].contiguous(), y[it])


def test_tensor_core_predict_large(gpu_lib):
    import torch
    wh = gpu_lib
    n = (1 << 21) + 19
    g = torch.Generator(device="cuda").manual_seed(5)
    X = torch.randint(0, 3, (n, 192), device="cuda", generator=g).to(torch.bfloat16)
    X[:, 128:132] = torch.rand((n, 4), device="cuda", generator=g).to(torch.bfloat16)
    p = bf16_params(4)
    s = wh.Surrogate(0)
    s.set_params(wh.pack_params(p))
    y = s.predict(X)
    assert s.status() == 0
    s.close()
    idx = torch.cat([torch.arange(64), torch.arange(n - 64, n),
                     torch.randint(0, n, (256,), generator=torch.Generator().manual_seed(6))]).cuda()
    forward_checked(wh, p, X[idx].contiguous(), y[idx])


def test_predict_rejects_misaligned_rows(gpu_lib):
    import torch
    wh = gpu_lib
    flat = torch.zeros(192 * 9 + 1, dtype=torch.bfloat16, device="cuda")
    X = flat[1:].view(9, 192)                 # 2-byte offset
    s = wh.Surrogate(0)
    with pytest.raises(RuntimeError):
        s.predict(X)
    s.close()


@pytest.mark.parametrize("n", [1024, 4096 + 37])
def test_train_step_matches_oracle(gpu_lib, n):
    """One training step, element by element: forward intermediates, dy,
    the back-propagated dZ2 and dZ1, the loss and every gradient entry
    against the oracle's trace with derived per-element bounds
    (tests/mlp_chain); then the Adam update and the prediction with the
    updated weights."""
    import torch
    wh = gpu_lib
    X, t = batch(wh, n_plans=24)
    assert X.shape[0] >= n
    X, t = X[:n].contiguous(), t[:n].contiguous()
    p = bf16_params(2)
    s = wh.Surrogate(0)
    p0 = wh.pack_params(p)
    s.set_params(p0)
    loss = s.train_step(X, t, 1e-3)
    dev = s.trace(n)
    torch.cuda.synchronize()
    p1, g = s.params()
    Xh = X.float().cpu().numpy()
    th = t.cpu().numpy().astype(np.float64)
    want_loss, orc, want_g = oracle.mlp_train_trace(p, Xh, th)
    d = mlp_chain.check_forward(p, Xh, dev, orc)
    mlp_chain.check_backward(p, Xh, th, dev, orc, d, float(loss.item()), wh.unpack_params(g), want_g, want_loss)
    # Adam: the device step (fp32) equals the oracle's step (float64) on the
    # device's own gradients: |error| <= a few fp32 roundings of p and of the
    # step lr * m / (sqrt(v) + eps), which is at most lr in size
    q = p0.astype(np.float64)
    m, v = np.zeros_like(q), np.zeros_like(q)
    oracle.adam(q, m, v, g.astype(np.float64), 1e-3, 1)
    np.testing.assert_allclose(p1, q, rtol=4 * mlp_chain.U, atol=16 * mlp_chain.U * 1e-3)
    # prediction after the step uses the updated weights: w1, w2 as bf16,
    # the biases and w3 as fp32 master values
    p1d = wh.unpack_params(p1)
    w = {k: (oracle.bf16(v) if k in ("w1", "w2") else v) for k, v in p1d.items()}
    y1 = s.predict(X)
    s.close()
    forward_checked(wh, w, X, y1)


def test_training_reduces_error(gpu_lib):
    import torch
    wh = gpu_lib
    X, t = batch(wh, n_plans=96)
    n = X.shape[0]
    idx = torch.randperm(n, generator=torch.Generator().manual_seed(0)).cuda()
    train, held = idx[: n - 2000], idx[n - 2000:]
    s = wh.Surrogate(7)
    err0 = ((s.predict(X[held]) - t[held]).abs() / t[held].clamp_min(1e-6)).mean().item()
    g = torch.Generator(device="cuda").manual_seed(1)
    for step in range(400):
        b = train[torch.randint(0, train.numel(), (2048,), device="cuda", generator=g)]
        s.train_step(X[b].contiguous(), t[b].contiguous(), 2e-3)
    torch.cuda.synchronize()
    rel = ((s.predict(X[held]) - t[held]).abs() / t[held].clamp_min(1e-6))
    err1 = rel.mean().item()
    assert err1 < 0.5 * err0 and err1 < 0.15, (err0, err1)
    s.close()


def test_features_full_paperscale_sampled(gpu_lib):
    """Features of every tour of the 16,384-plan paper-scale population with
    per-plan slottings (2.7 M tours, the prescreen's workload); sampled rows
    bit-equal to the oracle's."""
    import torch
    wh = gpu_lib
    n_plans = 16384
    inst = wh_gen.paperscale(seed=4, n_plans=n_plans)
    lay = wh.Layout.of(inst.layout)
    base = wh.to_device(inst)
    prob = wh.DeviceProblem(base.order_off, base.line_sku, base.slot_map.repeat(n_plans), base.plan_tour_off,
                            base.tour_off, base.order_seq, inst.n_sku, inst.n_sku)
    X = wh.features(lay, prob).view(torch.int16)
    assert lay.status() == 0
    rng = np.random.default_rng(1)
    rows = np.concatenate([[0, inst.n_tours - 1], rng.integers(0, inst.n_tours, 300)])
    got = X[torch.as_tensor(rows).cuda()].cpu().numpy()
    for r, t in enumerate(rows):
        want = oracle.bf16(oracle.features(inst.layout, tour_locs(inst, int(t), inst.slot_map)))
        assert np.array_equal(got[r], torch.from_numpy(want).to(torch.bfloat16).view(torch.int16).numpy()), t
    lay.close()


def test_bounded_wait_runs_out_and_context_stays_usable(gpu_lib):
    """The tensor-core kernel's failure path: with the producer stopped
    before one tile and a 200-microsecond wait limit, the wait for that tile
    runs out; the kernel returns, the status word reports WH_STATUS_TIMEOUT,
    and the next normal predictions on the same context are exact again."""
    import torch
    wh = gpu_lib
    sms = torch.cuda.get_device_properties(0).multi_processor_count   # one CTA per SM
    n = sms * 128 * 2 + 5
    Xh = rand_features(7, n)
    X = torch.from_numpy(Xh).to(torch.bfloat16).cuda()
    s = wh.Surrogate(0)
    s.set_params(wh.pack_params(bf16_params(5)))
    y0 = s.predict(X).clone()
    assert s.status() == 0
    for skip in (0, sms + 1):      # the first tile of CTA 0; the second tile of CTA 1
        y = torch.zeros(n, dtype=torch.float32, device="cuda")
        wh.wh_surrogate_predict_timeout_test(s.handle, X.data_ptr(), n, y.data_ptr(), skip, 200000)
        torch.cuda.synchronize()
        assert s.status() & wh.WH_STATUS_TIMEOUT
        # tiles of the other CTAs were scored as usual
        other = torch.arange(n, device="cuda") // 128 % sms != skip % sms
        assert torch.equal(y[other], y0[other])
        y1 = s.predict(X)
        torch.cuda.synchronize()
        assert s.status() == 0
        assert torch.equal(y1, y0)
    s.close()
