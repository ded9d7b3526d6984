"""K-means slotting on the GPU against the oracle: features, seeds (given or
K-means++), centroids, assignment and slotting all bit-exact (every step is
integer arithmetic), on the category workloads and on edge cases."""
import numpy as np
import pytest

import oracle
import wh_gen

pytestmark = pytest.mark.gpu


def draws(seed, k):
    return np.array([wh_gen.stream_word(seed, 11, i) for i in range(k)], np.uint64)


def run(wh, inst, signs, k, iters, fw, init=None, u=None):
    import torch
    lay = wh.Layout.of(inst.layout)
    prob = wh.to_device(inst)
    sg = torch.as_tensor(signs).cuda()
    ini = None if init is None else torch.as_tensor(np.asarray(init, np.int32)).cuda()
    uu = None if u is None else torch.as_tensor(u.view(np.int64)).cuda()
    out = lay.kmeans_slotting(prob, sg, k, iters, fw, init=ini, u=uu)
    torch.cuda.synchronize()
    st = lay.status()
    lay.close()
    return [t.cpu().numpy() for t in out], st


def check(wh, inst, k, iters, fw, init=None, useed=5, sseed=3):
    signs = wh_gen.gen_signs(sseed, (inst.n_sku, 32))
    u = None if init is not None else draws(useed, k)
    (x, seeds, cent, assign, smap), st = run(wh, inst, signs, k, iters, fw, init, u)
    assert st == 0
    wx, wseeds, wcent, wassign, wsmap = oracle.kmeans_slotting(inst.layout, inst.order_off, inst.line_sku,
                                                                inst.n_sku, signs, fw, k, iters, init=init, u=u)
    assert np.array_equal(x, wx)
    assert np.array_equal(seeds, wseeds)
    assert np.array_equal(cent, wcent)
    assert np.array_equal(assign, wassign)
    assert np.array_equal(smap, wsmap)
    return smap


@pytest.mark.parametrize("k,iters,fw", [(64, 20, 64), (16, 5, 0), (200, 8, 256), (1, 3, 64)])
def test_midsize_categories(gpu_lib, k, iters, fw):
    inst = wh_gen.midsize_cat(seed=6, n_plans=1)
    check(gpu_lib, inst, k, iters, fw)


def test_given_seeds_and_zero_iterations(gpu_lib):
    inst = wh_gen.midsize_cat(seed=6, n_plans=1)
    rng = np.random.default_rng(2)
    init = rng.choice(inst.n_sku, 48, replace=False).astype(np.int32)
    check(gpu_lib, inst, 48, 0, 32, init=init)
    check(gpu_lib, inst, 48, 12, 32, init=init)


def test_paperscale_categories(gpu_lib):
    """50,000 SKUs in 256 categories over 200,000 locations, 256 clusters."""
    inst = wh_gen.paperscale_cat(seed=7, n_plans=1)
    check(gpu_lib, inst, 256, 6, 64)


def test_tiny_uniform_orders(gpu_lib):
    inst = wh_gen.tiny(seed=2, n_plans=1)          # 600 SKUs, many never ordered
    check(gpu_lib, inst, 24, 10, 64)
    check(gpu_lib, inst, 256, 4, 1)


def test_slotting_scores_like_the_oracle(gpu_lib):
    """The K-means slotting fed to the evaluator: the same plan costs as the
    oracle's evaluation under the oracle's slotting."""
    import torch
    inst = wh_gen.midsize_cat(seed=6, n_plans=16)
    smap = check(gpu_lib, inst, 64, 10, 64)
    lay = gpu_lib.Layout.of(inst.layout)
    prob = gpu_lib.to_device(inst, slot_map=smap)
    costs = gpu_lib.evaluate(lay, prob)
    torch.cuda.synchronize()
    lay.close()
    want = oracle.eval_plans(inst, slot_map=smap)
    assert np.array_equal(costs.plan_rr[:inst.n_plans].cpu().numpy(), want[3])
    assert np.array_equal(costs.plan_s[:inst.n_plans].cpu().numpy(), want[2])


def test_bad_ids_flagged(gpu_lib):
    inst = wh_gen.tiny(seed=2, n_plans=1)
    bad = wh_gen.Instance(inst.layout, inst.n_sku, inst.order_off, inst.line_sku.copy(), inst.slot_map,
                          inst.plan_tour_off, inst.tour_off, inst.order_seq)
    bad.line_sku[3] = inst.n_sku + 5
    signs = wh_gen.gen_signs(1, (inst.n_sku, 32))
    _, st = run(gpu_lib, bad, signs, 8, 2, 64, u=draws(1, 8))
    assert st & gpu_lib.WH_STATUS_BAD_SKU
    init = np.array([0, 1, inst.n_sku], np.int32)
    _, st = run(gpu_lib, inst, signs, 3, 2, 64, init=init)
    assert st & gpu_lib.WH_STATUS_BAD_SKU


def test_argument_errors(gpu_lib):
    import torch
    inst = wh_gen.tiny(seed=2, n_plans=1)
    lay = gpu_lib.Layout.of(inst.layout)
    prob = gpu_lib.to_device(inst)
    sg = torch.as_tensor(wh_gen.gen_signs(1, (inst.n_sku, 32))).cuda()
    u = torch.zeros(300, dtype=torch.int64, device="cuda")
    with pytest.raises(gpu_lib.WhError):
        lay.kmeans_slotting(prob, sg, 257, 2, 64, u=u)              # more than 256 clusters
    with pytest.raises(gpu_lib.WhError):
        lay.kmeans_slotting(prob, sg, 8, 2, 257, u=u)               # frequency weight above 256
    with pytest.raises(gpu_lib.WhError):
        lay.kmeans_slotting(prob, sg, 8, -1, 64, u=u)
    small = gpu_lib.Layout(2, 10)                                   # fewer locations than SKUs
    with pytest.raises(gpu_lib.WhError):
        small.kmeans_slotting(prob, sg, 8, 2, 64, u=u)
    small.close()
    lay.close()
