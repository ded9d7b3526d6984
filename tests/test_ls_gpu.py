"""Local search on the GPU step by step against the oracle: the same moves
give the same applied indices, identical edited plans (order sequences, tour
offsets, slottings) and identical costs after every step."""
import numpy as np
import pytest

import oracle
import wh_gen

pytestmark = pytest.mark.gpu


def occupancy_bits(maps, n_loc):
    words = (n_loc + 31) // 32
    out = np.zeros((maps.shape[0], words), np.uint32)
    for p in range(maps.shape[0]):
        for loc in maps[p]:
            out[p, loc >> 5] |= np.uint32(1 << (int(loc) & 31))
    return out.view(np.int32).ravel()


def run(wh, inst, steps, M, max_orders, max_lines=0, per_plan_maps=False, seed=9, reloc=0, maps=None):
    import torch
    n = inst.n_plans
    stride = inst.n_sku if per_plan_maps else 0
    if maps is not None:
        smap = maps.ravel().astype(np.int32)
    else:
        smap = np.tile(inst.slot_map, (n, 1)).ravel().astype(np.int32) if per_plan_maps else inst.slot_map.copy()
    lay = wh.Layout.of(inst.layout)
    prob = wh.to_device(inst, slot_map=smap, slot_map_stride=stride)
    if reloc:
        lay.occupancy(prob)
    costs = wh.evaluate(lay, prob)
    cur = wh_gen.Instance(inst.layout, inst.n_sku, inst.order_off, inst.line_sku, smap, inst.plan_tour_off,
                          inst.tour_off.copy(), inst.order_seq.copy())
    for step in range(steps):
        mv = wh_gen.gen_moves(seed, step, cur, M - reloc)
        if reloc:
            mv = np.concatenate([mv, wh_gen.gen_relocations(seed + 1, step, cur, reloc)], axis=1)
        mv[..., 3] = np.arange(n)[:, None]
        mv = mv.reshape(-1, 4)
        to, seq, sm2, applied = oracle.ls_step(cur, mv, M, max_orders, max_lines, slot_map=cur.slot_map,
                                               slot_map_stride=stride)
        got = lay.ls_step(prob, costs, torch.as_tensor(mv).cuda(), M, max_orders, max_lines).cpu().numpy()
        torch.cuda.synchronize()
        assert np.array_equal(got, applied), f"step {step}: applied differs"
        assert np.array_equal(prob.tour_off.cpu().numpy(), to), f"step {step}: tour_off differs"
        assert np.array_equal(prob.order_seq.cpu().numpy(), seq), f"step {step}: order_seq differs"
        assert np.array_equal(prob.slot_map.cpu().numpy(), sm2), f"step {step}: slotting differs"
        if reloc:
            want_bits = occupancy_bits(sm2.reshape(n, -1), inst.layout.n_loc)
            assert np.array_equal(prob.loc_used.cpu().numpy(), want_bits), f"step {step}: occupancy differs"
        cur = wh_gen.Instance(inst.layout, inst.n_sku, inst.order_off, inst.line_sku, sm2, inst.plan_tour_off,
                              to, seq)
        want = oracle.eval_plans(cur, slot_map=sm2, slot_map_stride=stride)
        assert np.array_equal(costs.plan_rr[:n].cpu().numpy(), want[3])
        assert np.array_equal(costs.tour_rr[:prob.n_tours].cpu().numpy(), want[1])
    assert lay.status() == 0
    lay.close()
    return cur


def test_tiny_trajectory_shared_slotting(gpu_lib):
    run(gpu_lib, wh_gen.tiny(seed=13, n_plans=6), steps=5, M=32, max_orders=8)


def test_tiny_trajectory_per_plan_slottings(gpu_lib):
    run(gpu_lib, wh_gen.tiny(seed=14, n_plans=5), steps=5, M=32, max_orders=8, per_plan_maps=True)


def test_paperscale_trajectory(gpu_lib):
    run(gpu_lib, wh_gen.paperscale(seed=15, n_plans=2), steps=3, M=16, max_orders=24, per_plan_maps=True)


def test_trajectory_with_relocations(gpu_lib):
    """tiny's orders on a half-empty 20 x 30 layout, per-plan random
    slottings, a third of the moves relocations into empty locations; the
    occupancy bits follow every applied relocation."""
    base = wh_gen.tiny(seed=16, n_plans=5)
    lay = wh_gen.Layout(20, 30)
    inst = wh_gen.Instance(lay, base.n_sku, base.order_off, base.line_sku, base.slot_map, base.plan_tour_off,
                           base.tour_off, base.order_seq)
    rng = np.random.default_rng(16)
    maps = np.stack([rng.permutation(lay.n_loc)[:inst.n_sku] for _ in range(5)]).astype(np.int32)
    run(gpu_lib, inst, steps=6, M=48, max_orders=8, per_plan_maps=True, reloc=16, maps=maps)
