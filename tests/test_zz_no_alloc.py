"""wh_eval_plans_noalloc against wh_eval_plans and the CPU oracle.

The no-allocation entry point exists for callers that may not let a library
call cudaMalloc / cudaFree (a serving process whose device memory is all
reserved by its own pool, or a loop that cannot afford the synchronisation an
allocation can cause).  It must return exactly what wh_eval_plans returns, and
both must equal the oracle, under every routing mask, with one shared
slotting or one slotting per plan, with or without a caller status word, on
two calls in a row (the second sees the first call's leftovers in the shared
array).  This file is collected last so that a run stopping at the first
failure has already run every other test; it also passes when run on its own.
"""
import numpy as np
import pytest

import oracle
import wh_gen

pytestmark = pytest.mark.gpu

PREFILL = -12345


def _per_plan_maps(inst, seed):
    rng = np.random.default_rng(seed)
    maps = np.stack([rng.permutation(inst.layout.n_loc)[: inst.n_sku] for _ in range(inst.n_plans)])
    return np.ascontiguousarray(maps.astype(np.int32).ravel())


def _outputs(costs, prob):
    return [t.cpu().numpy() for t in (costs.tour_s[:prob.n_tours], costs.tour_rr[:prob.n_tours],
                                      costs.plan_s[:prob.n_plans], costs.plan_rr[:prob.n_plans])]


def _fresh_costs(wh, prob):
    costs = wh.alloc_costs(prob.n_tours, prob.n_plans)
    for t in (costs.tour_s, costs.tour_rr, costs.plan_s, costs.plan_rr):
        t.fill_(PREFILL)
    return costs


def _check(got, want, mask, what):
    names = ("tour_s", "tour_rr", "plan_s", "plan_rr")
    for i, (n, g, w) in enumerate(zip(names, got, want)):
        rule = 1 if i in (0, 2) else 2
        if mask & rule:
            bad = np.nonzero(g != w)[0]
            assert bad.size == 0, f"{what}: {n} differs at {bad[:5]}: got {g[bad[:5]]} want {w[bad[:5]]}"
        else:
            assert (g == PREFILL).all(), f"{what}: {n} written although mask {mask} leaves it out"


WORKLOADS = {
    "tiny": lambda: wh_gen.tiny(seed=1),
    "midsize": lambda: wh_gen.midsize(seed=2, n_plans=128),
    "paperscale": lambda: wh_gen.paperscale(seed=4, n_plans=6),
}


@pytest.mark.parametrize("slotting", ["shared", "per_plan"])
@pytest.mark.parametrize("mask", [1, 2, 3])
@pytest.mark.parametrize("name", list(WORKLOADS))
def test_noalloc_matches_eval_plans_and_oracle_twice(gpu_lib, name, mask, slotting):
    import torch
    wh = gpu_lib
    inst = WORKLOADS[name]()
    if slotting == "per_plan":
        maps = _per_plan_maps(inst, 7)
        stride = inst.n_sku
        want = oracle.eval_plans(inst, slot_map=maps, slot_map_stride=stride)
        prob = wh.to_device(inst, slot_map=maps, slot_map_stride=stride)
    else:
        want = oracle.eval_plans(inst)
        prob = wh.to_device(inst)
    # the allocating entry point on the same device inputs
    lay = wh.Layout.of(inst.layout)
    ref_costs = _fresh_costs(wh, prob)
    lay.eval_plans(prob, ref_costs, mask)
    torch.cuda.synchronize()
    assert lay.status() == 0
    lay.close()
    ref = _outputs(ref_costs, prob)
    _check(ref, want, mask, "wh_eval_plans vs oracle")

    lo = inst.layout
    desc = wh.wh_layout_desc(lo.n_aisles, lo.slots_per_side, lo.aisle_pitch, lo.slot_pitch, lo.cross_aisle_width)
    # one case per workload runs without a status word (NULL)
    use_status = not (mask == 3 and slotting == "per_plan")
    status = torch.full((1,), 0xFFFF, dtype=torch.int32, device="cuda")
    for call in range(2):
        costs = _fresh_costs(wh, prob)
        wh.wh_eval_plans_noalloc(desc, prob.orders(), prob.plans(), mask, costs.c(),
                                 status.data_ptr() if use_status else 0)
        torch.cuda.synchronize()
        if use_status:
            assert int(status.item()) == 0, f"call {call}: status {status.item()}"
        got = _outputs(costs, prob)
        _check(got, ref, mask, f"call {call} vs wh_eval_plans")
        _check(got, want, mask, f"call {call} vs oracle")


def test_noalloc_status_word_is_cleared_between_calls(gpu_lib):
    """A call that finds a bad SKU id sets a status bit; the next clean call
    on the same word reports 0 again, and the bad tours cost -1."""
    import torch
    wh = gpu_lib
    inst = wh_gen.tiny(seed=3, n_plans=4)
    lo = inst.layout
    desc = wh.wh_layout_desc(lo.n_aisles, lo.slots_per_side, lo.aisle_pitch, lo.slot_pitch, lo.cross_aisle_width)
    bad_lines = inst.line_sku.copy()
    bad_lines[0] = inst.n_sku + 5
    bad = wh_gen.Instance(inst.layout, inst.n_sku, inst.order_off, bad_lines, inst.slot_map,
                          inst.plan_tour_off, inst.tour_off, inst.order_seq)
    status = torch.zeros((1,), dtype=torch.int32, device="cuda")
    prob = wh.to_device(bad)
    costs = _fresh_costs(wh, prob)
    wh.wh_eval_plans_noalloc(desc, prob.orders(), prob.plans(), 3, costs.c(), status.data_ptr())
    torch.cuda.synchronize()
    assert int(status.item()) & wh.WH_STATUS_BAD_SKU
    assert (costs.tour_rr[:prob.n_tours] == -1).any()
    prob = wh.to_device(inst)
    costs = _fresh_costs(wh, prob)
    wh.wh_eval_plans_noalloc(desc, prob.orders(), prob.plans(), 3, costs.c(), status.data_ptr())
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    _check(_outputs(costs, prob), oracle.eval_plans(inst), 3, "clean call after a bad one")


def test_noalloc_rejects_sizes_beyond_its_limit(gpu_lib):
    wh = gpu_lib
    desc = wh.wh_layout_desc(10, 30, 3, 1, 2)
    o = wh.wh_orders(1, wh.WH_NOALLOC_MAX_LINES + 1, 10, 8, 8)
    p = wh.wh_plans(1, 1, 1, 8, 0, 8, 8, 8)
    with pytest.raises(wh.WhError) as e:
        wh.wh_eval_plans_noalloc(desc, o, p, 3, wh.wh_costs(0, 0, 0, 0))
    assert e.value.code == wh.WH_ERANGE
    p = wh.wh_plans(1, wh.WH_NOALLOC_MAX_TOURS + 1, 1, 8, 0, 8, 8, 8)
    o = wh.wh_orders(1, 1, 10, 8, 8)
    with pytest.raises(wh.WhError) as e:
        wh.wh_eval_plans_noalloc(desc, o, p, 3, wh.wh_costs(0, 0, 0, 0))
    assert e.value.code == wh.WH_ERANGE
