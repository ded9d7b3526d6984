"""wh_eval_plans_noalloc against wh_eval_plans.

The no-allocation entry point exists for callers that may not let a library
call cudaMalloc / cudaFree (a serving process whose device memory is all
reserved by its own pool, or a loop that cannot afford the synchronisation an
allocation can cause).  It must return exactly what wh_eval_plans returns.
This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes when run on its own.
"""
import numpy as np
import pytest

import wh_gen

pytestmark = pytest.mark.gpu


def _reference(wh, inst):
    import torch
    lay = wh.Layout.of(inst.layout)
    prob = wh.to_device(inst)
    costs = wh.evaluate(lay, prob, mask=3)
    torch.cuda.synchronize()
    assert lay.status() == 0
    lay.close()
    return prob, [t.cpu().numpy() for t in (costs.tour_s[:prob.n_tours], costs.tour_rr[:prob.n_tours],
                                           costs.plan_s[:prob.n_plans], costs.plan_rr[:prob.n_plans])]


@pytest.mark.parametrize("make", [lambda: wh_gen.tiny(seed=1),
                                  lambda: wh_gen.midsize(seed=2, n_plans=128),
                                  lambda: wh_gen.paperscale(seed=4, n_plans=6)])
def test_noalloc_matches_eval_plans_twice(gpu_lib, make):
    import torch
    wh = gpu_lib
    inst = make()
    prob, want = _reference(wh, inst)
    lay = inst.layout
    desc = wh.wh_layout_desc(lay.n_aisles, lay.slots_per_side, lay.aisle_pitch, lay.slot_pitch,
                             lay.cross_aisle_width)
    status = torch.full((1,), 0xFFFF, dtype=torch.int32, device="cuda")
    for call in range(2):
        costs = wh.alloc_costs(prob.n_tours, prob.n_plans)
        for t in (costs.tour_s, costs.tour_rr, costs.plan_s, costs.plan_rr):
            t.fill_(-12345)
        wh.wh_eval_plans_noalloc(desc, prob.orders(), prob.plans(), 3, costs.c(), status.data_ptr())
        torch.cuda.synchronize()
        assert int(status.item()) == 0, f"call {call}: status {status.item()}"
        got = [t.cpu().numpy() for t in (costs.tour_s[:prob.n_tours], costs.tour_rr[:prob.n_tours],
                                         costs.plan_s[:prob.n_plans], costs.plan_rr[:prob.n_plans])]
        for g, w in zip(got, want):
            assert np.array_equal(g, w), f"call {call} differs from wh_eval_plans"


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
