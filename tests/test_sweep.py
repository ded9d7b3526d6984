"""Layout sweep (Eq. (1) reading): the utilisation and feasibility formulas
on hand-computed layouts and the Pareto filter (CPU); on the GPU, every
swept layout's mean plan lengths equal the oracle's on the same layout,
slotting and plans."""
import numpy as np
import pytest

import oracle
import wh_gen
from paper_2110_13693_gb300 import sweep


def test_utilisation_and_feasibility_by_hand():
    # 10 aisles, 30 slots of pitch 1, racks 1 deep, pitch 3 (aisle width 1), cross-aisles 2:
    # storage 10*2*1*30 = 600, floor 10*3*(30+4) = 1020
    assert sweep.utilisation(10, 30, 3, 1, 2, 1.0) == pytest.approx(600 / 1020)
    # wider aisles cost floor area
    assert sweep.utilisation(10, 30, 5, 1, 2, 1.0) < sweep.utilisation(10, 30, 3, 1, 2, 1.0)
    assert sweep.feasible(3, 1.0, 1.0, 1.0) and not sweep.feasible(3, 1.0, 1.5, 1.0)
    assert sweep.feasible(4, 1.0, 1.5, 1.0)


def test_pareto_front():
    rows = [{"utilisation": u, "mean_plan_optimal": d, "feasible": f}
            for u, d, f in [(0.5, 100, True), (0.6, 120, True), (0.55, 130, True), (0.7, 90, False),
                            (0.4, 100, True)]]
    front = sweep.pareto(rows)
    assert [(r["utilisation"], r["mean_plan_optimal"]) for r in front] == [(0.5, 100), (0.6, 120)]


@pytest.mark.gpu
def test_sweep_lengths_match_oracle(gpu_lib):
    inst = wh_gen.tiny(seed=5, n_plans=6)
    rows = sweep.layout_sweep(gpu_lib, inst, aisle_counts=[5, 10, 15], pitches=[3, 5], n_loc=600)
    assert len(rows) == 6
    for r in rows:
        lay = wh_gen.Layout(r["A"], r["L"], r["P"], 1, 2)
        slot = wh_gen.gen_slot_abc(1, lay, inst.n_sku, 0.0)
        cur = wh_gen.Instance(lay, inst.n_sku, inst.order_off, inst.line_sku, slot, inst.plan_tour_off,
                              inst.tour_off, inst.order_seq)
        _, _, ps, pr = oracle.eval_plans(cur)
        assert r["mean_plan_sshape"] == pytest.approx(ps.mean(), abs=1e-6)
        assert r["mean_plan_optimal"] == pytest.approx(pr.mean(), abs=1e-6)
