"""The benchmark's accounting on the host: the algorithmic counts behind its
roofline fractions, recounted here with plain loops over a generated
instance, and the JSON line of its reference arm (the oracle on the host
cores), which needs no GPU."""
import json
import os
import subprocess
import sys

import numpy as np

import wh_gen

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _tours(inst):
    for t in range(inst.n_tours):
        lines = []
        for o in inst.order_seq[inst.tour_off[t]:inst.tour_off[t + 1]]:
            lines.extend(range(int(inst.order_off[o]), int(inst.order_off[o + 1])))
        yield lines


def test_dp_ops_count_every_aisle_up_to_the_rightmost_pick():
    """Sum over tours of (rightmost pick aisle + 1) x 77."""
    inst = wh_gen.tiny(seed=21, n_plans=6)
    L = inst.layout.slots_per_side
    want = 0
    for lines in _tours(inst):
        aisles = [int(inst.slot_map[inst.line_sku[l]]) // (2 * L) for l in lines]
        if aisles:
            want += (max(aisles) + 1) * 77
    assert bench.dp_alg_ops(inst) == want > 0


def test_dp_ops_with_empty_orders_and_tours():
    """An empty order adds no aisle and an empty tour counts nothing."""
    inst = wh_gen.tiny(seed=22, n_plans=3)
    off = np.asarray(inst.order_off).copy()
    # empty the first order (its lines go to the second) and add an empty tour
    off[1] = off[0]
    inst.order_off = off
    to = np.asarray(inst.tour_off)
    inst.tour_off = np.concatenate([to, to[-1:]])
    inst.plan_tour_off = np.asarray(inst.plan_tour_off).copy()
    inst.plan_tour_off[-1] += 1
    L = inst.layout.slots_per_side
    want = 0
    for lines in _tours(inst):
        if lines:
            want += (max(int(inst.slot_map[inst.line_sku[l]]) // (2 * L) for l in lines) + 1) * 77
    assert bench.dp_alg_ops(inst) == want


def test_algorithmic_bytes():
    """4 B per line of every tour, 4 B per tour offset, 4 B per tour and rule
    written, 8 B per plan and rule, 4 B per SKU of the slotting."""
    inst = wh_gen.tiny(seed=23, n_plans=5)
    lines = sum(len(x) for x in _tours(inst))
    T, P = inst.n_tours, inst.n_plans
    assert bench.algorithmic_bytes(inst) == 4 * lines + 4 * (T + 1) + 2 * 4 * T + 2 * 8 * P + 4 * inst.n_sku
    assert bench.algorithmic_bytes_one_rule(inst) == 4 * lines + 4 * (T + 1) + 4 * T + 8 * P + 4 * inst.n_sku


def test_reference_arm_json_line():
    """`bench.py --impl reference`: one JSON line, the oracle timed on the
    host cores, with the contract's keys and zero copy bytes."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads(out.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["value"] > 0 and d["unit"] == "tours/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "tours/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
