"""Layout sweep (subsystem 1 of the paper, Eq. (1): warehouse utilisation
against the aisle design variable), scored by the exact evaluator.

Reading of Eq. (1) (the printed symbols are incomplete): a layout of A
aisles with L slots per side at slot pitch S, racks of depth r on both sides
of every aisle (back to back between neighbouring aisles, so the aisle pitch
P is the aisle width w plus 2r) and front and back cross-aisles of width W.

    storage area   A_ind = A * 2r * L*S
    floor area     A_max = A*P * (L*S + 2W)
    utilisation    A_ind / A_max = 2r L S / (P (L S + 2W))
    constraint     w = P - 2r >= k * delta   (the aisle fits a picker of
                   width delta with safety factor k: k*delta - w <= 0)

For every (A, P) of the sweep the location count stays near `n_loc` (L =
n_loc / 2A), the SKUs are slotted by popularity (ABC, wh_gen) and the same
orders and plans are scored on the device; each row reports the utilisation,
feasibility and the plans' mean S-shape and optimal lengths.  Python only
sequences the calls; every length comes from the library's kernels.
"""
from __future__ import annotations

import numpy as np


def utilisation(A: int, L: int, P: int, S: int, W: int, rack_depth: float) -> float:
    """A_ind / A_max of the layout (see the module docstring)."""
    return (A * 2.0 * rack_depth * L * S) / (A * P * (L * S + 2.0 * W))


def feasible(P: int, rack_depth: float, k: float, delta: float) -> bool:
    """k * delta - (P - 2 * rack_depth) <= 0."""
    return k * delta - (P - 2.0 * rack_depth) <= 0.0


def layout_sweep(wh, inst, aisle_counts, pitches, n_loc: int, rack_depth: float = 1.0, k: float = 1.0,
                 delta: float = 1.0, slot_seed: int = 1, swap_frac: float = 0.0, device=None):
    """Score `inst`'s orders and plans on every layout (A, P) of the sweep.
    Returns one dict per layout: A, L, P, utilisation, feasible,
    mean_plan_sshape, mean_plan_optimal (device-evaluated)."""
    import torch
    import wh_gen
    rows = []
    S, W = inst.layout.slot_pitch, inst.layout.cross_aisle_width
    for A in aisle_counts:
        L = max(1, n_loc // (2 * A))
        if A * 2 * L < inst.n_sku:
            continue                          # not enough locations for the SKUs
        for P in pitches:
            lay = wh_gen.Layout(A, L, P, S, W)
            slot = wh_gen.gen_slot_abc(slot_seed, lay, inst.n_sku, swap_frac)
            cur = wh_gen.Instance(lay, inst.n_sku, inst.order_off, inst.line_sku, slot, inst.plan_tour_off,
                                  inst.tour_off, inst.order_seq)
            handle = wh.Layout.of(lay)
            prob = wh.to_device(cur, device or "cuda")
            costs = wh.evaluate(handle, prob)
            ps = costs.plan_s[:prob.n_plans].double().mean().item()
            pr = costs.plan_rr[:prob.n_plans].double().mean().item()
            assert handle.status() == 0
            handle.close()
            rows.append({"A": A, "L": L, "P": P, "utilisation": utilisation(A, L, P, S, W, rack_depth),
                         "feasible": feasible(P, rack_depth, k, delta), "mean_plan_sshape": ps,
                         "mean_plan_optimal": pr})
    return rows


def pareto(rows):
    """The feasible layouts not dominated in (utilisation up, optimal length down)."""
    ok = [r for r in rows if r["feasible"]]
    front = []
    for r in ok:
        if not any(q["utilisation"] >= r["utilisation"] and q["mean_plan_optimal"] <= r["mean_plan_optimal"]
                   and (q["utilisation"] > r["utilisation"] or q["mean_plan_optimal"] < r["mean_plan_optimal"])
                   for q in ok):
            front.append(r)
    return sorted(front, key=lambda r: r["utilisation"])
