"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Every check here is independent of the oracle's own code: scipy's Dijkstra on
the explicit corridor graph, the S-shape rule written out as a closed form,
pure-Python enumeration of routes, hand-worked routes walked segment by
segment, and invariants that any correct optimal route length satisfies.
"""
import itertools
import json
import os

import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import dijkstra

import oracle
import wh_gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_tours.json")

LAYOUTS = [
    wh_gen.Layout(10, 30),            # the worked-example geometry
    wh_gen.Layout(3, 5, 2, 1, 2),
    wh_gen.Layout(6, 8, 5, 2, 4),     # wider cross-aisles, slot pitch 2
    wh_gen.Layout(1, 10),             # a single aisle
    wh_gen.Layout(20, 4, 1, 3, 6),    # pitch smaller than the slot pitch
    wh_gen.Layout(40, 100),           # the mid-size warehouse
]


def Ydepth(lay):
    return lay.cross_aisle_width + (lay.slots_per_side - 1) * lay.slot_pitch


def depth_of(lay, k):
    return lay.cross_aisle_width // 2 + k * lay.slot_pitch


def loc_of(lay, a, y, side=0):
    k = (y - lay.cross_aisle_width // 2) // lay.slot_pitch
    return lay.loc(a, k, side)


def decode(lay, loc):
    a = loc // (2 * lay.slots_per_side)
    k = loc % lay.slots_per_side
    return a, depth_of(lay, k)


def corridor_graph(lay):
    """Explicit graph: per aisle a node at the front end, one per slot depth,
    one at the back end; aisle edges between consecutive depths; cross-aisle
    edges between neighbouring aisle ends."""
    Y = Ydepth(lay)
    depths = [0] + [depth_of(lay, k) for k in range(lay.slots_per_side)] + [Y]
    idx = {}
    for a in range(lay.n_aisles):
        for y in depths:
            idx[(a, y)] = len(idx)
    rows, cols, w = [], [], []

    def edge(u, v, c):
        rows.extend([idx[u], idx[v]]); cols.extend([idx[v], idx[u]]); w.extend([c, c])

    for a in range(lay.n_aisles):
        for y0, y1 in zip(depths, depths[1:]):
            edge((a, y0), (a, y1), y1 - y0)
        if a + 1 < lay.n_aisles:
            edge((a, 0), (a + 1, 0), lay.aisle_pitch)
            edge((a, Y), (a + 1, Y), lay.aisle_pitch)
    n = len(idx)
    m = coo_matrix((np.asarray(w, float), (rows, cols)), shape=(n, n)).tocsr()
    return idx, dijkstra(m, directed=False)


# ------------------------------------------------------------------ distances

@pytest.mark.parametrize("lay", LAYOUTS[:5])
def test_distance_equals_dijkstra_all_pairs(lay):
    idx, D = corridor_graph(lay)
    nodes = [p for p in idx if 0 < p[1] < Ydepth(lay)] + [(0, 0)]
    for (a1, y1) in nodes:
        for (a2, y2) in nodes:
            assert oracle.dist(lay, a1, y1, a2, y2) == int(D[idx[(a1, y1)], idx[(a2, y2)]])


# ---------------------------------------------------------------- S-shape rule

def sshape_closed_form(lay, locs):
    """2*x_r + (m even ? m*Y : (m-1)*Y + 2*d_r): m pick aisles, r the
    rightmost, d_r its deepest pick; 0 for no pick."""
    picks = {decode(lay, l) for l in locs}
    if not picks:
        return 0
    aisles = sorted({a for a, _ in picks})
    m, r = len(aisles), aisles[-1]
    d_r = max(y for a, y in picks if a == r)
    Y = Ydepth(lay)
    return 2 * r * lay.aisle_pitch + (m * Y if m % 2 == 0 else (m - 1) * Y + 2 * d_r)


@pytest.mark.parametrize("lay", LAYOUTS)
def test_sshape_walk_equals_closed_form(lay):
    rng = np.random.default_rng(11)
    for _ in range(400):
        n = int(rng.integers(0, 40))
        locs = rng.integers(0, lay.n_loc, size=n)
        assert oracle.sshape(lay, locs) == sshape_closed_form(lay, locs)


# ------------------------------------------------------------- worked vectors

def walk_route(lay, route):
    """Length of a corridor route; asserts every leg stays in a corridor."""
    Y = Ydepth(lay)
    total = 0
    for (a1, y1), (a2, y2) in zip(route, route[1:]):
        if a1 == a2:
            total += abs(y1 - y2)
        else:
            assert y1 == y2 and y1 in (0, Y), "horizontal legs run along a cross-aisle"
            total += lay.aisle_pitch * abs(a1 - a2)
    return total


def route_visits(route, pick):
    a, y = pick
    for (a1, y1), (a2, y2) in zip(route, route[1:]):
        if a1 == a2 == a and min(y1, y2) <= y <= max(y1, y2):
            return True
    return False


def test_worked_tours():
    g = json.load(open(GOLDEN))
    lay = wh_gen.Layout(**g["layout"])
    for t in g["tours"]:
        picks = [tuple(p) for p in t["picks"]]
        locs = [loc_of(lay, a, y) for a, y in picks]
        route = [tuple(p) for p in t["route"]]
        assert route[0] == (0, 0) and route[-1] == (0, 0)
        assert all(route_visits(route, p) for p in picks)
        assert walk_route(lay, route) == t["optimal"]
        assert sshape_closed_form(lay, locs) == t["sshape"]
        assert oracle.sshape(lay, locs) == t["sshape"]
        assert oracle.rr(lay, locs) == t["optimal"]
        assert oracle.heldkarp(lay, locs) == t["optimal"]
        assert oracle.permutation(lay, locs) == t["optimal"]


# ---------------------------------------------------------- exact small tours

@pytest.mark.parametrize("lay", LAYOUTS[:3])
def test_exact_tours_equal_python_enumeration(lay):
    """Pure-Python enumeration of picking sequences over Dijkstra distances."""
    idx, D = corridor_graph(lay)
    rng = np.random.default_rng(5)
    for _ in range(60):
        n = int(rng.integers(1, 7))
        locs = rng.integers(0, lay.n_loc, size=n)
        pts = sorted({decode(lay, l) for l in locs})
        best = min(
            D[idx[(0, 0)], idx[seq[0]]]
            + sum(D[idx[u], idx[v]] for u, v in zip(seq, seq[1:]))
            + D[idx[seq[-1]], idx[(0, 0)]]
            for seq in itertools.permutations(pts))
        assert oracle.heldkarp(lay, locs) == int(best)
        assert oracle.permutation(lay, locs) == int(best)


def random_tour(rng, lay, n):
    """Uniform picks, or picks crowded into a few aisles, or near the back."""
    kind = rng.integers(0, 3)
    if kind == 0:
        return rng.integers(0, lay.n_loc, size=n)
    if kind == 1:
        na = int(rng.integers(1, 4))
        a = rng.integers(0, min(na, lay.n_aisles), size=n)
    else:
        a = rng.integers(0, lay.n_aisles, size=n)
    lo = lay.slots_per_side // 2 if kind == 2 else 0
    k = rng.integers(lo, lay.slots_per_side, size=n)
    return (a * 2 + rng.integers(0, 2, size=n)) * lay.slots_per_side + k


@pytest.mark.parametrize("lay", LAYOUTS)
def test_rr_equals_heldkarp_small_tours(lay):
    rng = np.random.default_rng(1983)
    for _ in range(1500):
        locs = random_tour(rng, lay, int(rng.integers(0, 11)))
        assert oracle.rr(lay, locs) == oracle.heldkarp(lay, locs), (lay, locs.tolist())


def test_rr_equals_heldkarp_spot_16():
    rng = np.random.default_rng(7)
    for lay in LAYOUTS[:3]:
        for _ in range(6):
            locs = random_tour(rng, lay, int(rng.integers(11, 17)))
            assert oracle.rr(lay, locs) == oracle.heldkarp(lay, locs)


def test_permutation_equals_heldkarp():
    rng = np.random.default_rng(8)
    for lay in LAYOUTS[:4]:
        for _ in range(100):
            locs = random_tour(rng, lay, int(rng.integers(0, 8)))
            assert oracle.permutation(lay, locs) == oracle.heldkarp(lay, locs)


# ------------------------------------------------------------------ invariants

@pytest.mark.parametrize("lay", LAYOUTS)
def test_route_invariants(lay):
    rng = np.random.default_rng(99)
    Y = Ydepth(lay)
    for _ in range(300):
        locs = random_tour(rng, lay, int(rng.integers(1, 60)))
        opt, s = oracle.rr(lay, locs), oracle.sshape(lay, locs)
        picks = [decode(lay, l) for l in locs]
        r = max(a for a, _ in picks)
        dmax = max(y for _, y in picks)
        assert opt <= s
        # depth changes only inside aisles and the walk starts and ends at
        # depth 0; x changes only along cross-aisles and ends at x = 0
        assert opt >= 2 * dmax + 2 * r * lay.aisle_pitch
        assert opt % 2 == 0 and s % 2 == 0
        perm = rng.permutation(locs)
        assert oracle.rr(lay, perm) == opt and oracle.sshape(lay, perm) == s
        dup = np.concatenate([locs, locs[: len(locs) // 2]])
        assert oracle.rr(lay, dup) == opt and oracle.sshape(lay, dup) == s
        # the other side of the same aisle position is the same point
        flipped = [(l // lay.slots_per_side ^ 1) * lay.slots_per_side + l % lay.slots_per_side for l in locs]
        assert oracle.rr(lay, flipped) == opt
        extra = np.concatenate([locs, rng.integers(0, lay.n_loc, size=1)])
        assert oracle.rr(lay, extra) >= opt


def test_special_cases():
    for lay in LAYOUTS:
        assert oracle.rr(lay, []) == 0 and oracle.sshape(lay, []) == 0
        Y = Ydepth(lay)
        # aisle 0 only: in and out of the depot aisle
        ks = [0, lay.slots_per_side - 1, lay.slots_per_side // 2]
        locs = [lay.loc(0, k) for k in ks]
        dmax = max(depth_of(lay, k) for k in ks)
        assert oracle.rr(lay, locs) == oracle.sshape(lay, locs) == 2 * dmax
        # one pick in aisle a: the cheaper of in-and-out and a loop through the back
        for a in range(min(lay.n_aisles, 4)):
            for k in (0, lay.slots_per_side - 1):
                y = depth_of(lay, k)
                want = 2 * a * lay.aisle_pitch + (2 * y if a == 0 else min(2 * y, 2 * Y))
                assert oracle.rr(lay, [lay.loc(a, k)]) == want


def test_rejects_bad_layout_and_locations():
    with pytest.raises(ValueError):
        oracle.rr(wh_gen.Layout(10, 30, 3, 1, 3), [0])      # odd cross-aisle width
    with pytest.raises(ValueError):
        oracle.rr(wh_gen.Layout(10, 30), [600])            # location out of range
    with pytest.raises(ValueError):
        oracle.sshape(wh_gen.Layout(10, 30), [-1])


# ------------------------------------------------------------------ plan sums

def test_eval_plans_equals_per_tour_sums():
    inst = wh_gen.tiny(seed=3, n_plans=6)
    ts, tr, ps, pr = oracle.eval_plans(inst)
    lay = inst.layout
    for p in range(inst.n_plans):
        sum_s = sum_r = 0
        for t in range(inst.plan_tour_off[p], inst.plan_tour_off[p + 1]):
            locs = []
            for o in inst.order_seq[inst.tour_off[t]:inst.tour_off[t + 1]]:
                locs.extend(inst.slot_map[inst.line_sku[inst.order_off[o]:inst.order_off[o + 1]]].tolist())
            assert ts[t] == sshape_closed_form(lay, locs)
            assert tr[t] == oracle.rr(lay, locs)
            sum_s += int(ts[t]); sum_r += int(tr[t])
        assert ps[p] == sum_s and pr[p] == sum_r


def test_eval_plans_per_plan_slot_maps():
    inst = wh_gen.tiny(seed=4, n_plans=3)
    maps = np.stack([np.random.default_rng(p).permutation(inst.layout.n_loc)[: inst.n_sku]
                     for p in range(3)]).astype(np.int32)
    _, tr, _, pr = oracle.eval_plans(inst, slot_map=maps.ravel(), slot_map_stride=inst.n_sku)
    for p in range(3):
        one = inst.subset_plans([p])
        one.slot_map = maps[p]
        assert oracle.eval_plans(one)[3][0] == pr[p]
