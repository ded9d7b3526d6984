"""Explicit optimal routes on the GPU against the oracle.  Several optimal
pick sequences can exist, so the check is on what is unique: the route lists
every distinct pick point of the tour exactly once, and walking it with
shortest paths (the oracle's grid distance) from the depot and back covers
exactly the optimal tour length (the oracle's Ratliff-Rosenthal DP, itself
pinned against Held-Karp and brute force), which the kernel also reports."""
import numpy as np
import pytest

import oracle
import wh_gen

pytestmark = pytest.mark.gpu


def tour_locs(inst, t, smap):
    locs = []
    for o in inst.order_seq[inst.tour_off[t]:inst.tour_off[t + 1]]:
        locs.extend(smap[inst.line_sku[inst.order_off[o]:inst.order_off[o + 1]]].tolist())
    return locs


def points_of(lay, locs):
    """Distinct pick points (aisle, slot) of a list of location ids
    (loc = (aisle * 2 + side) * L + slot)."""
    L = lay.slots_per_side
    return sorted({(loc // (2 * L), loc % L) for loc in locs})


def walk_length(lay, route):
    y = [lay.cross_aisle_width // 2 + k * lay.slot_pitch for _, k in route]
    a = [ai for ai, _ in route]
    pts = list(zip([0] + a + [0], [0] + y + [0]))
    return sum(oracle.dist(lay, pts[i][0], pts[i][1], pts[i + 1][0], pts[i + 1][1]) for i in range(len(pts) - 1))


def run(wh, inst, tours, maps=None, max_points=256):
    import torch
    lay = wh.Layout.of(inst.layout)
    prob = wh.to_device(inst, slot_map=None if maps is None else maps.ravel(),
                        slot_map_stride=0 if maps is None else inst.n_sku)
    pts, npt, length = lay.routes(prob, torch.as_tensor(np.asarray(tours, np.int32)).cuda(), max_points)
    torch.cuda.synchronize()
    st = lay.status()
    lay.close()
    return pts.cpu().numpy(), npt.cpu().numpy(), length.cpu().numpy(), st


def plan_of(inst, t):
    return int(np.searchsorted(inst.plan_tour_off, t, side="right") - 1)


def check(wh, inst, tours, maps=None):
    pts, npt, length, st = run(wh, inst, tours, maps)
    assert st == 0
    lay = inst.layout
    for i, t in enumerate(tours):
        smap = inst.slot_map if maps is None else maps[plan_of(inst, t)]
        locs = tour_locs(inst, t, smap)
        want = points_of(lay, locs)
        route = [(int(k) >> 16, int(k) & 0xFFFF) for k in pts[i, :npt[i]]]
        assert npt[i] == len(want), (t, npt[i], len(want))
        assert sorted(route) == want, t                 # each point exactly once
        opt = oracle.rr(lay, locs) if locs else 0
        assert length[i] == opt, (t, length[i], opt)
        assert walk_length(lay, route) == opt, (t, route)
    return pts, npt, length


def test_tiny_all_tours(gpu_lib):
    inst = wh_gen.tiny(seed=3, n_plans=8)
    check(gpu_lib, inst, list(range(inst.n_tours)))


def test_midsize_sampled(gpu_lib):
    """40 aisles x 100 slots, ABC slotting: 600 tours of the plans."""
    inst = wh_gen.midsize(seed=5, n_plans=64)
    rng = np.random.default_rng(5)
    check(gpu_lib, inst, rng.choice(inst.n_tours, 600, replace=False).tolist())


def test_paperscale_sampled(gpu_lib):
    inst = wh_gen.paperscale(seed=4, n_plans=32)
    rng = np.random.default_rng(4)
    check(gpu_lib, inst, rng.choice(inst.n_tours, 400, replace=False).tolist())


def test_per_plan_slottings(gpu_lib):
    inst = wh_gen.tiny(seed=9, n_plans=6)
    rng = np.random.default_rng(9)
    maps = np.stack([rng.permutation(inst.layout.n_loc)[:inst.n_sku] for _ in range(inst.n_plans)])
    check(gpu_lib, inst, list(range(inst.n_tours))[::-1], maps.astype(np.int32))


def single_order_instance(lay, tours_locs):
    """One order per tour, one plan; SKU s sits at location s."""
    sizes = [len(x) for x in tours_locs]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    line_sku = np.concatenate([np.asarray(x, np.int32) for x in tours_locs] + [np.zeros(0, np.int32)])
    n = len(tours_locs)
    return wh_gen.Instance(lay, lay.n_loc, off, line_sku, np.arange(lay.n_loc, dtype=np.int32),
                           np.array([0, n], np.int32), np.arange(n + 1, dtype=np.int32),
                           np.arange(n, dtype=np.int32))


@pytest.mark.parametrize("geom", [(12, 30, 3, 1, 2), (25, 16, 5, 2, 4), (7, 60, 4, 3, 6), (60, 9, 2, 1, 2)])
def test_random_layouts(gpu_lib, geom):
    """Random tours on layouts of several pitches and widths: 1 to 120 lines,
    picks crowded at the front and back ends, the depot aisle, duplicates."""
    lay = wh_gen.Layout(*geom)
    rng = np.random.default_rng(sum(geom))
    L = lay.slots_per_side
    tours = []
    for i in range(300):
        n = int(rng.integers(1, 121)) if i % 3 else int(rng.integers(1, 8))
        aisles = rng.integers(0, lay.n_aisles, n) if i % 4 else rng.integers(0, min(3, lay.n_aisles), n)
        mode = i % 5
        if mode == 0:
            slot = rng.integers(0, max(1, L // 4), n)           # near the front
        elif mode == 1:
            slot = rng.integers(L - max(1, L // 4), L, n)       # near the back
        elif mode == 2:
            slot = np.where(rng.random(n) < 0.5, 0, L - 1)      # both ends
        else:
            slot = rng.integers(0, L, n)
        side = rng.integers(0, 2, n)
        tours.append(((aisles * 2 + side) * L + slot).astype(np.int32).tolist())
    inst = single_order_instance(lay, tours)
    check(gpu_lib, inst, list(range(len(tours))))


def test_wide_tours_up_to_256_points(gpu_lib):
    """Tours spread over up to every aisle (one pick aisle per point) and up
    to the 256-point limit; beyond it the tour is flagged."""
    lay = wh_gen.Layout(255, 40, 3, 1, 2)
    rng = np.random.default_rng(21)
    L = lay.slots_per_side
    tours = []
    for n in (64, 200, 255, 256):
        a = rng.choice(lay.n_aisles, min(n, lay.n_aisles), replace=False)
        a = np.concatenate([a, rng.integers(0, lay.n_aisles, n - len(a))])
        slot = rng.integers(0, L, n)
        keys = set()
        locs = []
        for ai, k in zip(a, slot):                  # distinct points
            while (int(ai), int(k)) in keys:
                k = (k + 1) % L
            keys.add((int(ai), int(k)))
            locs.append(int((ai * 2 + rng.integers(0, 2)) * L + k))
        tours.append(locs)
    inst = single_order_instance(lay, tours)
    pts, npt, length = check(gpu_lib, inst, list(range(len(tours))))
    assert npt.tolist() == [64, 200, 255, 256]
    # 257 distinct points: flagged, nothing written
    big = tours[3] + [next(int((ai * 2) * L + k) for ai in range(lay.n_aisles) for k in range(L)
                           if (ai, k) not in {(x // (2 * L), x % L) for x in tours[3]})]
    inst2 = single_order_instance(lay, [big, tours[0]])
    pts, npt, length, st = run(gpu_lib, inst2, [0, 1])
    assert st == gpu_lib.WH_STATUS_TOUR_TOO_LONG
    assert npt[0] == -1 and length[0] == -1 and npt[1] == 64


def test_edge_cases(gpu_lib):
    lay = wh_gen.Layout(6, 10, 3, 1, 2)
    L = lay.slots_per_side
    tours = [
        [],                                   # an empty tour
        [0],                                  # one pick in the depot's aisle, at the front
        [L - 1],                              # ... at the back
        [(5 * 2 + 1) * L + L - 1],            # the far corner
        [3, L + 3, 3],                        # both sides at one depth, and a duplicate line
        [(a * 2) * L + (a % 2) * (L - 1) for a in range(6)],   # alternating front and back
        [(a * 2 + 1) * L + k for a in (0, 5) for k in range(L)],  # two full aisles
    ]
    inst = single_order_instance(lay, tours)
    pts, npt, length = check(gpu_lib, inst, list(range(len(tours))))
    assert npt[0] == 0 and length[0] == 0
    assert npt[4] == 1


def test_bad_tour_index_and_small_capacity(gpu_lib):
    inst = wh_gen.tiny(seed=3, n_plans=2)
    pts, npt, length, st = run(gpu_lib, inst, [0, inst.n_tours, -1, 1])
    assert st == gpu_lib.WH_STATUS_BAD_OFFSET
    assert npt[1] == -1 and npt[2] == -1 and npt[0] >= 0 and npt[3] >= 0
    # capacity below a tour's point count: that tour is flagged
    sizes = [len(points_of(inst.layout, tour_locs(inst, t, inst.slot_map))) for t in range(4)]
    cap = max(1, min(sizes))
    pts, npt, length, st = run(gpu_lib, inst, [0, 1, 2, 3], max_points=cap)
    for i in range(4):
        if sizes[i] > cap:
            assert npt[i] == -1
        else:
            assert npt[i] == sizes[i]
    assert (st == gpu_lib.WH_STATUS_TOUR_TOO_LONG) == any(s > cap for s in sizes)
