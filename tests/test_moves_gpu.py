"""wh_eval_moves against the oracle's apply-and-rescore deltas (exact int64)
and status codes, on shared and per-plan slottings, short and long tours."""
import numpy as np
import pytest

import oracle
import wh_gen

pytestmark = pytest.mark.gpu


def gpu_moves(wh, inst, moves, max_orders=0, max_lines=0, maps=None, occupancy=True):
    import torch
    lay = wh.Layout.of(inst.layout)
    stride = inst.n_sku if maps is not None else 0
    prob = wh.to_device(inst, slot_map=None if maps is None else maps.ravel(), slot_map_stride=stride)
    if maps is not None and occupancy:
        lay.occupancy(prob)
    costs = wh.evaluate(lay, prob)
    mv = torch.as_tensor(np.ascontiguousarray(moves.reshape(-1, 4)), dtype=torch.int32).cuda()
    delta, status = lay.eval_moves(prob, costs, mv, max_orders, max_lines)
    torch.cuda.synchronize()
    st = lay.status()
    lay.close()
    return delta.cpu().numpy(), status.cpu().numpy(), st


def moves_for(inst, seed, per_plan):
    mv = wh_gen.gen_moves(seed, 0, inst, per_plan)
    mv[..., 3] = np.arange(inst.n_plans)[:, None]
    return mv.reshape(-1, 4)


def check(wh, inst, mv, max_orders=0, max_lines=0, maps=None):
    d, s, st = gpu_moves(wh, inst, mv, max_orders, max_lines, maps)
    kw = {} if maps is None else {"slot_map": maps.ravel(), "slot_map_stride": inst.n_sku}
    wd, ws = oracle.eval_moves(inst, mv, max_orders, max_lines, **kw)
    assert np.array_equal(s, ws), f"status differs at {np.nonzero(s != ws)[0][:5]}"
    bad = np.nonzero((d != wd).any(axis=1))[0]
    assert bad.size == 0, f"delta differs at {bad[:5]}: got {d[bad[:3]]} want {wd[bad[:3]]} moves {mv[bad[:3]]}"
    return s, st


def test_tiny_shared_slotting(gpu_lib):
    inst = wh_gen.tiny(seed=3, n_plans=8)
    s, st = check(gpu_lib, inst, moves_for(inst, 1, 64), max_orders=8)
    assert st == 0 and (s == 0).sum() > 100 and (s == 3).sum() > 50


def test_tiny_per_plan_slottings(gpu_lib):
    inst = wh_gen.tiny(seed=4, n_plans=6)
    rng = np.random.default_rng(0)
    maps = np.stack([rng.permutation(inst.layout.n_loc)[: inst.n_sku] for _ in range(6)]).astype(np.int32)
    s, st = check(gpu_lib, inst, moves_for(inst, 2, 64), max_orders=8, maps=maps)
    assert st == 0 and (s == 0).sum() > 250


def test_midsize_with_caps(gpu_lib):
    inst = wh_gen.midsize(seed=5, n_plans=8)
    maps = np.tile(inst.slot_map, (8, 1)).astype(np.int32)
    s, st = check(gpu_lib, inst, moves_for(inst, 3, 48), max_orders=20, max_lines=60, maps=maps)
    assert st == 0 and (s == 1).sum() > 0 and (s == 0).sum() > 200


def test_paperscale_long_tours_and_popular_skus(gpu_lib):
    """32-bit keys (500 aisles), tours beyond 64 lines, and SKU swaps of the
    most popular SKUs, which touch most tours of a plan."""
    inst = wh_gen.paperscale(seed=6, n_plans=3)
    maps = np.tile(inst.slot_map, (3, 1)).astype(np.int32)
    mv = moves_for(inst, 4, 24)
    hot = np.asarray([[2, 0, 1, 0], [2, 1, 30000, 1], [2, 0, 49999, 2], [2, 2, 3, 0]], np.int32)
    mv = np.concatenate([mv, hot])
    s, st = check(gpu_lib, inst, mv, max_orders=24, maps=maps)
    assert st == 0 and (s == 0).sum() > 40


def long_instance(lay, seed, n_orders=400, lines=(8, 12), per_tour=8, n_plans=3):
    """Orders of many lines on a random slotting, tours of `per_tour` orders
    (about 80 lines each, all above the one-tour-per-thread limit of 64)."""
    rng = np.random.default_rng(seed)
    n_sku = lay.n_loc
    slot = rng.permutation(lay.n_loc).astype(np.int32)
    sizes = rng.integers(lines[0], lines[1] + 1, n_orders)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    line_sku = np.concatenate([rng.choice(n_sku, size=int(k), replace=False) for k in sizes]).astype(np.int32)
    pto, to, seq = [0], [0], []
    for _ in range(n_plans):
        perm = rng.permutation(n_orders)
        for t0 in range(0, n_orders, per_tour):
            seq.extend(perm[t0:t0 + per_tour].tolist())
            to.append(len(seq))
        pto.append(len(to) - 1)
    return wh_gen.Instance(lay, n_sku, off, line_sku, slot, np.asarray(pto, np.int32), np.asarray(to, np.int32),
                           np.asarray(seq, np.int32))


@pytest.mark.parametrize("lay", [wh_gen.Layout(40, 100), wh_gen.Layout(300, 10)])
def test_long_tasks_batched_and_wide(gpu_lib, lay):
    """Tasks of about 80 lines: on 40 aisles every task's records fit the
    batched per-lane DP; on 300 aisles most tasks visit more aisles than it
    keeps and take the single-lane path.  Several batches of 32 per warp."""
    inst = long_instance(lay, lay.n_aisles)
    assert (inst.tour_lines() > 64).all()
    maps = np.tile(inst.slot_map, (inst.n_plans, 1)).astype(np.int32)
    s, st = check(gpu_lib, inst, moves_for(inst, 7, 64), maps=maps)
    assert st == 0 and (s == 0).sum() > 150


def test_status_cases(gpu_lib):
    inst = wh_gen.tiny(seed=7, n_plans=2)
    t0, t1 = inst.plan_tour_off[0], inst.plan_tour_off[1]
    tours = [inst.order_seq[inst.tour_off[t]:inst.tour_off[t + 1]].tolist() for t in range(t0, t1)]
    big = max(range(len(tours)), key=lambda i: len(tours[i]))
    a = tours[big][0]
    same = tours[big][1] if len(tours[big]) > 1 else a
    other = [t for i, t in enumerate(tours) if i != big][0][0]
    mv = np.asarray([[0, a, same, 0], [1, a, big, 0], [0, a, 10_000, 0], [1, a, 10_000, 0], [2, 1, 2, 0],
                     [9, 1, 2, 0], [0, a, other, 5], [1, other, big, 0], [0, a, other, 0], [1, a, -1, 1]],
                    np.int32)
    s, st = check(gpu_lib, inst, mv, max_orders=len(tours[big]))
    assert s.tolist()[:8] == [2, 2, 3, 3, 3, 3, 3, 1]


def test_repeat_and_empty(gpu_lib):
    import torch
    wh = gpu_lib
    inst = wh_gen.tiny(seed=9, n_plans=4)
    mv = moves_for(inst, 5, 32)
    a = gpu_moves(wh, inst, mv, 8)
    b = gpu_moves(wh, inst, mv, 8)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    lay = wh.Layout.of(inst.layout)
    prob = wh.to_device(inst)
    costs = wh.evaluate(lay, prob)
    d, s = lay.eval_moves(prob, costs, torch.zeros((0, 4), dtype=torch.int32, device="cuda"))
    assert d.shape[0] == 0 and s.shape[0] == 0
    lay.close()


def test_paperscale_full_size_sampled(gpu_lib):
    """The benchmark's launch: 16,384 paper-scale plans with their own
    slottings x 64 moves (1,048,576 moves, long tasks included).  Sampled
    moves are re-scored one by one by the oracle on their plan alone; every
    status is in range and every non-zero status has zero deltas."""
    import torch
    wh = gpu_lib
    n_plans, M = 16384, 64
    inst = wh_gen.paperscale(seed=4, n_plans=n_plans)
    lay = wh.Layout.of(inst.layout)
    base = wh.to_device(inst)
    prob = wh.DeviceProblem(base.order_off, base.line_sku, base.slot_map.repeat(n_plans), base.plan_tour_off,
                            base.tour_off, base.order_seq, inst.n_sku, inst.n_sku)
    costs = wh.evaluate(lay, prob)
    mv = wh_gen.gen_moves(17, 0, inst, M)
    mv[..., 3] = np.arange(n_plans)[:, None]
    mv = mv.reshape(-1, 4)
    delta, status = lay.eval_moves(prob, costs, torch.as_tensor(mv).cuda(), 24)
    d, s = delta.cpu().numpy(), status.cpu().numpy()
    assert lay.status() == 0
    assert set(np.unique(s).tolist()) <= {0, 1, 2, 3} and (s == 0).mean() > 0.5
    assert (d[s != 0] == 0).all()
    rng = np.random.default_rng(0)
    picks = np.concatenate([[0, len(mv) - 1], rng.integers(0, len(mv), 250)])
    for k in picks:
        p = int(mv[k, 3])
        one = inst.subset_plans([p])
        m1 = mv[k].copy()
        m1[3] = 0
        wd, ws = oracle.eval_moves(one, m1[None], 24, 0, slot_map=inst.slot_map, slot_map_stride=inst.n_sku)
        assert s[k] == ws[0] and (d[k] == wd[0]).all(), (k, mv[k], d[k], wd[0], s[k], ws[0])
    lay.close()


def half_full(seed, n_plans):
    """tiny's orders on a 20 x 30 layout: per-plan random slottings of the 600
    SKUs over 1,200 locations (half of them empty)."""
    inst = wh_gen.tiny(seed=seed, n_plans=n_plans)
    lay = wh_gen.Layout(20, 30)
    rng = np.random.default_rng(seed)
    maps = np.stack([rng.permutation(lay.n_loc)[:inst.n_sku] for _ in range(n_plans)]).astype(np.int32)
    return wh_gen.Instance(lay, inst.n_sku, inst.order_off, inst.line_sku, maps[0], inst.plan_tour_off,
                           inst.tour_off, inst.order_seq), maps


def relocation_moves(inst, maps, seed, per_plan):
    mv = wh_gen.gen_relocations(seed, 0, inst, per_plan).reshape(-1, 4)
    mv[::11, 2] = maps[mv[::11, 3], mv[::11, 1]]          # some onto the SKU's own location (no-op)
    return mv


def test_relocations_into_empty_locations(gpu_lib):
    inst, maps = half_full(21, 6)
    mv = np.concatenate([moves_for(inst, 5, 32), relocation_moves(inst, maps, 6, 48)])
    s, st = check(gpu_lib, inst, mv, max_orders=8, maps=maps)
    r = mv[:, 0] == 3
    assert st == 0 and (s[r] == 0).sum() > 100 and (s[r] == 3).sum() > 80 and (s[r] == 2).sum() > 10


def test_relocations_paperscale(gpu_lib):
    """50,000 SKUs over 200,000 locations: relocations of the most popular
    SKUs (in most tours of a plan, long tours included) and of random ones."""
    inst = wh_gen.paperscale(seed=6, n_plans=3)
    maps = np.tile(inst.slot_map, (3, 1)).astype(np.int32)
    mv = relocation_moves(inst, maps, 8, 40)
    hot = np.asarray([[3, 0, 199_999, 0], [3, 1, 150_000, 1], [3, 2, 123_457, 2], [3, 0, int(maps[0, 1]), 0]],
                     np.int32)
    s, st = check(gpu_lib, inst, np.concatenate([mv, hot]), max_orders=24, maps=maps)
    assert st == 0 and (s == 0).sum() > 60


def test_relocation_needs_occupancy_bits(gpu_lib):
    inst, maps = half_full(22, 2)
    mv = relocation_moves(inst, maps, 9, 16)
    d, s, st = gpu_moves(gpu_lib, inst, mv, maps=maps, occupancy=False)
    assert (s == 3).all() and (d == 0).all()
    d, s, st = gpu_moves(gpu_lib, inst, mv[:4])            # shared slotting
    assert (s == 3).all()


def test_move_stats_count_the_changed_tours(gpu_lib):
    """wh_get_move_stats after a call: the changed tours the moves rewrite
    (two per accepted order swap or relocation, one per order holding a
    swapped SKU) and their line counts, recounted here from the plans."""
    import torch
    wh = gpu_lib
    inst = wh_gen.paperscale(seed=8, n_plans=6)
    maps = np.tile(inst.slot_map, (inst.n_plans, 1)).astype(np.int32)
    mv = moves_for(inst, 9, 64)
    lay = wh.Layout.of(inst.layout)
    prob = wh.to_device(inst, slot_map=maps.ravel(), slot_map_stride=inst.n_sku)
    costs = wh.evaluate(lay, prob)
    _, status = lay.eval_moves(prob, costs, torch.as_tensor(mv).cuda(), 24, 0)
    tours, lines = lay.move_stats()
    status = status.cpu().numpy()
    assert lay.status() == 0
    lay.close()
    ol = np.diff(inst.order_off)                        # lines per order
    line_order = np.repeat(np.arange(inst.n_orders), ol)
    orders_of = {}
    for l, sku in enumerate(inst.line_sku):
        orders_of.setdefault(int(sku), []).append(int(line_order[l]))
    want_t = want_l = 0
    for m, (typ, a, b, p) in enumerate(mv):
        if status[m] != 0:
            continue
        t0, t1 = inst.plan_tour_off[p], inst.plan_tour_off[p + 1]
        tour_of = {}
        for t in range(t0, t1):
            for o in inst.order_seq[inst.tour_off[t]:inst.tour_off[t + 1]]:
                tour_of[int(o)] = t
        tl = lambda t: int(ol[inst.order_seq[inst.tour_off[t]:inst.tour_off[t + 1]]].sum())
        if typ == 0:
            want_t += 2
            want_l += tl(tour_of[a]) - ol[a] + ol[b] + tl(tour_of[b]) - ol[b] + ol[a]
        elif typ == 1:
            want_t += 2
            want_l += tl(tour_of[a]) - ol[a] + tl(t0 + b) + ol[a]
        else:
            for sku in (a, b):
                for o in orders_of.get(int(sku), []):
                    want_t += 1
                    want_l += tl(tour_of[o])
    assert (tours, lines) == (want_t, int(want_l))


def test_moved_tours_over_the_record_slots(gpu_lib):
    """Moves on tours that visit more pick aisles than a thread keeps records
    for (64 aisles, one- and two-line orders spread over them): the changed
    tours go to the long-task pass and the deltas equal the oracle's."""
    import test_parity_gpu as tp
    inst = tp._wide_instance(n_plans=4)
    rng = np.random.default_rng(1)
    maps = np.stack([inst.slot_map if p == 0 else rng.permutation(inst.layout.n_loc)[: inst.n_sku]
                     for p in range(4)]).astype(np.int32)
    s, st = check(gpu_lib, inst, moves_for(inst, 3, 64), maps=maps)
    assert st == 0 and (s == 0).sum() > 150


def test_bad_location_past_the_short_limit(gpu_lib):
    """Three long tours of plan 0 reach a SKU whose slot-map entry is out of
    range only after their first 64 lines (the short-task pass stops before
    it; the long-task pass walks those tours in full).  Every move whose
    changed tours include one of them scores status 3; every other move
    scores as the oracle scores it on the intact slot maps."""
    lay = wh_gen.Layout(40, 100)
    inst = long_instance(lay, 11)
    maps = np.tile(inst.slot_map, (inst.n_plans, 1)).astype(np.int32)
    ol = np.diff(inst.order_off)
    t0, t1 = inst.plan_tour_off[0], inst.plan_tour_off[1]
    tour_of = {}
    for t in range(t0, t1):
        for o in inst.order_seq[inst.tour_off[t]:inst.tour_off[t + 1]]:
            tour_of[int(o)] = t
    bad_tours, bad_skus = set(), set()
    for t in range(t0, t1):
        orders = inst.order_seq[inst.tour_off[t]:inst.tour_off[t + 1]]
        if ol[orders[:-1]].sum() < 65:
            continue
        sku = int(inst.line_sku[inst.order_off[orders[-1]]])
        if (inst.line_sku == sku).sum() != 1:
            continue
        bad_tours.add(t)
        bad_skus.add(sku)
        if len(bad_tours) == 3:
            break
    assert len(bad_tours) == 3
    mv = moves_for(inst, 12, 64)
    keep = [m for m in range(mv.shape[0]) if not (mv[m, 0] >= 2 and (mv[m, 1] in bad_skus or mv[m, 2] in bad_skus))]
    mv = mv[keep]
    want_d, want_s = oracle.eval_moves(inst, mv, 0, 0, slot_map=maps.ravel(), slot_map_stride=inst.n_sku)
    broken = maps.copy()
    for sku in bad_skus:
        broken[0, sku] = -1
    d, s, _ = gpu_moves(gpu_lib, inst, mv, maps=broken)
    line_order = np.repeat(np.arange(inst.n_orders), ol)
    touched = 0
    for m, (typ, a, b, p) in enumerate(mv):
        hit = False
        if p == 0 and want_s[m] == 0:
            if typ == 0:
                hit = tour_of[int(a)] in bad_tours or tour_of[int(b)] in bad_tours
            elif typ == 1:
                hit = tour_of[int(a)] in bad_tours or t0 + int(b) in bad_tours
            else:
                skus = (a, b) if typ == 2 else (a,)
                orders = {int(line_order[l]) for l in np.nonzero(np.isin(inst.line_sku, skus))[0]}
                hit = any(tour_of[o] in bad_tours for o in orders)
        if hit:
            touched += 1
            assert s[m] == 3 and (d[m] == 0).all(), (m, mv[m], s[m], d[m])
        else:
            assert s[m] == want_s[m] and (d[m] == want_d[m]).all(), (m, mv[m], s[m], want_s[m], d[m], want_d[m])
    assert touched > 0 and (s == 0).sum() > 100
