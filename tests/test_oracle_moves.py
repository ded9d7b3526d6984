"""Pins of the oracle's move deltas: every moved plan is rebuilt here in
Python, independently of the oracle's move code, and re-scored with
``eval_plans``; status codes are checked on hand-picked cases."""
import numpy as np
import pytest

import oracle
import wh_gen


def plan_tours(inst, p):
    t0, t1 = inst.plan_tour_off[p], inst.plan_tour_off[p + 1]
    return [inst.order_seq[inst.tour_off[t]:inst.tour_off[t + 1]].tolist() for t in range(t0, t1)]


def one_plan(inst, tours, slot_map=None):
    to = np.concatenate([[0], np.cumsum([len(t) for t in tours])]).astype(np.int32)
    seq = np.asarray([o for t in tours for o in t], np.int32)
    return wh_gen.Instance(inst.layout, inst.n_sku, inst.order_off, inst.line_sku,
                           inst.slot_map if slot_map is None else slot_map,
                           np.asarray([0, len(tours)], np.int32), to, seq)


def plan_cost(inst, tours, slot_map=None):
    _, _, ps, pr = oracle.eval_plans(one_plan(inst, tours, slot_map))
    return int(ps[0]), int(pr[0])


def find(tours, o):
    for i, t in enumerate(tours):
        if o in t:
            return i
    return -1


def expected(inst, move, maps=None, max_orders=0, max_lines=0):
    typ, a, b, p = move
    tours = plan_tours(inst, p)
    smap = inst.slot_map if maps is None else maps[p]
    sizes = np.diff(inst.order_off)
    before = plan_cost(inst, tours, smap)
    lines = lambda t: int(sizes[t].sum()) if t else 0
    if typ == 0:
        ta, tb = find(tours, a), find(tours, b)
        if ta < 0 or tb < 0:
            return (0, 0), 3
        if ta == tb:
            return (0, 0), 2
        tours[ta] = [b if o == a else o for o in tours[ta]]
        tours[tb] = [a if o == b else o for o in tours[tb]]
        if max_lines and (lines(tours[ta]) > max_lines or lines(tours[tb]) > max_lines):
            return (0, 0), 1
        after = plan_cost(inst, tours, smap)
    elif typ == 1:
        ta = find(tours, a)
        if ta < 0 or not (0 <= b < len(tours)):
            return (0, 0), 3
        if ta == b:
            return (0, 0), 2
        tours[ta] = [o for o in tours[ta] if o != a]
        tours[b] = tours[b] + [a]
        if (max_orders and len(tours[b]) > max_orders) or (max_lines and lines(tours[b]) > max_lines):
            return (0, 0), 1
        after = plan_cost(inst, tours, smap)
    elif typ == 2:
        if maps is None or not (0 <= a < inst.n_sku and 0 <= b < inst.n_sku):
            return (0, 0), 3
        if a == b:
            return (0, 0), 2
        m2 = smap.copy()
        m2[a], m2[b] = m2[b], m2[a]
        after = plan_cost(inst, tours, m2)
    elif typ == 3:
        if maps is None or not (0 <= a < inst.n_sku and 0 <= b < inst.layout.n_loc):
            return (0, 0), 3
        if smap[a] == b:
            return (0, 0), 2
        if b in set(smap.tolist()):
            return (0, 0), 3                  # the target holds another SKU
        m2 = smap.copy()
        m2[a] = b
        after = plan_cost(inst, tours, m2)
    else:
        return (0, 0), 3
    return (after[0] - before[0], after[1] - before[1]), 0


def test_moves_match_rebuilt_plans():
    inst = wh_gen.tiny(seed=5, n_plans=4)
    moves = wh_gen.gen_moves(3, 0, inst, 40)
    moves[..., 3] = np.arange(4)[:, None]
    mv = moves.reshape(-1, 4)
    d, st = oracle.eval_moves(inst, mv, max_orders=8)
    for m in range(mv.shape[0]):
        want_d, want_st = expected(inst, tuple(mv[m]), max_orders=8)
        assert st[m] == want_st, (m, mv[m])
        assert tuple(d[m]) == want_d, (m, mv[m])
    assert (st == 0).sum() > 20 and (st == 3).sum() > 5    # SKU swaps under a shared slotting


def test_sku_swaps_with_per_plan_slottings():
    inst = wh_gen.tiny(seed=6, n_plans=3)
    rng = np.random.default_rng(2)
    maps = np.stack([rng.permutation(inst.layout.n_loc)[: inst.n_sku] for _ in range(3)]).astype(np.int32)
    moves = wh_gen.gen_moves(4, 1, inst, 30)
    moves[..., 3] = np.arange(3)[:, None]
    mv = moves.reshape(-1, 4)
    d, st = oracle.eval_moves(inst, mv, slot_map=maps.ravel(), slot_map_stride=inst.n_sku)
    for m in range(mv.shape[0]):
        want_d, want_st = expected(inst, tuple(mv[m]), maps=maps)
        assert st[m] == want_st and tuple(d[m]) == want_d, (m, mv[m])
    assert ((mv[:, 0] == 2) & (st == 0)).sum() > 5


def half_full(seed, n_plans):
    """tiny's orders on a 20 x 30 layout (1,200 locations for 600 SKUs): every
    plan its own random slotting, half the locations empty."""
    inst = wh_gen.tiny(seed=seed, n_plans=n_plans)
    lay = wh_gen.Layout(20, 30)
    rng = np.random.default_rng(seed)
    maps = np.stack([rng.permutation(lay.n_loc)[:inst.n_sku] for _ in range(n_plans)]).astype(np.int32)
    big = wh_gen.Instance(lay, inst.n_sku, inst.order_off, inst.line_sku, maps[0], inst.plan_tour_off,
                          inst.tour_off, inst.order_seq)
    return big, maps


def test_relocations_into_empty_locations():
    inst, maps = half_full(9, 3)
    moves = wh_gen.gen_relocations(5, 0, inst, 40).reshape(-1, 4)
    # a few targets that are the SKU's own location (no-op)
    moves[::13, 2] = maps[moves[::13, 3], moves[::13, 1]]
    d, st = oracle.eval_moves(inst, moves, slot_map=maps.ravel(), slot_map_stride=inst.n_sku)
    for m in range(moves.shape[0]):
        want_d, want_st = expected(inst, tuple(moves[m]), maps=maps)
        assert st[m] == want_st and tuple(d[m]) == want_d, (m, moves[m])
    assert (st == 0).sum() > 20 and (st == 3).sum() > 20 and (st == 2).sum() >= 5
    # under a shared slotting relocations are invalid
    _, st = oracle.eval_moves(inst, moves[:5])
    assert (st == 3).all()


def test_status_cases():
    inst = wh_gen.tiny(seed=7, n_plans=2)
    tours = plan_tours(inst, 0)
    big = max(range(len(tours)), key=lambda i: len(tours[i]))
    a = tours[big][0]
    same = tours[big][1] if len(tours[big]) > 1 else a
    other = [t for i, t in enumerate(tours) if i != big][0][0]
    cases = [
        ((0, a, same, 0), 2),                 # both orders in one tour
        ((1, a, big, 0), 2),                  # relocate into its own tour
        ((0, a, 10_000, 0), 3),               # order id out of range
        ((1, a, 10_000, 0), 3),               # tour index out of range
        ((2, 1, 2, 0), 3),                    # SKU swap under a shared slotting
        ((9, 1, 2, 0), 3),                    # unknown type
        ((0, a, other, 5), 3),                # plan out of range
        ((1, other, big, 0), 1),              # relocate over an order cap of len(big)
    ]
    mv = np.asarray([c[0] for c in cases], np.int32)
    d, st = oracle.eval_moves(inst, mv, max_orders=len(tours[big]))
    assert st.tolist() == [c[1] for c in cases]
    assert (d[st != 0] == 0).all()


def test_relocate_can_empty_a_tour():
    inst = wh_gen.tiny(seed=8, n_plans=1)
    tours = plan_tours(inst, 0)
    single = [i for i, t in enumerate(tours) if len(t) == 1]
    if not single:
        pytest.skip("no single-order tour in this seed")
    src = single[0]
    dst = (src + 1) % len(tours)
    d, st = oracle.eval_moves(inst, np.asarray([[1, tours[src][0], dst, 0]], np.int32))
    assert st[0] == 0
    want, _ = expected(inst, (1, tours[src][0], dst, 0))
    assert tuple(d[0]) == want
