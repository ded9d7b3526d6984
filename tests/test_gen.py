"""Checks of the seeded workload generator (inputs only, no cost arithmetic)."""
import numpy as np

import wh_gen


def test_deterministic_and_seed_sensitive():
    a, b, c = wh_gen.tiny(seed=1), wh_gen.tiny(seed=1), wh_gen.tiny(seed=2)
    for f in ("order_off", "line_sku", "slot_map", "plan_tour_off", "tour_off", "order_seq"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    assert not np.array_equal(a.line_sku[:50], c.line_sku[:50])
    assert wh_gen.stream_word(5, 1, 0) != wh_gen.stream_word(5, 1, 1)
    assert wh_gen.stream_word(5, 1, 0, 0) != wh_gen.stream_word(5, 1, 0, 1)


def check_partition(inst, max_orders, max_lines=None):
    sizes = np.diff(inst.order_off)
    for p in range(inst.n_plans):
        t0, t1 = inst.plan_tour_off[p], inst.plan_tour_off[p + 1]
        s0, s1 = inst.tour_off[t0], inst.tour_off[t1]
        assert sorted(inst.order_seq[s0:s1].tolist()) == list(range(inst.n_orders))
        for t in range(t0, t1):
            orders = inst.order_seq[inst.tour_off[t]:inst.tour_off[t + 1]]
            assert 1 <= len(orders) <= max_orders
            if max_lines:
                assert sizes[orders].sum() <= max_lines


def test_tiny_shape():
    inst = wh_gen.tiny()
    assert inst.n_orders == 200 and inst.n_sku == 600 and inst.n_plans == 64
    sizes = np.diff(inst.order_off)
    assert sizes.min() >= 1 and sizes.max() <= 5
    assert sorted(inst.slot_map.tolist()) == list(range(600))
    check_partition(inst, 8)


def test_midsize_shape():
    inst = wh_gen.midsize(n_plans=64)
    sizes = np.diff(inst.order_off)
    assert sizes.min() >= 1 and sizes.max() <= 12
    assert abs(sizes.mean() - 2.47) < 0.1            # truncated geometric, p = 0.4
    for o in range(0, inst.n_orders, 97):            # distinct SKUs within an order
        s = inst.line_sku[inst.order_off[o]:inst.order_off[o + 1]]
        assert len(set(s.tolist())) == len(s)
    assert len(set(inst.slot_map.tolist())) == inst.n_sku
    assert inst.slot_map.min() >= 0 and inst.slot_map.max() < inst.layout.n_loc
    # Zipf(1.1) popularity: SKU 0 is the most frequent line
    counts = np.bincount(inst.line_sku, minlength=inst.n_sku)
    assert counts.argmax() == 0
    check_partition(inst, 20, 60)


def test_abc_slotting_swaps_only_a_tenth():
    lay = wh_gen.Layout(40, 100)
    plain = wh_gen.gen_slot_abc(3, lay, 8000, 0.0)
    swapped = wh_gen.gen_slot_abc(3, lay, 8000, 0.10)
    assert (plain != swapped).sum() <= 2 * 400
    # most popular SKU sits in the depot aisle, the least popular far away
    assert plain[0] // (2 * lay.slots_per_side) == 0
    assert plain[-1] // (2 * lay.slots_per_side) == lay.n_aisles - 1


def test_paperscale_shape():
    inst = wh_gen.paperscale(n_plans=8)
    assert inst.layout.n_loc == 200_000 and inst.n_sku == 50_000
    assert 9_000 < inst.n_lines < 11_000
    check_partition(inst, 24)


def test_batched_instances_uneven():
    insts = [wh_gen.batched_instance(9, i, n_plans=2) for i in range(6)]
    assert len({(i.layout.n_aisles, i.layout.slots_per_side, i.n_orders) for i in insts}) == 6
    for inst in insts:
        assert 8 <= inst.layout.n_aisles <= 64 and 20 <= inst.layout.slots_per_side <= 200
        assert 100 <= inst.n_orders <= 5000 and inst.n_sku == inst.layout.n_loc
        check_partition(inst, 20, 60)


def test_moves_in_range():
    inst = wh_gen.tiny(n_plans=4)
    mv = wh_gen.gen_moves(7, 0, inst, 64)
    assert mv.shape == (4, 64, 4)
    assert set(np.unique(mv[..., 0]).tolist()) <= {0, 1, 2}
    ntours = np.diff(inst.plan_tour_off)
    for p in range(4):
        for t, a, b, _ in mv[p]:
            if t == 0:
                assert 0 <= a < inst.n_orders and 0 <= b < inst.n_orders
            elif t == 1:
                assert 0 <= a < inst.n_orders and 0 <= b < ntours[p]
            else:
                assert 0 <= a < inst.n_sku and 0 <= b < inst.n_sku
    assert np.array_equal(mv, wh_gen.gen_moves(7, 0, inst, 64))
    assert not np.array_equal(mv, wh_gen.gen_moves(7, 1, inst, 64))


def test_category_orders():
    """Category order books: sizes in range, SKUs distinct within an order and
    about 80 % of the lines from the order's category (s mod n_cat)."""
    inst = wh_gen.midsize_cat(seed=6, n_plans=2)
    off, lines = inst.order_off, inst.line_sku
    sizes = np.diff(off)
    assert sizes.min() >= 1 and sizes.max() <= 12 and inst.n_sku == 8000
    check_partition(inst, 20, 60)
    share = []
    for o in range(inst.n_orders):
        ls = lines[off[o]:off[o + 1]]
        assert len(set(ls.tolist())) == len(ls)
        share.append(np.bincount(ls % 64).max() / len(ls))
    assert 0.8 < float(np.mean(share)) < 0.97
    a = wh_gen.gen_orders_cat(3, 100, 1000, 8, 0.4, 1.0, 10, 0.0)
    b = wh_gen.gen_orders_cat(3, 100, 1000, 8, 0.4, 1.0, 10, 1.0)
    assert np.array_equal(np.diff(a[0]), np.diff(b[0]))          # sizes drawn from their own stream
    for o in range(100):                                          # p_in = 1: one category per order
        assert len(set((b[1][b[0][o]:b[0][o + 1]] % 10).tolist())) == 1


def test_sign_rows_and_relocations():
    s = wh_gen.gen_signs(9, (500, 32))
    assert s.dtype == np.int8 and set(np.unique(s).tolist()) == {-1, 1}
    assert abs(float(s.mean())) < 0.05 and np.array_equal(s, wh_gen.gen_signs(9, (500, 32)))
    inst = wh_gen.tiny(seed=3, n_plans=4)
    mv = wh_gen.gen_relocations(2, 0, inst, 16)
    assert (mv[..., 0] == 3).all()
    assert np.isin(mv[..., 1], np.unique(inst.line_sku)).all()
    assert ((mv[..., 2] >= 0) & (mv[..., 2] < inst.layout.n_loc)).all()
    assert (mv[..., 3] == np.arange(4)[:, None]).all()
