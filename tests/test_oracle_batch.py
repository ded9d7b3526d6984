"""Pins of the oracle's seed-and-grow batch formation against its definition:
the output is a partition of the orders within the capacities, every tour
starts with the longest remaining order alone, every insertion is the fitting
order that lengthens the tour least (ties: lowest id), and a tour closes only
at capacity or when no remaining order fits.  Tour lengths come from the
Ratliff-Rosenthal DP, which is pinned to Held-Karp elsewhere."""
import numpy as np
import pytest

import oracle
import wh_gen


def locs_of(inst, orders):
    return [int(inst.slot_map[s]) for o in orders for s in inst.line_sku[inst.order_off[o]:inst.order_off[o + 1]]]


def lines_of(inst, o):
    return int(inst.order_off[o + 1] - inst.order_off[o])


def small_instance(seed, n_orders):
    lay = wh_gen.Layout(12, 20)
    rng = np.random.default_rng(seed)
    sizes = rng.integers(1, 6, n_orders)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    n_sku = lay.n_loc
    lines = np.concatenate([rng.choice(n_sku, int(k), replace=False) for k in sizes]).astype(np.int32)
    slot = rng.permutation(lay.n_loc).astype(np.int32)
    return wh_gen.Instance(lay, n_sku, off, lines, slot, np.zeros(2, np.int32), np.zeros(2, np.int32),
                           np.zeros(0, np.int32))


@pytest.mark.parametrize("caps", [(6, 0), (0, 14), (5, 12), (1, 0)])
def test_seed_and_grow_follows_its_definition(caps):
    max_orders, max_lines = caps
    inst = small_instance(sum(caps), 60)
    lay = inst.layout
    to, seq = oracle.batch_grow(lay, inst.order_off, inst.line_sku, inst.n_sku, inst.slot_map, max_orders, max_lines)
    # a partition of the orders
    assert sorted(seq.tolist()) == list(range(inst.n_orders))
    assert to[0] == 0 and to[-1] == inst.n_orders and (np.diff(to) > 0).all()
    alone = [oracle.rr(lay, locs_of(inst, [o])) for o in range(inst.n_orders)]
    left = set(range(inst.n_orders))
    for t in range(len(to) - 1):
        tour = seq[to[t]:to[t + 1]].tolist()
        # the seed: the longest remaining order alone, ties to the lowest id
        best = max(alone[o] for o in left)
        assert tour[0] == min(o for o in left if alone[o] == best)
        left.discard(tour[0])
        cur = [tour[0]]
        lines = lines_of(inst, tour[0])
        for nxt in tour[1:] + [None]:
            fits = [o for o in sorted(left) if max_lines == 0 or lines + lines_of(inst, o) <= max_lines]
            at_cap = max_orders > 0 and len(cur) >= max_orders
            if nxt is None:
                # closed: at capacity, or nothing fits
                assert at_cap or not fits
                break
            assert not at_cap and nxt in fits
            cost = {o: oracle.rr(lay, locs_of(inst, cur + [o])) for o in fits}
            least = min(cost.values())
            assert nxt == min(o for o in fits if cost[o] == least)
            cur.append(nxt)
            left.discard(nxt)
            lines += lines_of(inst, nxt)
        if max_orders:
            assert len(tour) <= max_orders
        if max_lines:
            assert len(tour) == 1 or sum(lines_of(inst, o) for o in tour) <= max_lines
    assert not left


def test_batching_beats_random_plans():
    """Formed tours are shorter than random tours of the same capacity (the
    purpose of the method: orders picked together whose picks are close)."""
    inst = wh_gen.tiny(seed=3, n_plans=16)
    to, seq = oracle.batch_grow(inst.layout, inst.order_off, inst.line_sku, inst.n_sku, inst.slot_map, 8, 0)
    formed = wh_gen.Instance(inst.layout, inst.n_sku, inst.order_off, inst.line_sku, inst.slot_map,
                             np.asarray([0, len(to) - 1], np.int32), to, seq)
    grown = oracle.eval_plans(formed)[3][0]
    random_plans = oracle.eval_plans(inst)[3]
    assert grown < 0.8 * random_plans.min()
