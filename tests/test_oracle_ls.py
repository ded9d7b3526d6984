"""Pins of the oracle's local-search step: the applied move is the argmin
rule computed here from the move deltas, the new plan cost equals the old
cost plus that delta, plans stay partitions of the order book, and a run of
steps never increases the optimal cost."""
import numpy as np

import oracle
import wh_gen


def with_plans(inst, to, seq, smap=None):
    return wh_gen.Instance(inst.layout, inst.n_sku, inst.order_off, inst.line_sku,
                           inst.slot_map if smap is None else smap, inst.plan_tour_off, to, seq)


def test_ls_step_applies_argmin_and_delta():
    inst = wh_gen.tiny(seed=11, n_plans=6)
    rng = np.random.default_rng(3)
    maps = np.stack([rng.permutation(inst.layout.n_loc)[: inst.n_sku] for _ in range(6)]).astype(np.int32).ravel()
    M = 32
    mv = wh_gen.gen_moves(5, 0, inst, M)
    mv[..., 3] = np.arange(6)[:, None]
    mv = mv.reshape(-1, 4)
    d, st = oracle.eval_moves(inst, mv, 8, 0, slot_map=maps, slot_map_stride=inst.n_sku)
    to, seq, smap, applied = oracle.ls_step(inst, mv, M, 8, 0, slot_map=maps, slot_map_stride=inst.n_sku)
    before = oracle.eval_plans(inst, slot_map=maps, slot_map_stride=inst.n_sku)
    after = oracle.eval_plans(with_plans(inst, to, seq, smap), slot_map=smap, slot_map_stride=inst.n_sku)
    for p in range(6):
        k = np.arange(p * M, (p + 1) * M)
        ok = (st[k] == 0) & (d[k, 1] < 0)
        want = -1 if not ok.any() else int(np.flatnonzero(ok)[np.argmin(d[k, 1][ok])])
        assert applied[p] == want
        if want >= 0:
            assert after[3][p] == before[3][p] + d[p * M + want, 1]
            assert after[2][p] == before[2][p] + d[p * M + want, 0]
        else:
            assert after[3][p] == before[3][p]
        s0, s1 = to[inst.plan_tour_off[p]], to[inst.plan_tour_off[p + 1]]
        assert sorted(seq[s0:s1].tolist()) == list(range(inst.n_orders))
    assert (applied >= 0).sum() >= 4


def test_ls_trajectory_is_monotone():
    inst = wh_gen.tiny(seed=12, n_plans=3)
    M = 16
    cur = inst
    cost = oracle.eval_plans(cur)[3].copy()
    for step in range(6):
        mv = wh_gen.gen_moves(9, step, cur, M)
        mv[..., 3] = np.arange(3)[:, None]
        to, seq, _, applied = oracle.ls_step(cur, mv.reshape(-1, 4), M, 8)
        cur = with_plans(cur, to, seq)
        new = oracle.eval_plans(cur)[3]
        assert (new <= cost).all()
        assert ((new < cost) == (applied >= 0)).all()
        cost = new.copy()


def test_ls_step_with_relocations():
    """Relocations into empty locations mixed with the other moves: the
    applied one follows the argmin rule, a relocation sets exactly the SKU's
    slot and keeps the slotting injective."""
    base = wh_gen.tiny(seed=13, n_plans=4)
    lay = wh_gen.Layout(20, 30)
    inst = wh_gen.Instance(lay, base.n_sku, base.order_off, base.line_sku, base.slot_map, base.plan_tour_off,
                           base.tour_off, base.order_seq)
    rng = np.random.default_rng(4)
    maps = np.stack([rng.permutation(lay.n_loc)[:inst.n_sku] for _ in range(4)]).astype(np.int32)
    M = 48
    mv = np.concatenate([wh_gen.gen_moves(6, 0, inst, 16), wh_gen.gen_relocations(7, 0, inst, 32)], axis=1)
    mv[..., 3] = np.arange(4)[:, None]
    mv = mv.reshape(-1, 4)
    d, st = oracle.eval_moves(inst, mv, 8, 0, slot_map=maps.ravel(), slot_map_stride=inst.n_sku)
    to, seq, smap, applied = oracle.ls_step(inst, mv, M, 8, 0, slot_map=maps.ravel(), slot_map_stride=inst.n_sku)
    smap = smap.reshape(4, -1)
    n_reloc = 0
    for p in range(4):
        k = np.arange(p * M, (p + 1) * M)
        ok = (st[k] == 0) & (d[k, 1] < 0)
        want = -1 if not ok.any() else int(np.flatnonzero(ok)[np.argmin(d[k, 1][ok])])
        assert applied[p] == want
        assert len(set(smap[p].tolist())) == inst.n_sku
        if want >= 0 and mv[p * M + want, 0] == 3:
            n_reloc += 1
            s, loc = mv[p * M + want, 1], mv[p * M + want, 2]
            changed = np.flatnonzero(smap[p] != maps[p])
            assert changed.tolist() == [s] and smap[p, s] == loc
    assert n_reloc >= 1
