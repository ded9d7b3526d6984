"""Seed-and-grow batch formation on the GPU (one CTA per slotting) against
the oracle: identical tours, order by order, under several slottings,
capacities and edge cases."""
import numpy as np
import pytest

import oracle
import wh_gen

pytestmark = pytest.mark.gpu


def run(wh, inst, maps, max_orders, max_lines):
    import torch
    lay = wh.Layout.of(inst.layout)
    prob = wh.to_device(inst)
    tour_off, order_seq, n_tours = lay.batch_grow(prob, torch.as_tensor(maps).cuda(), max_orders, max_lines)
    torch.cuda.synchronize()
    st = lay.status()
    lay.close()
    return tour_off.cpu().numpy(), order_seq.cpu().numpy(), n_tours.cpu().numpy(), st


def check(wh, inst, maps, max_orders, max_lines):
    to, seq, nt, st = run(wh, inst, maps, max_orders, max_lines)
    assert st == 0
    for p in range(maps.shape[0]):
        wto, wseq = oracle.batch_grow(inst.layout, inst.order_off, inst.line_sku, inst.n_sku, maps[p],
                                      max_orders, max_lines)
        assert nt[p] == len(wto) - 1, p
        assert np.array_equal(to[p, :nt[p] + 1], wto), p
        assert np.array_equal(seq[p], wseq), (p, np.nonzero(seq[p] != wseq)[0][:5])
    return to, seq, nt


@pytest.mark.parametrize("caps", [(8, 0), (0, 20), (5, 14), (1, 0)])
def test_tiny_several_slottings(gpu_lib, caps):
    inst = wh_gen.tiny(seed=11, n_plans=1)
    rng = np.random.default_rng(sum(caps))
    maps = np.stack([inst.slot_map] + [rng.permutation(inst.layout.n_loc)[: inst.n_sku] for _ in range(5)])
    check(gpu_lib, inst, maps.astype(np.int32), *caps)


def test_midsize_layout_capped(gpu_lib):
    """40 aisles x 100 slots, Zipf / ABC slotting and a perturbed one, tours of
    <= 20 orders / 60 lines, 500 orders."""
    full = wh_gen.midsize(seed=12, n_plans=1)
    n = 500
    inst = wh_gen.Instance(full.layout, full.n_sku, full.order_off[:n + 1].copy(),
                           full.line_sku[:full.order_off[n]].copy(), full.slot_map, full.plan_tour_off,
                           full.tour_off, full.order_seq)
    rng = np.random.default_rng(3)
    alt = inst.slot_map.copy()
    i, j = rng.integers(0, inst.n_sku, 400), rng.integers(0, inst.n_sku, 400)
    for a, b in zip(i, j):
        alt[a], alt[b] = alt[b], alt[a]
    check(gpu_lib, inst, np.stack([inst.slot_map, alt]).astype(np.int32), 20, 60)


def test_empty_orders_and_errors(gpu_lib):
    import paper_2110_13693_gb300 as wh
    lay = wh_gen.Layout(6, 10)
    sizes = [3, 0, 2, 0, 5, 1]
    rng = np.random.default_rng(0)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    lines = rng.integers(0, lay.n_loc, off[-1]).astype(np.int32)
    slot = np.arange(lay.n_loc, dtype=np.int32)
    inst = wh_gen.Instance(lay, lay.n_loc, off, lines, slot, np.zeros(2, np.int32), np.zeros(2, np.int32),
                           np.zeros(0, np.int32))
    check(gpu_lib, inst, slot[None], 3, 0)
    # an invalid slotting: that slotting reports -1 and a status bit, the other is scored
    bad = slot.copy()
    bad[lines[0]] = lay.n_loc + 3
    to, seq, nt, st = run(gpu_lib, inst, np.stack([slot, bad]), 3, 0)
    assert nt[1] == -1 and nt[0] > 0 and st & wh.WH_STATUS_BAD_LOC
