"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tour and plan costs are integers, so every comparison is exact (bit-equal
int32 / int64).  Sizes: every tour of the tiny workload; 256 plans of the
mid-size one; the full 4,096-plan mid-size launch (the benchmark's launch)
with sampled plans re-scored by the oracle and size-independent properties on
all outputs; long tours of the paper-scale workload; hand-built edge cases.
"""
import json
import os

import numpy as np
import pytest

import oracle
import wh_gen

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_tours.json")


def gpu_eval(wh, inst, mask=3, slot_map=None, stride=0, prefill=None):
    import torch
    lay = wh.Layout.of(inst.layout)
    prob = wh.to_device(inst, slot_map=slot_map, slot_map_stride=stride)
    costs = wh.alloc_costs(prob.n_tours, prob.n_plans)
    if prefill is not None:
        for t in (costs.tour_s, costs.tour_rr, costs.plan_s, costs.plan_rr):
            t.fill_(prefill)
    lay.eval_plans(prob, costs, mask)
    torch.cuda.synchronize()
    status = lay.status()
    lay.close()
    nt, npl = prob.n_tours, prob.n_plans
    return (costs.tour_s[:nt].cpu().numpy(), costs.tour_rr[:nt].cpu().numpy(),
            costs.plan_s[:npl].cpu().numpy(), costs.plan_rr[:npl].cpu().numpy(), status)


def assert_exact(got, want):
    names = ("tour_s", "tour_rr", "plan_s", "plan_rr")
    for n, g, w in zip(names, got[:4], want):
        assert g.shape == w.shape, n
        bad = np.nonzero(g != w)[0]
        assert bad.size == 0, f"{n}: {bad.size} mismatches, first at {bad[:5]}: got {g[bad[:5]]} want {w[bad[:5]]}"


def make_instance(lay, orders, slot_map, plans, n_sku=None):
    """Instance from explicit orders (lists of SKUs) and plans (lists of
    tours, each a list of order ids)."""
    off = np.zeros(len(orders) + 1, np.int32)
    off[1:] = np.cumsum([len(o) for o in orders])
    lines = np.asarray([s for o in orders for s in o], np.int32)
    pto, to, seq = [0], [0], []
    for plan in plans:
        for tour in plan:
            seq.extend(tour)
            to.append(len(seq))
        pto.append(len(to) - 1)
    return wh_gen.Instance(lay, n_sku or len(slot_map), off, lines, np.asarray(slot_map, np.int32),
                           np.asarray(pto, np.int32), np.asarray(to, np.int32), np.asarray(seq, np.int32))


# ------------------------------------------------------------------ workloads

def test_tiny_every_tour(gpu_lib):
    inst = wh_gen.tiny(seed=1)
    got = gpu_eval(gpu_lib, inst)
    assert got[4] == 0
    assert_exact(got, oracle.eval_plans(inst))


@pytest.mark.parametrize("seed", [2, 11, 12])
def test_midsize_256_plans(gpu_lib, seed):
    inst = wh_gen.midsize(seed=seed, n_plans=256)
    got = gpu_eval(gpu_lib, inst)
    assert got[4] == 0
    assert_exact(got, oracle.eval_plans(inst))


def test_midsize_full_launch_sampled(gpu_lib):
    """The benchmark's launch: 4,096 plans in one call.  48 sampled plans are
    re-scored by the oracle; every output is checked for the properties that
    hold at any size."""
    inst = wh_gen.midsize(seed=2)
    ts, tr, ps, pr, status = gpu_eval(gpu_lib, inst)
    assert status == 0
    assert (tr >= 0).all() and (tr <= ts).all()
    assert (ts % 2 == 0).all() and (tr % 2 == 0).all()
    seg = inst.plan_tour_off
    assert np.array_equal(ps, np.add.reduceat(ts.astype(np.int64), seg[:-1]))
    assert np.array_equal(pr, np.add.reduceat(tr.astype(np.int64), seg[:-1]))
    rng = np.random.default_rng(0)
    sample = np.sort(rng.choice(inst.n_plans, 48, replace=False))
    sub = inst.subset_plans(sample)
    want = oracle.eval_plans(sub)
    idx = np.concatenate([np.arange(seg[p], seg[p + 1]) for p in sample])
    assert np.array_equal(ts[idx], want[0]) and np.array_equal(tr[idx], want[1])
    assert np.array_equal(ps[sample], want[2]) and np.array_equal(pr[sample], want[3])


def test_paperscale_long_tours(gpu_lib):
    inst = wh_gen.paperscale(seed=4, n_plans=24)
    assert (inst.tour_lines() > 64).mean() > 0.1       # the long-tour kernel runs
    got = gpu_eval(gpu_lib, inst)
    assert got[4] == 0
    assert_exact(got, oracle.eval_plans(inst))


@pytest.mark.parametrize("i", [0, 1, 2, 3])
def test_batched_instances_one_by_one(gpu_lib, i):
    inst = wh_gen.batched_instance(9, i, n_plans=16)
    got = gpu_eval(gpu_lib, inst)
    assert got[4] == 0
    assert_exact(got, oracle.eval_plans(inst))


@pytest.mark.parametrize("lay", [wh_gen.Layout(6, 8, 5, 2, 4), wh_gen.Layout(20, 4, 1, 3, 6),
                                 wh_gen.Layout(1, 10), wh_gen.Layout(64, 200)])
def test_other_geometries(gpu_lib, lay):
    rng = np.random.default_rng(lay.n_aisles)
    n_sku = min(lay.n_loc, 500)
    slot = rng.permutation(lay.n_loc)[:n_sku]
    orders = [rng.integers(0, n_sku, size=int(rng.integers(1, 6))).tolist() for _ in range(120)]
    plans = []
    for _ in range(10):
        perm = rng.permutation(len(orders)).tolist()
        cuts = np.sort(rng.choice(np.arange(1, len(orders)), 20, replace=False)).tolist()
        plans.append([perm[a:b] for a, b in zip([0] + cuts, cuts + [len(orders)])])
    inst = make_instance(lay, orders, slot, plans, n_sku)
    got = gpu_eval(gpu_lib, inst)
    assert got[4] == 0
    assert_exact(got, oracle.eval_plans(inst))


def test_routing_mask_selects_outputs(gpu_lib):
    inst = wh_gen.tiny(seed=5, n_plans=7)
    full = gpu_eval(gpu_lib, inst, mask=3)
    s_only = gpu_eval(gpu_lib, inst, mask=1, prefill=-7)
    r_only = gpu_eval(gpu_lib, inst, mask=2, prefill=-7)
    assert np.array_equal(s_only[0], full[0]) and np.array_equal(s_only[2], full[2])
    assert (s_only[1] == -7).all() and (s_only[3] == -7).all()
    assert np.array_equal(r_only[1], full[1]) and np.array_equal(r_only[3], full[3])
    assert (r_only[0] == -7).all() and (r_only[2] == -7).all()


def test_per_plan_slot_maps(gpu_lib):
    for inst in (wh_gen.tiny(seed=6, n_plans=9), wh_gen.paperscale(seed=6, n_plans=5)):
        rng = np.random.default_rng(1)
        maps = np.stack([rng.permutation(inst.layout.n_loc)[: inst.n_sku] for _ in range(inst.n_plans)])
        maps = np.ascontiguousarray(maps.astype(np.int32).ravel())
        got = gpu_eval(gpu_lib, inst, slot_map=maps, stride=inst.n_sku)
        assert got[4] == 0
        assert_exact(got, oracle.eval_plans(inst, slot_map=maps, slot_map_stride=inst.n_sku))


# ----------------------------------------------------------------- edge cases

def test_worked_tours_and_edges(gpu_lib):
    g = json.load(open(GOLDEN))
    lay = wh_gen.Layout(**g["layout"])
    slot = np.arange(lay.n_loc, dtype=np.int32)           # SKU id = location id
    L = lay.slots_per_side
    orders = [[lay.loc(a, y - 1) for a, y in t["picks"]] for t in g["tours"]]
    worked = list(range(len(orders)))
    extra = {
        "aisle0": [lay.loc(0, 3), lay.loc(0, 20, 1)],
        "single_front": [lay.loc(4, 0)],
        "single_back": [lay.loc(9, L - 1)],
        "last_aisle": [lay.loc(9, k) for k in range(0, L, 3)],
        "dups": [lay.loc(3, 5), lay.loc(3, 5, 1), lay.loc(3, 5)],
        "zero_lines": [],
        "every_aisle_front": [lay.loc(a, 0) for a in range(10)],
        "every_aisle_back": [lay.loc(a, L - 1, a & 1) for a in range(10)],
    }
    base = len(orders)
    orders += list(extra.values())
    rng = np.random.default_rng(3)
    # tours whose line counts sit on the kernel's size boundaries
    sized = []
    for n in (1, 15, 16, 17, 31, 32, 33, 63, 64, 65, 128, 300, 2048):
        sized.append(len(orders))
        orders.append(rng.integers(0, lay.n_loc, size=n).tolist())
    tours = [[i] for i in worked] + [[base + i] for i in range(len(extra))] + [[i] for i in sized]
    tours += [[], [0, 1, 2], [base + 5, base + 5], [sized[8], sized[0]], [base, 0, base + 4]]
    plans = [tours[:9], tours[9:20], [], tours[20:], [[]]]
    inst = make_instance(lay, orders, slot, plans)
    got = gpu_eval(gpu_lib, inst)
    assert got[4] == 0
    want = oracle.eval_plans(inst)
    assert_exact(got, want)
    for i, t in enumerate(g["tours"]):
        assert got[0][i] == t["sshape"] and got[1][i] == t["optimal"]


def test_tour_too_long_is_flagged(gpu_lib):
    import paper_2110_13693_gb300 as wh
    lay = wh_gen.Layout(10, 30)
    slot = np.arange(lay.n_loc, dtype=np.int32)
    orders = [list(range(600)) * 3 + [1, 2], [5]]      # 1,802 lines
    orders.append(list(range(300)))                    # with order 0: 2,102 lines
    inst = make_instance(lay, orders, slot, [[[0], [1]], [[0, 2], [1]]])
    ts, tr, ps, pr, status = gpu_eval(gpu_lib, inst)
    assert status & wh.WH_STATUS_TOUR_TOO_LONG
    assert ts[2] == -1 and tr[2] == -1
    want = oracle.eval_plans(inst.subset_plans([0]))
    assert ts[0] == want[0][0] and tr[1] == want[1][1] and pr[0] == want[3][0]


@pytest.mark.parametrize("mask", [3, 1])
def test_bad_ids_are_flagged_not_faulted(gpu_lib, mask):
    """Invalid ids are flagged and their tours report -1, under both rules
    and under the S-shape rule alone (its own kernels)."""
    import paper_2110_13693_gb300 as wh
    lay = wh_gen.Layout(10, 30)
    slot = np.arange(lay.n_loc, dtype=np.int32)
    good = make_instance(lay, [[1, 2], [3], [4]], slot, [[[0], [1, 2]]])
    want = oracle.eval_plans(good)
    col = 1 if mask == 3 else 0           # the optimal cost, or the S-shape one

    def run(inst):
        got = gpu_eval(gpu_lib, inst, mask=mask)
        return got[col], got[4]

    bad_order = make_instance(lay, [[1, 2], [3], [4]], slot, [[[0], [1, 7]]])
    c, st = run(bad_order)
    assert st & wh.WH_STATUS_BAD_ORDER and c[1] == -1 and c[0] == want[col][0]

    bad_sku = make_instance(lay, [[1, 2], [3], [4]], slot, [[[0], [1, 2]]])
    bad_sku.line_sku = np.asarray([1, 2, 3, 9999], np.int32)
    c, st = run(bad_sku)
    assert st & wh.WH_STATUS_BAD_SKU and c[1] == -1 and c[0] == want[col][0]

    bad_loc = make_instance(lay, [[1, 2], [3], [4]], slot.copy(), [[[0], [1, 2]]])
    bad_loc.slot_map[4] = lay.n_loc + 5
    c, st = run(bad_loc)
    assert st & wh.WH_STATUS_BAD_LOC and c[1] == -1

    bad_off = make_instance(lay, [[1, 2], [3], [4]], slot, [[[0], [1, 2]]])
    bad_off.tour_off = np.asarray([0, 2, 1], np.int32)
    c, st = run(bad_off)
    assert st & wh.WH_STATUS_BAD_OFFSET and c[1] == -1


def test_repeatable(gpu_lib):
    inst = wh_gen.midsize(seed=7, n_plans=64)
    a = gpu_eval(gpu_lib, inst)
    b = gpu_eval(gpu_lib, inst)
    for x, y in zip(a[:4], b[:4]):
        assert np.array_equal(x, y)


def test_large_order_book_global_tables(gpu_lib):
    """An order book too large for shared memory (the kernel reads offsets
    and 32-bit keys from global memory) on a layout that uses 16-bit keys."""
    lay = wh_gen.Layout(60, 150)
    off, lines = wh_gen.gen_orders(21, 24000, 18000, 12, 0.4, 1.1)
    slot = wh_gen.gen_slot_abc(21, lay, 18000, 0.1)
    pto, to, seq = wh_gen.gen_plans(21, 1, off, 3, 20, 60)
    inst = wh_gen.Instance(lay, 18000, off, lines, slot, pto, to, seq)
    assert 4 * (inst.n_orders + inst.n_lines) > 112 * 1024
    got = gpu_eval(gpu_lib, inst)
    assert got[4] == 0
    assert_exact(got, oracle.eval_plans(inst))


def random_instance(lay, seed, n_orders=300, n_plans=8, max_tour=40):
    rng = np.random.default_rng(seed)
    n_sku = min(lay.n_loc, 2000)
    slot = rng.permutation(lay.n_loc)[:n_sku]
    orders = [rng.integers(0, n_sku, size=int(rng.integers(1, 8))).tolist() for _ in range(n_orders)]
    plans = []
    for _ in range(n_plans):
        perm = rng.permutation(n_orders).tolist()
        cuts, at = [], 0
        while at < n_orders:
            at += int(rng.integers(1, max_tour + 1))
            cuts.append(min(at, n_orders))
        plans.append([perm[a:b] for a, b in zip([0] + cuts[:-1], cuts)])
    return make_instance(lay, orders, slot, plans, n_sku)


def sshape_cases():
    yield "tiny", wh_gen.tiny(seed=31, n_plans=16), None
    yield "midsize", wh_gen.midsize(seed=32, n_plans=64), None
    inst = wh_gen.paperscale(seed=33, n_plans=6)
    yield "paperscale", inst, None
    rng = np.random.default_rng(3)
    maps = np.stack([rng.permutation(inst.layout.n_loc)[: inst.n_sku] for _ in range(inst.n_plans)])
    yield "paperscale_maps", inst, np.ascontiguousarray(maps.astype(np.int32).ravel())
    # the widest bitmap (2,048 aisles = 64 words) and one aisle past it (the
    # general kernel takes over), long tours of up to 40 orders
    yield "a2048", random_instance(wh_gen.Layout(2048, 3), 34), None
    yield "a2049", random_instance(wh_gen.Layout(2049, 3), 35), None
    yield "a1", random_instance(wh_gen.Layout(1, 40), 36), None


@pytest.mark.parametrize("case", [c[0] for c in sshape_cases()])
def test_sshape_only_kernel(gpu_lib, case):
    """Routing mask S-shape only runs the sort-free kernel: tour and plan
    S-shape costs bit-equal to the oracle's, the optimal outputs untouched."""
    name, inst, maps = next(c for c in sshape_cases() if c[0] == case)
    stride = inst.n_sku if maps is not None else 0
    got = gpu_eval(gpu_lib, inst, mask=1, slot_map=maps, stride=stride, prefill=-7)
    want = oracle.eval_plans(inst, slot_map=maps, slot_map_stride=stride) if maps is not None else oracle.eval_plans(inst)
    assert got[4] == 0
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[2], want[2])
    assert (got[1] == -7).all() and (got[3] == -7).all()


def test_sshape_only_large_order_book(gpu_lib):
    lay = wh_gen.Layout(60, 150)
    off, lines = wh_gen.gen_orders(22, 24000, 18000, 12, 0.4, 1.1)
    slot = wh_gen.gen_slot_abc(22, lay, 18000, 0.1)
    pto, to, seq = wh_gen.gen_plans(22, 1, off, 3, 20, 60)
    inst = wh_gen.Instance(lay, 18000, off, lines, slot, pto, to, seq)
    got = gpu_eval(gpu_lib, inst, mask=1, prefill=-7)
    want = oracle.eval_plans(inst)
    assert got[4] == 0
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[2], want[2])


def test_host_pipeline_matches_oracle(gpu_lib):
    """HostPipeline (copies of one batch overlapping the evaluation of the
    previous one) returns every batch's plan costs, equal to the oracle's."""
    import torch
    wh = gpu_lib
    insts = [wh_gen.midsize(seed=40 + i, n_plans=48) for i in range(3)]
    lay = wh.Layout.of(insts[0].layout)
    host, bufs, outs = [], [], []
    for inst in insts:
        host.append(wh.DeviceProblem(*(torch.as_tensor(getattr(inst, f)).pin_memory() for f in
                                       ("order_off", "line_sku", "slot_map", "plan_tour_off", "tour_off",
                                        "order_seq")), inst.n_sku))
        prob = wh.to_device(inst)
        bufs.append((prob, wh.alloc_costs(prob.n_tours, prob.n_plans)))
        outs.append(torch.zeros((2, inst.n_plans), dtype=torch.int64).pin_memory())
    pipe = wh.HostPipeline(lay, bufs, 3)
    tickets = [pipe.submit(host[i % 3], outs[i % 3])[0] for i in range(6)]
    for t in tickets:
        pipe.wait(t)
    for inst, out in zip(insts, outs):
        want = oracle.eval_plans(inst)
        assert np.array_equal(out[0].numpy(), want[2]) and np.array_equal(out[1].numpy(), want[3])
    assert lay.status() == 0
    lay.close()


def test_host_pipeline_16bit_order_ids(gpu_lib):
    """Order ids shipped as 16 bits and widened on the device give the same
    plan costs as the int32 path; ids above 32,767 survive the widening."""
    import torch
    wh = gpu_lib
    inst = wh_gen.midsize(seed=44, n_plans=32)
    lay = wh.Layout.of(inst.layout)
    fields = ("order_off", "line_sku", "slot_map", "plan_tour_off", "tour_off")
    host = wh.DeviceProblem(*(torch.as_tensor(getattr(inst, f)).pin_memory() for f in fields),
                            torch.as_tensor(inst.order_seq.astype(np.uint16).view(np.int16)).pin_memory(),
                            inst.n_sku)
    prob = wh.to_device(inst)
    out = torch.zeros((2, inst.n_plans), dtype=torch.int64).pin_memory()
    pipe = wh.HostPipeline(lay, [(prob, wh.alloc_costs(prob.n_tours, prob.n_plans))], 3)
    ticket, h2d, _ = pipe.submit(host, out)
    pipe.wait(ticket)
    assert h2d == sum(getattr(inst, f).nbytes for f in fields) + 2 * inst.order_seq.size
    assert np.array_equal(prob.order_seq.cpu().numpy(), inst.order_seq)
    want = oracle.eval_plans(inst)
    assert np.array_equal(out[0].numpy(), want[2]) and np.array_equal(out[1].numpy(), want[3])
    # the widening alone, on values across the whole 16-bit range and a ragged tail
    vals = np.arange(0, 65536, 7, dtype=np.uint16)
    src_all = torch.as_tensor(vals.view(np.int16)).cuda()
    for off in (0, 1, 3):                       # 1 and 3: unaligned buffers take the scalar path
        src = src_all[off:]
        dst = torch.full((src.numel() + off,), -1, dtype=torch.int32, device="cuda")[off:]
        wh._check(wh.load().wh_widen_u16(wh.ctypes.c_void_p(src.data_ptr()), wh.ctypes.c_void_p(dst.data_ptr()),
                                         src.numel(), None), "wh_widen_u16")
        torch.cuda.synchronize()
        assert np.array_equal(dst.cpu().numpy(), vals[off:].astype(np.int32))
    assert lay.status() == 0
    lay.close()


def _wide_instance(n_plans=3):
    """Tours of at most 64 lines that visit more than 32 aisles (the
    per-thread record slots): 64 aisles, one-line orders spread over them."""
    lay = wh_gen.Layout(64, 20)
    rng = np.random.default_rng(40)
    n_sku = lay.n_loc
    slot = rng.permutation(lay.n_loc).astype(np.int32)
    # SKU s sits at location slot[s]; order o holds SKUs of aisle o % 64
    by_aisle = [np.nonzero(slot // (2 * lay.slots_per_side) == a)[0] for a in range(64)]
    orders = [[int(rng.choice(by_aisle[o % 64]))] + ([int(rng.choice(by_aisle[(o * 7) % 64]))] if o % 3 == 0 else [])
              for o in range(400)]
    plans = []
    for p in range(n_plans):
        perm = rng.permutation(len(orders)).tolist()
        sizes = [40, 33, 20, 47, 5]            # orders per tour (<= 64 lines each)
        tours, i = [], 0
        while i < len(perm):
            k = sizes[len(tours) % len(sizes)]
            tours.append(perm[i:i + k])
            i += k
        plans.append(tours)
    return make_instance(lay, orders, slot, plans, n_sku)


def test_tours_over_the_record_slots_go_to_the_long_pass(gpu_lib):
    """Tours of <= 64 lines with more pick aisles than a thread keeps records
    for are handed to the long-tour pass: single launch, batched launch and
    per-plan slottings all equal the oracle."""
    import torch
    inst = _wide_instance()
    want = oracle.eval_plans(inst)
    aisles = [len({int(inst.slot_map[s]) // 40 for o in inst.order_seq[inst.tour_off[t]:inst.tour_off[t + 1]]
                   for s in inst.line_sku[inst.order_off[o]:inst.order_off[o + 1]]}) for t in range(inst.n_tours)]
    lines = inst.tour_lines()
    assert sum(1 for a, n in zip(aisles, lines) if a > 32 and n <= 64) >= 6
    got = gpu_eval(gpu_lib, inst)
    assert got[4] == 0
    assert_exact(got, want)
    maps = np.tile(inst.slot_map, (inst.n_plans, 1)).ravel().astype(np.int32)
    got = gpu_eval(gpu_lib, inst, slot_map=maps, stride=inst.n_sku)
    assert got[4] == 0
    assert_exact(got, want)
    wh = gpu_lib
    lay = inst.layout
    prob = wh.to_device(inst)
    costs = wh.alloc_costs(prob.n_tours, prob.n_plans)
    b = wh.Batch([((lay.n_aisles, lay.slots_per_side, lay.aisle_pitch, lay.slot_pitch, lay.cross_aisle_width),
                   prob, costs)])
    b.eval(3)
    torch.cuda.synchronize()
    assert b.status() == 0
    got = (costs.tour_s[:prob.n_tours].cpu().numpy(), costs.tour_rr[:prob.n_tours].cpu().numpy(),
           costs.plan_s[:prob.n_plans].cpu().numpy(), costs.plan_rr[:prob.n_plans].cpu().numpy())
    assert_exact(got, want)
    b.close()
