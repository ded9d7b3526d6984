"""Batched persistent launch: many uneven instances in one call, eager and
replayed from a CUDA graph, under several launch shapes and the autotuner;
bit-exact against the CPU oracle and against one-instance calls."""
import json
import os

import numpy as np
import pytest

import oracle
import wh_gen

pytestmark = pytest.mark.gpu


def build_batch(wh, insts, dev="cuda", id16=False):
    """Batch over device copies of `insts`; with id16 each instance passes
    its order ids only as 16-bit values (no int32 copy)."""
    import torch
    items = []
    for inst in insts:
        lay = inst.layout
        desc = (lay.n_aisles, lay.slots_per_side, lay.aisle_pitch, lay.slot_pitch, lay.cross_aisle_width)
        prob = wh.to_device(inst, dev)
        if id16:
            seq16 = torch.as_tensor(np.asarray(inst.order_seq).astype(np.uint16).view(np.int16)).to(dev)
            prob.order_seq, prob.order_seq16 = None, seq16
        costs = wh.alloc_costs(prob.n_tours, prob.n_plans, dev)
        for t in (costs.tour_s, costs.tour_rr, costs.plan_s, costs.plan_rr):
            t.fill_(-99)
        items.append((desc, prob, costs))
    return wh.Batch(items), items


def results(items, i):
    _, prob, c = items[i]
    return (c.tour_s[:prob.n_tours].cpu().numpy(), c.tour_rr[:prob.n_tours].cpu().numpy(),
            c.plan_s[:prob.n_plans].cpu().numpy(), c.plan_rr[:prob.n_plans].cpu().numpy())


def assert_same(got, want, tag):
    for name, g, w in zip(("tour_s", "tour_rr", "plan_s", "plan_rr"), got, want):
        assert np.array_equal(g, w), f"{tag}: {name} differs"


def test_batch_matches_oracle_eager_and_graph(gpu_lib):
    import torch
    insts = [wh_gen.batched_instance(9, i, n_plans=6) for i in range(24)]
    want = [oracle.eval_plans(inst) for inst in insts]
    batch, items = build_batch(gpu_lib, insts)
    batch.eval(3)
    torch.cuda.synchronize()
    assert batch.status() == 0
    for i in range(len(insts)):
        assert_same(results(items, i), want[i], f"eager instance {i}")
    for rep in range(2):
        for _, _, c in items:
            for t in (c.tour_s, c.tour_rr, c.plan_s, c.plan_rr):
                t.fill_(-99)
        batch.eval(3, graph=True)
        torch.cuda.synchronize()
        assert batch.status() == 0
        for i in range(len(insts)):
            assert_same(results(items, i), want[i], f"graph replay {rep} instance {i}")
    batch.close()


@pytest.mark.parametrize("shape", [(256, 16, 1), (128, 2, 1), (256, 64, 1), (64, 1, 0), (256, 7, 0)])
def test_batch_launch_shapes_agree(gpu_lib, shape):
    import torch
    insts = [wh_gen.batched_instance(5, i, n_plans=12) for i in range(40)]
    batch, items = build_batch(gpu_lib, insts)
    batch.set_tuning(*shape)
    batch.eval(3)
    torch.cuda.synchronize()
    assert batch.status() == 0
    rng = np.random.default_rng(shape[1])
    for i in rng.choice(len(insts), 6, replace=False):
        assert_same(results(items, i), oracle.eval_plans(insts[i]), f"shape {shape} instance {i}")
    batch.close()


def test_batch_equals_single_calls(gpu_lib):
    """The batch and one wh_eval_plans call per instance give identical results."""
    import torch
    wh = gpu_lib
    insts = [wh_gen.batched_instance(7, i, n_plans=64) for i in range(32)]
    batch, items = build_batch(wh, insts)
    batch.eval(3, graph=True)
    torch.cuda.synchronize()
    assert batch.status() == 0
    for i, inst in enumerate(insts):
        lay = wh.Layout.of(inst.layout)
        prob = items[i][1]
        costs = wh.evaluate(lay, prob)
        torch.cuda.synchronize()
        single = (costs.tour_s[:prob.n_tours].cpu().numpy(), costs.tour_rr[:prob.n_tours].cpu().numpy(),
                  costs.plan_s[:prob.n_plans].cpu().numpy(), costs.plan_rr[:prob.n_plans].cpu().numpy())
        assert_same(results(items, i), single, f"instance {i}")
        lay.close()
    batch.close()


def test_batch_routing_masks(gpu_lib):
    import torch
    insts = [wh_gen.batched_instance(2, i, n_plans=4) for i in range(8)]
    want = [oracle.eval_plans(inst) for inst in insts]
    batch, items = build_batch(gpu_lib, insts)
    batch.eval(1, graph=True)
    torch.cuda.synchronize()
    for i in range(len(insts)):
        got = results(items, i)
        assert np.array_equal(got[0], want[i][0]) and np.array_equal(got[2], want[i][2])
        assert (got[1] == -99).all() and (got[3] == -99).all()
    batch.eval(2)
    torch.cuda.synchronize()
    for i in range(len(insts)):
        got = results(items, i)
        assert np.array_equal(got[1], want[i][1]) and np.array_equal(got[3], want[i][3])
    batch.close()


def test_batch_with_long_tours_and_mixed_layouts(gpu_lib):
    """Instances whose layout needs 32-bit keys and tours beyond 64 lines go
    through the long-tour kernel inside the batch."""
    import torch
    insts = [wh_gen.paperscale(seed=8, n_plans=3), wh_gen.tiny(seed=2, n_plans=5),
             wh_gen.batched_instance(4, 0, n_plans=3)]
    want = [oracle.eval_plans(inst) for inst in insts]
    batch, items = build_batch(gpu_lib, insts)
    batch.eval(3, graph=True)
    torch.cuda.synchronize()
    assert batch.status() == 0
    for i in range(len(insts)):
        assert_same(results(items, i), want[i], f"instance {i}")
    batch.close()


@pytest.mark.parametrize("shape", [(384, 16, 1), (256, 3, 0), (96, 1, 1)])
def test_batch_16bit_order_ids(gpu_lib, shape):
    """Order ids passed only as 16-bit values: the same results as the oracle
    under every routing mask, with and without staged order books, with
    16-bit and 32-bit keys and with tours that go to the long-tour kernel."""
    import torch
    insts = [wh_gen.paperscale(seed=8, n_plans=2), wh_gen.tiny(seed=2, n_plans=5)] + \
            [wh_gen.batched_instance(13, i, n_plans=5) for i in range(10)]
    want = [oracle.eval_plans(inst) for inst in insts]
    batch, items = build_batch(gpu_lib, insts, id16=True)
    if shape[0] > 256:
        shape = (256,) + shape[1:]   # the paper-scale layout needs 32-bit keys: CTAs of at most 256
    batch.set_tuning(*shape)
    for mask in (3, 1, 2):
        for _, _, c in items:
            for t in (c.tour_s, c.tour_rr, c.plan_s, c.plan_rr):
                t.fill_(-99)
        batch.eval(mask, graph=mask == 3)
        torch.cuda.synchronize()
        assert batch.status() == 0
        for i in range(len(insts)):
            got = results(items, i)
            if mask & 1:
                assert np.array_equal(got[0], want[i][0]) and np.array_equal(got[2], want[i][2]), (mask, i)
            if mask & 2:
                assert np.array_equal(got[1], want[i][1]) and np.array_equal(got[3], want[i][3]), (mask, i)
    batch.close()
    # 16-bit keys only (all batched layouts), the 384-thread shape
    b16, items16 = build_batch(gpu_lib, insts[2:], id16=True)
    b16.set_tuning(384, 16, 1)
    b16.eval(3)
    torch.cuda.synchronize()
    assert b16.status() == 0
    for i in range(len(insts) - 2):
        assert_same(results(items16, i), want[i + 2], f"16-bit keys instance {i}")
    b16.close()


def test_batch_16bit_ids_rejections(gpu_lib):
    """16-bit ids on some instances but not all, or on an order book of more
    than 65,536 orders, are WH_EINVAL."""
    import torch
    wh = gpu_lib
    insts = [wh_gen.batched_instance(13, i, n_plans=2) for i in range(2)]
    _, items = build_batch(wh, insts[:1], id16=True)
    _, items32 = build_batch(wh, insts[1:])
    with pytest.raises(wh.WhError) as e:
        wh.Batch(items + items32)
    assert e.value.code == wh.WH_EINVAL
    z = lambda n: torch.zeros(n, dtype=torch.int32, device="cuda")
    one = torch.tensor([0, 1], dtype=torch.int32, device="cuda")
    prob = wh.DeviceProblem(z(65538), z(0), z(1), one, one, None, 1,
                            order_seq16=torch.zeros(1, dtype=torch.int16, device="cuda"))
    costs = wh.alloc_costs(1, 1)
    with pytest.raises(wh.WhError) as e:
        wh.Batch([((8, 20, 3, 1, 2), prob, costs)])
    assert e.value.code == wh.WH_EINVAL


def test_autotune_and_cache(gpu_lib, tmp_path):
    import torch
    insts = [wh_gen.batched_instance(11, i, n_plans=16) for i in range(48)]
    batch, items = build_batch(gpu_lib, insts)
    cache = tmp_path / "tune.json"
    th, ch, hit = batch.autotune(3, str(cache))
    assert hit == 0 and th in (128, 256, 384) and ch >= 1
    entries = json.loads(cache.read_text())
    assert len(entries) == 1 and list(entries.values())[0]["threads"] == th
    assert batch.tuning()[:2] == (th, ch)
    batch.set_tuning(64, 3, 1)
    th2, ch2, hit2 = batch.autotune(3, str(cache))
    assert hit2 == 1 and (th2, ch2) == (th, ch)
    batch.eval(3, graph=True)
    torch.cuda.synchronize()
    assert batch.status() == 0
    for i in (0, 17, 47):
        assert_same(results(items, i), oracle.eval_plans(insts[i]), f"tuned instance {i}")
    batch.close()


def test_batched_full_size_sampled(gpu_lib):
    """1,024 instances x 256 plans in one graph-replayed launch; 12 sampled
    plans from 6 sampled instances re-scored by the oracle, size-independent
    properties on every output of those instances."""
    import torch
    insts = [wh_gen.batched_instance(3, i, n_plans=256) for i in range(1024)]
    batch, items = build_batch(gpu_lib, insts)
    batch.eval(3, graph=True)
    torch.cuda.synchronize()
    assert batch.status() == 0
    rng = np.random.default_rng(1)
    for i in rng.choice(1024, 6, replace=False):
        inst = insts[i]
        ts, tr, ps, pr = results(items, i)
        assert (tr >= 0).all() and (tr <= ts).all() and (tr % 2 == 0).all()
        seg = inst.plan_tour_off
        assert np.array_equal(pr, np.add.reduceat(tr.astype(np.int64), seg[:-1]))
        plans = np.sort(rng.choice(inst.n_plans, 2, replace=False))
        sub = oracle.eval_plans(inst.subset_plans(plans))
        idx = np.concatenate([np.arange(seg[p], seg[p + 1]) for p in plans])
        assert np.array_equal(tr[idx], sub[1]) and np.array_equal(ts[idx], sub[0])
        assert np.array_equal(pr[plans], sub[3]) and np.array_equal(ps[plans], sub[2])
    batch.close()


def test_packed_instances_device_set_and_host_pipeline(gpu_lib):
    """The benchmark's packed layout: all instances' int32 arrays in one flat
    buffer and the order ids as 16-bit values, which the batch reads
    directly.  The
    device set scores every instance exactly as the oracle does; the host
    pipeline (two device sets, copies overlapping evaluation) returns the same
    plan costs on every submitted step; per-kernel timing counts the eager
    launches only."""
    import torch
    wh = gpu_lib
    insts = [wh_gen.batched_instance(9, i, n_plans=5) for i in range(20)]
    want = [oracle.eval_plans(inst) for inst in insts]
    packed = wh.PackedInstances(insts)
    d = packed.device_set()
    d.load()
    d.batch.set_timing(True)
    d.batch.eval(3)
    d.batch.eval(3, graph=True)
    kt = d.batch.timing()
    d.batch.set_timing(False)
    torch.cuda.synchronize()
    assert d.batch.status() == 0
    assert kt["k_eval_batch"][0] == 1 and kt["k_prep_batch"][0] == 1 and kt["k_eval_batch"][1] > 0
    for i, (_, prob, c) in enumerate(d.items):
        got = (c.tour_s[:prob.n_tours].cpu().numpy(), c.tour_rr[:prob.n_tours].cpu().numpy(),
               c.plan_s[:prob.n_plans].cpu().numpy(), c.plan_rr[:prob.n_plans].cpu().numpy())
        assert_same(got, want[i], f"packed instance {i}")
    all_s = np.concatenate([w[2] for w in want])
    all_r = np.concatenate([w[3] for w in want])
    packed.pin()
    pipe = wh.PackedPipeline(packed, 3, tuning=d.batch.tuning())
    tickets = [pipe.submit() for _ in range(3)]
    assert tickets[0][1] == packed.h2d_bytes and tickets[0][2] == 16 * packed.total_plans
    for tk, _, _ in tickets[-2:]:
        out = pipe.wait(tk)
        assert np.array_equal(out[0, :packed.total_plans].numpy(), all_s)
        assert np.array_equal(out[1, :packed.total_plans].numpy(), all_r)
    for s in pipe.sets:
        assert s.batch.status() == 0
    pipe.close()
    d.close()
