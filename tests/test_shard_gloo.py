"""The multi-rank split on CPU: two gloo ranks get disjoint plan batches,
generate different plans, and combine time (max) and work (sum) the way the
benchmark does under torchrun."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2110_13693_gb300 import shard


def test_plan_ranges_disjoint_and_covering():
    r = shard.plan_ranges(4, 3, 4096)
    spans = sorted((a, b) for _, _, a, b in r)
    assert spans[0][0] == 0 and all(spans[i][1] == spans[i + 1][0] for i in range(len(spans) - 1))
    assert spans[-1][1] == 4 * 3 * 4096
    with pytest.raises(ValueError):
        shard.plan_base(0, 3, 3, 10)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import numpy as np
    import torch.distributed as dist
    import wh_gen
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    inst = wh_gen.tiny(seed=2, n_plans=8, plan_base=shard.plan_base(rank, 0, 1, 8))
    elapsed = 10.0 + rank          # rank 1 is the slow one
    t, w = shard.combine(elapsed, inst.n_tours)
    out[rank] = (t, w, inst.n_tours, int(np.asarray(inst.order_seq[:50]).sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        (t0, w0, n0, s0), (t1, w1, n1, s1) = out[0], out[1]
    assert t0 == t1 == 11.0                 # max over ranks
    assert w0 == w1 == n0 + n1              # sum over ranks
    assert s0 != s1                         # different plans on each rank


def _exchange_worker(rank, world, port, split, out):
    import numpy as np
    import torch
    import torch.distributed as dist
    import oracle
    import wh_gen
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    inst = wh_gen.tiny(seed=3, n_plans=split[-1])
    lo, hi = split[rank], split[rank + 1]
    # this rank's plans scored by the oracle (test data; the exchange is the
    # code under test)
    _, _, ps, pr = oracle.eval_plans(inst.subset_plans(np.arange(lo, hi)))
    local = torch.from_numpy(np.stack([ps, pr], axis=1).astype(np.int64))
    gathered = shard.gather_plan_costs(local)
    best = shard.best_plan(local[:, 1], lo)
    out[rank] = (gathered.numpy().tolist(), best)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("split", [(0, 5, 8), (0, 0, 6), (0, 7, 7)])
def test_two_gloo_ranks_exchange_plan_costs(split):
    """Plans split unevenly over two ranks (one rank may have none): the
    all-gathered costs equal the unsplit oracle run in plan order, and the
    best-plan reduction returns its minimum optimal cost with the lowest plan
    index among ties."""
    import numpy as np
    import oracle
    import wh_gen
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_exchange_worker, args=(r, 2, port, split, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    _, _, ps, pr = oracle.eval_plans(wh_gen.tiny(seed=3, n_plans=split[-1]))
    want = np.stack([ps, pr], axis=1).tolist()
    k = int(np.argmin(pr))
    for r in range(2):
        assert res[r][0] == want
        assert res[r][1] == (int(pr[k]), k)


def test_best_plan_ties_go_to_the_lowest_index():
    import torch
    c = torch.tensor([7, 3, 5, 3], dtype=torch.int64)
    assert shard.best_plan(c, 10) == (3, 11)
    assert shard.gather_plan_costs(c) is c
