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
