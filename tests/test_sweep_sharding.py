"""Host logic of multi-rank sweeps, on CPU: sharding covers every instance
once with balanced cost, and results gathered over 2 gloo ranks come back in
instance order."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1204_4098_gb300 import inputs, sweep


def test_shard_partitions_and_balances():
    inst = inputs.sweep_instances(512, seed=4)
    for world in (1, 2, 3, 8):
        parts = [sweep.shard(inst, world, r) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(inst)))
        loads = [sum(inst[i]["nx"] * inst[i]["ny"] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(d["nx"] * d["ny"] for d in inst)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    inst = inputs.sweep_instances(n, seed=9)
    mine = sweep.shard(inst, world, rank)
    local = [dict(rank=rank, cells=inst[i]["nx"] * inst[i]["ny"]) for i in mine]
    allres = sweep.gather_results(mine, local, n, world)
    if rank == 0:
        q.put(allres)
    dist.destroy_process_group()


def test_gather_over_two_gloo_ranks():
    n, world = 37, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    inst = inputs.sweep_instances(n, seed=9)
    assert all(r is not None for r in res)
    assert [r["cells"] for r in res] == [d["nx"] * d["ny"] for d in inst]
    assert {r["rank"] for r in res} == {0, 1}
    for i, r in enumerate(res):
        assert i in sweep.shard(inst, world, r["rank"])
