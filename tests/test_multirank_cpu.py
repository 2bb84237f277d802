"""Multi-rank path on CPU: instances sharded over world_size-2 gloo ranks
with no data-path collective; every rank fits its shard and the union equals
one single-process run.  (The fits here use the CPU oracle, which is what a
CPU rank can run; on GPUs each rank runs the same shard through lse_fit_batch.)"""
import os

import numpy as np
import pytest

from paper_1705_06073_gb300 import shard, synth


def _instances():
    rs = synth.Stream(4242)
    out = []
    for i in range(7):
        N = 24 + int(rs.uniform(1)[0] * 80)
        out.append(synth.make_instance(N, 2, 20.0, 4300 + i))
    return out


def test_balanced_shards_cover_every_instance_once():
    sizes = [128, 8192, 300, 4096, 4096, 77, 1000, 2048, 129]
    for world in (1, 2, 3, 8):
        sh = shard.balanced_shards(sizes, world)
        flat = sorted(i for s in sh for i in s)
        assert flat == list(range(len(sizes)))
        loads = [sum(shard.fit_cost(sizes[i]) for i in s) for s in sh]
        # LPT bound: no rank exceeds the ideal share by more than the largest job
        assert max(loads) <= sum(loads) / world + max(shard.fit_cost(s) for s in sizes)
    # equal instances split evenly, and one rank takes everything in order
    assert [len(s) for s in shard.balanced_shards([4096] * 128, 4)] == [32] * 4
    assert shard.balanced_shards([4096] * 64, 1) == [list(range(64))]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import fit as ofit
    insts = _instances()
    mine = shard.rank_shard([i.N for i in insts], world, rank)
    res = {i: ofit.fit(insts[i].y, synth.default_grid_size(insts[i].N)).theta.tolist() for i in mine}
    gathered = [None] * world
    dist.all_gather_object(gathered, res)  # result collection for the check only
    if rank == 0:
        merged = {}
        for g in gathered:
            merged.update(g)
        q.put(merged)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_equal_single_process():
    mp = pytest.importorskip("torch.multiprocessing")
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    merged = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from oracle import fit as ofit
    insts = _instances()
    assert sorted(merged) == list(range(len(insts)))
    for i, inst in enumerate(insts):
        ref = ofit.fit(inst.y, synth.default_grid_size(inst.N)).theta
        assert np.array_equal(np.array(merged[i]), ref)
