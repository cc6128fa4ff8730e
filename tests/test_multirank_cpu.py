"""The N-GPU bench path on CPU ranks (gloo, world size 2): every rank builds its own
independent instances (weak scaling, no data-path collective) and the timing is the
maximum over ranks; the reported value is the units of all ranks over that time."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    insts = bench.make_instances("batch256", rank)
    units = sum(bench.units_per_step(sh, w, lev) for sh, w, lev, _ in insts)
    fake_time = torch.tensor([1.0 + rank], dtype=torch.float64)      # the slower rank decides
    dist.all_reduce(fake_time, op=dist.ReduceOp.MAX)
    u = torch.tensor([units], dtype=torch.float64)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    checksum = float(sum(float(t.sum()) for _, _, _, t in insts[:4]))
    q.put((rank, units, float(fake_time), float(u), checksum))
    dist.destroy_process_group()


def test_two_cpu_ranks_shard_instances_and_take_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, u0, t0, usum0, c0), (r1, u1, t1, usum1, c1) = out
    assert t0 == t1 == 2.0                      # max over ranks
    assert usum0 == usum1 == u0 + u1            # whole-job units
    assert c0 != c1                             # independent instances per rank
