"""Data-parallel sharding on CPU ranks (gloo, world size 2): every job is
carved exactly once, the load is balanced, and the gathered results equal a
single process carving everything (the oracle stands in for each rank's GPU)."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1903_03180_gb300 import shard, synth


def _specs():
    sp = synth.batch_spec(n_clips=9, T=3)
    for s in sp:   # tiny sizes so that the oracle carves them in a blink
        s["H"], s["W"] = s["H"] // 20, s["W"] // 20
        if s["aspect"] == "21:9":
            s["target_W"], s["target_H"] = s["W"], int(round(s["W"] * 9 / 21))
        else:
            num, den = (1, 1) if s["aspect"] == "1:1" else (4, 3)
            s["target_W"], s["target_H"] = min(s["W"], int(round(s["H"] * num / den))), s["H"]
        s["k"] = 4
    return sp


def _carve(s):
    import oracle
    f = synth.clip(s["T"], s["H"], s["W"], seed=s["seed"])
    out, _ = oracle.carve_job(f, s["target_W"], s["target_H"], s["k"])
    return out


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    specs = _specs()
    mine = shard.my_jobs(specs, rank, world)
    res = {i: _carve(specs[i]) for i in mine}
    gathered = [None] * world
    dist.all_gather_object(gathered, (rank, mine, res))
    if rank == 0:
        q.put(gathered)
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_is_lpt_and_deterministic():
    costs = [5.0, 3.0, 3.0, 2.0, 2.0, 1.0]
    assert shard.partition(costs, 2) == [0, 1, 1, 0, 1, 0]   # loads 8 and 8
    assert shard.partition(costs, 1) == [0] * 6
    owner = shard.partition(costs, 4)
    load = [sum(c for c, o in zip(costs, owner) if o == r) for r in range(4)]
    assert max(load) - min(load) <= max(costs)


def test_two_gloo_ranks_carve_every_job_once():
    import oracle
    oracle.build()
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    specs = _specs()
    seen = sorted(i for _, mine, _ in gathered for i in mine)
    assert seen == list(range(len(specs)))
    costs = [shard.job_cost(s["T"], s["H"], s["W"], s["target_W"], s["target_H"], s["k"])
             for s in specs]
    load = [sum(costs[i] for i in mine) for _, mine, _ in gathered]
    assert max(load) - min(load) <= max(costs)
    for _, mine, res in gathered:
        for i in mine:
            assert np.array_equal(res[i], _carve(specs[i]))


# ------------------------------------------- one clip, buffers over ranks
def _buffer_clip():
    return synth.clip(44, 30, 64, seed=4242, cuts=(6, 11))


def _oracle_scan(fr):
    import oracle
    return oracle.scan(oracle.energy(fr.numpy()))


def _oracle_carve_buffer(fb, prev, target, k):
    """One fixed buffer by the oracle; its first frame's motion is taken
    against the clip's frame before it (D = 0 only at the clip's start)."""
    import oracle
    f = fb.numpy()
    if prev is None:
        D = oracle.motion(f)
    else:
        D = oracle.motion(np.concatenate([prev.numpy()[None], f]))[1:]
    out, _, _ = oracle.carve_buffer(f, D, target, k)
    return torch.from_numpy(out)


def _buffer_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    frames = torch.from_numpy(_buffer_clip()) if rank == 0 else None
    out, starts, mine = shard.carve_clip_by_buffers(frames, 48, 4, _oracle_scan,
                                                    _oracle_carve_buffer)
    gathered = [None] * world
    dist.all_gather_object(gathered, (rank, mine))
    if rank == 0:
        q.put((out.numpy(), starts, gathered))
    dist.barrier()
    dist.destroy_process_group()


def test_deal_buffers_is_lpt():
    starts = [0, 10, 30, 31, 60, 64]
    owner = shard.deal_buffers(starts, 8, 16, 12, 2, 2)
    assert owner == shard.deal_buffers(starts, 8, 16, 12, 2, 2)   # deterministic
    cost = [b1 - b0 for b0, b1 in zip(starts, starts[1:])]
    load = [sum(c for c, o in zip(cost, owner) if o == r) for r in range(2)]
    assert max(load) - min(load) <= max(cost)
    assert shard.deal_buffers(starts, 8, 16, 12, 2, 1) == [0] * 5


def test_two_gloo_ranks_share_one_clips_buffers():
    """Rank 0 scans the clip, the buffers are dealt to both ranks, each
    carves its own as a fixed buffer, and the carved frames come back: the
    clip equals the oracle carving it whole."""
    import oracle
    oracle.build()
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_buffer_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out, starts, gathered = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    f = _buffer_clip()
    ref_out, ref_starts, _ = oracle.carve(f, 48, 4)
    assert list(starts) == list(ref_starts) and len(starts) >= 4
    carved = sorted(b for _, mine in gathered for b in mine)
    assert carved == list(range(len(starts) - 1))
    assert all(len(mine) >= 1 for _, mine in gathered)   # both ranks took buffers
    assert np.array_equal(out, ref_out)
