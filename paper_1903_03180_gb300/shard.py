"""Data-parallel sharding of retarget work over GPUs (one process per GPU).

Two units split across ranks.
- Clips (jobs) are independent, so they split with no exchange on the data
  path: each rank carves its own share with its own handle or server.
- Within one clip, the spatiotemporal buffers are independent once the scan
  has fixed them (Sec. 3.2: the seams of a buffer come from its own frames
  and are removed from every frame of it).  The scan itself runs frame after
  frame, so it stays on the rank that holds the clip; its buffers are then
  dealt to the ranks, each carves its own (scpl_carve_buffer on a GPU), and
  the carved frames come back to the owner.  The one exchange is the frames
  out and the carved frames back, point to point.

Every partition is a pure function of the costs and the world size, so every
rank computes the same one without communicating.  Longest processing time
first: units sorted by estimated cost (ties by index) go one by one to the
least-loaded rank (ties to the lowest rank).
"""
from __future__ import annotations


def job_cost(T: int, H: int, W: int, target_W: int, target_H: int, k: int) -> float:
    """Estimated work of a job.  Each pass scans T*H*W pixels once and then
    runs about ceil(removed / k) iterations over T*H*W-sized buffers."""
    cost = 0.0
    Wc = W
    if target_W < W:
        cost += T * H * W * (1.0 + (W - target_W) / max(k, 1))
        Wc = target_W
    if target_H < H:
        cost += T * H * Wc * (1.0 + (H - target_H) / max(k, 1))
    return cost


def partition(costs: list[float], world: int) -> list[int]:
    """Rank of every job (a list as long as costs)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    owner = [0] * len(costs)
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += costs[i]
    return owner


def my_jobs(specs: list[dict], rank: int, world: int) -> list[int]:
    """Indices of the jobs this rank carves.  specs are dicts with T, H, W,
    target_W, target_H and k."""
    costs = [job_cost(s["T"], s["H"], s["W"], s["target_W"], s["target_H"], s["k"])
             for s in specs]
    owner = partition(costs, world)
    return [i for i, o in enumerate(owner) if o == rank]


def buffer_cost(nt: int, H: int, W: int, target_W: int, k: int) -> float:
    """Estimated work of carving one buffer of nt frames: about
    ceil(removed / k) iterations over nt frames of H x W pixels."""
    return nt * H * W * (1.0 + (W - target_W) / max(k, 1))


def deal_buffers(starts: list[int], H: int, W: int, target_W: int, k: int,
                 world: int) -> list[int]:
    """Rank of every buffer of a clip whose scan gave `starts`."""
    costs = [buffer_cost(starts[b + 1] - starts[b], H, W, target_W, k)
             for b in range(len(starts) - 1)]
    return partition(costs, world)


def carve_clip_by_buffers(frames, target_W: int, k: int, scan, carve_buffer, group=None,
                          owner: int = 0, device=None):
    """Carve one clip with its buffers spread over the ranks of `group`.

    frames: on the owner rank the clip, a uint8 tensor [T,H,W,3] (on the
    device the backend sends from: CPU for gloo, the rank's GPU for NCCL);
    ignored elsewhere.  scan(frames) -> buffer starts (owner only).
    carve_buffer(frames_b, prev_frame, target_W, k) -> uint8 tensor
    [T_b,H,target_W,3]: carves the frames of one buffer as one fixed buffer,
    prev_frame [H,W,3] being the clip's frame just before them (None for the
    first buffer).  device: where a non-owner rank receives (CPU by default).

    Returns (out, starts, mine): on the owner the carved clip
    [T,H,target_W,3], elsewhere None; the starts; the buffers this rank
    carved."""
    import torch
    import torch.distributed as dist
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    meta = [None]
    if rank == owner:
        T, H, W, _ = frames.shape
        meta = [(int(T), int(H), int(W), [int(x) for x in scan(frames)])]
    dist.broadcast_object_list(meta, src=owner, group=group)
    T, H, W, starts = meta[0]
    nb = len(starts) - 1
    owners = deal_buffers(starts, H, W, target_W, k, world)
    mine = [b for b in range(nb) if owners[b] == rank]
    dev = frames.device if rank == owner else (device or torch.device("cpu"))

    def peer(r):   # a rank of `group` as the global rank send/recv address
        return r if group is None else dist.get_global_rank(group, r)

    # the frames out: each remote buffer with the frame before it
    got = {}
    if rank == owner:
        for b in range(nb):
            if owners[b] != owner:
                lo = max(starts[b] - 1, 0)
                dist.send(frames[lo:starts[b + 1]].contiguous(), dst=peer(owners[b]),
                          group=group)
    else:
        for b in mine:
            lo = max(starts[b] - 1, 0)
            buf = torch.empty((starts[b + 1] - lo, H, W, 3), dtype=torch.uint8, device=dev)
            dist.recv(buf, src=peer(owner), group=group)
            got[b] = buf
    # every rank carves its own buffers
    done = {}
    for b in mine:
        t0, t1 = starts[b], starts[b + 1]
        if rank == owner:
            fb, prev = frames[t0:t1], (frames[t0 - 1] if t0 > 0 else None)
        else:
            buf = got.pop(b)
            fb, prev = (buf[1:], buf[0]) if t0 > 0 else (buf, None)
        done[b] = carve_buffer(fb.contiguous(), None if prev is None else prev.contiguous(),
                               target_W, k)
    # the carved frames back to the owner
    if rank != owner:
        for b in mine:
            dist.send(done.pop(b).contiguous(), dst=peer(owner), group=group)
        return None, starts, mine
    out = torch.empty((T, H, target_W, 3), dtype=torch.uint8, device=dev)
    for b in range(nb):
        t0, t1 = starts[b], starts[b + 1]
        if owners[b] == owner:
            out[t0:t1] = done.pop(b)
        else:
            recv = torch.empty((t1 - t0, H, target_W, 3), dtype=torch.uint8, device=dev)
            dist.recv(recv, src=peer(owners[b]), group=group)
            out[t0:t1] = recv
    return out, starts, mine
