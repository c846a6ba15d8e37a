"""Batching and serving on the GPU (scpl_carve_batch, scpl_server_*): every
clip's result equals the oracle's and scpl_carve's for that clip alone,
bit for bit, whatever else runs beside it."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1903_03180_gb300 import scpl
    return scpl


@pytest.fixture(scope="module")
def synth():
    from paper_1903_03180_gb300 import synth as s
    return s


def _alone(lib, f, tw, th, k):
    """scpl_carve on one clip (width), then on the transposed result (height)."""
    r = lib.Retargeter()
    x = torch.from_numpy(f).cuda()
    T, H, W, _ = f.shape
    starts = None
    if tw < W:
        x, starts, _ = r.carve(x, tw, k)
    if th < H:
        xt = x.transpose(1, 2).contiguous()
        o, s2, _ = r.carve(xt, th, k)
        starts = s2 if starts is None else starts
        x = o.transpose(1, 2).contiguous()
    torch.cuda.synchronize()
    r.close()
    return x.cpu().numpy(), starts


# (T, H, W, target_W, target_H, k, seed): width only, height only, both,
# nothing to do, two clips of one size (one group), ragged sizes
JOBS = [(6, 48, 80, 60, 48, 8, 1), (5, 48, 80, 80, 30, 4, 2), (7, 48, 80, 50, 40, 16, 3),
        (4, 33, 50, 50, 33, 3, 4), (9, 40, 64, 40, 40, 5, 5), (3, 17, 129, 100, 17, 32, 6),
        (8, 64, 36, 36, 20, 2, 7)]


def _frames(synth, T, H, W, seed):
    return synth.clip(T, H, W, seed=seed, cuts=(T // 2, T // 2) if T >= 6 else None)


def test_batch_mixed_jobs_vs_oracle(orc, lib, synth):
    frames = [_frames(synth, T, H, W, s) for (T, H, W, tw, th, k, s) in JOBS]
    outs = [torch.zeros((T, th, tw, 3), dtype=torch.uint8, device="cuda")
            for (T, H, W, tw, th, k, s) in JOBS]
    starts = [np.full(T + 1, -1, np.int32) for (T, *_r) in JOBS]
    dev = [torch.from_numpy(f).cuda() for f in frames]
    jobs = [lib.make_job(dev[i], tw, th, k, outs[i], starts[i])
            for i, (T, H, W, tw, th, k, s) in enumerate(JOBS)]
    h = lib.scpl_create()
    res = lib.scpl_carve_batch(h, jobs)
    torch.cuda.synchronize()
    lib.scpl_destroy(h)
    for i, (T, H, W, tw, th, k, s) in enumerate(JOBS):
        ref, ref_starts = orc.carve_job(frames[i], tw, th, k)
        assert res[i][0] == lib.SCPL_OK
        assert np.array_equal(outs[i].cpu().numpy(), ref), f"job {i}"
        nb = res[i][1]
        if tw < W or th < H:
            assert nb == len(ref_starts) - 1
            assert np.array_equal(starts[i][: nb + 1], ref_starts), f"starts of job {i}"


def test_batch_equals_each_clip_alone(lib, synth):
    """360p-sized clips of two sizes and mixed targets: batch == alone."""
    spec = [(16, 360, 640, 480, 360, 16, 11), (12, 360, 640, 360, 360, 16, 12),
            (10, 240, 426, 320, 240, 16, 13), (14, 240, 426, 426, 183, 16, 14),
            (16, 360, 640, 640, 274, 16, 15)]
    frames = [synth.clip(T, H, W, seed=s, cuts=(T // 2, T // 2)) for (T, H, W, tw, th, k, s) in spec]
    outs = [torch.zeros((T, th, tw, 3), dtype=torch.uint8, device="cuda")
            for (T, H, W, tw, th, k, s) in spec]
    dev = [torch.from_numpy(f).cuda() for f in frames]
    jobs = [lib.make_job(dev[i], tw, th, k, outs[i]) for i, (T, H, W, tw, th, k, s)
            in enumerate(spec)]
    h = lib.scpl_create()
    lib.scpl_carve_batch(h, jobs)
    torch.cuda.synchronize()
    lib.scpl_destroy(h)
    for i, (T, H, W, tw, th, k, s) in enumerate(spec):
        ref, _ = _alone(lib, frames[i], tw, th, k)
        assert np.array_equal(outs[i].cpu().numpy(), ref), f"job {i}"


def test_batch_bad_job_fails_alone(lib, synth):
    f = torch.from_numpy(synth.clip(3, 20, 30, seed=21)).cuda()
    good = torch.zeros((3, 20, 24, 3), dtype=torch.uint8, device="cuda")
    bad = torch.zeros((3, 20, 24, 3), dtype=torch.uint8, device="cuda")
    j_good = lib.make_job(f, 24, 20, 2, good)
    j_bad = lib.make_job(f, 24, 20, 2, bad)
    j_bad.target_W = 31   # wider than the clip
    h = lib.scpl_create()
    with pytest.raises(lib.SCPLError):
        lib.scpl_carve_batch(h, [j_good, j_bad])
    lib.scpl_destroy(h)
    ref, _ = _alone(lib, f.cpu().numpy(), 24, 20, 2)
    assert np.array_equal(good.cpu().numpy(), ref)


def test_server_alone_and_in_the_mix(lib, synth):
    """Jobs arrive while others are on the GPU; a budget of about two jobs
    forces queueing; host and device jobs mixed.  Each result equals the
    clip carved alone."""
    spec = [(8, 96, 160, 120, 96, 8, 31), (6, 96, 160, 160, 60, 8, 32),
            (10, 72, 128, 100, 60, 4, 33), (5, 96, 160, 130, 96, 16, 34),
            (7, 64, 100, 80, 64, 8, 35), (9, 72, 128, 128, 50, 4, 36)]
    frames = [synth.clip(T, H, W, seed=s, cuts=(T // 2, T // 2)) for (T, H, W, tw, th, k, s) in spec]
    srcs, outs = [], []
    for i, ((T, H, W, tw, th, k, s), f) in enumerate(zip(spec, frames)):
        if i % 2:   # host job: page-locked arrays
            srcs.append(torch.from_numpy(f).pin_memory().numpy())
            outs.append(torch.zeros((T, th, tw, 3), dtype=torch.uint8).pin_memory().numpy())
        else:
            srcs.append(torch.from_numpy(f).cuda())
            outs.append(torch.zeros((T, th, tw, 3), dtype=torch.uint8, device="cuda"))
    fp = [lib.scpl_job_footprint(None, lib.make_job(srcs[i], tw, th, k, outs[i]))
          for i, (T, H, W, tw, th, k, s) in enumerate(spec)]
    budget = 2 * max(fp) + 2 * max(fp) // 3
    srv = lib.Server(hbm_budget=budget)
    tickets = {}
    max_active = 0
    for i, (T, H, W, tw, th, k, s) in enumerate(spec):
        tickets[srv.submit(srcs[i], tw, th, k, outs[i])] = i
        a, q = srv.progress(wait=False)
        max_active = max(max_active, a)
    done = {}
    while len(done) < len(spec):
        a, q = srv.progress(wait=True)
        max_active = max(max_active, a)
        for t, st in srv.poll():
            done[tickets[t]] = st
    st = srv.stats()
    srv.close()
    assert all(v == lib.SCPL_OK for v in done.values()), done
    assert st["completed"] == len(spec) and st["failed"] == 0
    assert st["peak_reserved_bytes"] <= budget
    assert max_active >= 2          # jobs overlapped on the device
    torch.cuda.synchronize()
    for i, ((T, H, W, tw, th, k, s), f) in enumerate(zip(spec, frames)):
        ref, _ = _alone(lib, f, tw, th, k)
        got = outs[i].cpu().numpy() if hasattr(outs[i], "cpu") else outs[i]
        assert np.array_equal(got, ref), f"job {i}"


def test_server_budget_of_one_job_serialises(lib, synth):
    f = [synth.clip(4, 50, 70, seed=41 + i) for i in range(3)]
    jobs_out = [torch.zeros((4, 50, 56, 3), dtype=torch.uint8, device="cuda") for _ in f]
    dev = [torch.from_numpy(x).cuda() for x in f]
    fp = lib.scpl_job_footprint(None, lib.make_job(dev[0], 56, 50, 4, jobs_out[0]))
    srv = lib.Server(hbm_budget=fp + fp // 4)
    for d, o in zip(dev, jobs_out):
        srv.submit(d, 56, 50, 4, o)
    max_active = 0
    while True:
        a, q = srv.progress(wait=True)
        max_active = max(max_active, a)
        if a == 0 and q == 0:
            break
    st = srv.stats()
    srv.close()
    assert max_active == 1 and st["completed"] == 3
    for x, o in zip(f, jobs_out):
        ref, _ = _alone(lib, x, 56, 50, 4)
        assert np.array_equal(o.cpu().numpy(), ref)


def test_server_graphs_and_launch_accounting(lib, synth):
    f = torch.from_numpy(synth.clip(6, 40, 90, seed=51)).cuda()
    o = torch.zeros((6, 40, 60, 3), dtype=torch.uint8, device="cuda")
    srv = lib.Server()
    srv.submit(f, 60, 40, 4, o)
    srv.drain()
    st = srv.stats()
    srv.close()
    assert st["scan_waves"] == 1 and st["groups"] == 1
    assert st["graphs_built"] >= 1 and st["chunks"] >= 1
    assert st["kernel_launches"] >= 2 * st["chunks"] + 3
