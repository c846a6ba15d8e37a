"""Failure detection and fault containment on the GPU, with no GPU fault.

- A device-wide wait that runs out: the buffer scan of arriving frames waits
  (bounded) on a counter that nothing raises, returns SCPL_ETIMEOUT, and the
  handle then scans correctly.
- Streaming ingest: frames copied in by a producer on another stream while
  the scan runs give the same buffers as the complete clip.
- Serving faults injected on the host: cancelled jobs (queued and admitted)
  and allocator refusals at every allocation of a run.  Every other job's
  result stays bit-identical to the clip carved alone, the memory accounting
  returns to zero and the server stays usable.
"""
from __future__ import annotations

import time

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
    if tw < W:
        x, _, _ = r.carve(x, tw, k)
    if th < H:
        o, _, _ = r.carve(x.transpose(1, 2).contiguous(), th, k)
        x = o.transpose(1, 2).contiguous()
    torch.cuda.synchronize()
    r.close()
    return x.cpu().numpy()


# ---- bounded device-wide waits ---------------------------------------------------
def test_arrival_wait_times_out_and_handle_stays_usable(lib, synth):
    f = torch.from_numpy(synth.clip(24, 64, 96, seed=61, cuts=(12, 12))).cuda()
    h = lib.scpl_create()
    ref = lib.scpl_scan(h, f)
    lib.scpl_set_wait_limit(h, 50_000_000)   # 50 ms
    counter = torch.zeros(1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    for raised in (0, 1, 2):   # nothing, the first chunk, the first two of three
        counter.fill_(raised)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with pytest.raises(lib.SCPLError) as ei:
            lib.scpl_scan_arrivals(h, f, counter, 8)
        assert ei.value.status == lib.SCPL_ETIMEOUT
        assert time.perf_counter() - t0 < 10.0
        assert "exceeded" in lib.scpl_last_error(h)
    # the same handle: a complete counter and a plain scan both give the buffers
    counter.fill_(3)
    torch.cuda.synchronize()
    assert np.array_equal(lib.scpl_scan_arrivals(h, f, counter, 8), ref)
    lib.scpl_set_wait_limit(h, 2_000_000_000)
    assert np.array_equal(lib.scpl_scan(h, f), ref)
    with pytest.raises(lib.SCPLError):
        lib.scpl_set_wait_limit(h, 10)
    lib.scpl_destroy(h)


def test_arrivals_from_a_producer_stream(lib, synth):
    """Frames copied chunk by chunk on another stream, each chunk announced by
    a stream memory operation, while the scan consumes them."""
    T, H, W = 70, 540, 960
    host = torch.from_numpy(synth.clip(T, H, W, seed=62, cuts=(20, 45))).pin_memory()
    full = host.cuda()
    h = lib.scpl_create()
    ref = lib.scpl_scan(h, full)
    for chunk in (1, 8, 16):
        dev = torch.empty_like(full)
        counter = torch.zeros(1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        side = torch.cuda.Stream()
        with torch.cuda.stream(side):
            for c in range((T + chunk - 1) // chunk):
                a, b = c * chunk, min(T, (c + 1) * chunk)
                dev[a:b].copy_(host[a:b], non_blocking=True)
                lib.scpl_signal_arrival(side, counter, c + 1)
        got = lib.scpl_scan_arrivals(h, dev, counter, chunk)
        torch.cuda.synchronize()
        assert np.array_equal(got, ref), chunk
    lib.scpl_destroy(h)


# ---- serving faults injected on the host -----------------------------------------
SPEC = [(6, 48, 80, 60, 48, 8, 71), (5, 48, 80, 64, 36, 4, 72), (7, 40, 64, 50, 40, 16, 73)]


def _jobs(lib, synth, host_mask=(False, True, False)):
    frames = [synth.clip(T, H, W, seed=s, cuts=(T // 2, T // 2)) for (T, H, W, tw, th, k, s) in SPEC]
    srcs, outs = [], []
    for on_host, (T, H, W, tw, th, k, s), f in zip(host_mask, SPEC, frames):
        if on_host:
            srcs.append(torch.from_numpy(f).pin_memory().numpy())
            outs.append(torch.zeros((T, th, tw, 3), dtype=torch.uint8).pin_memory().numpy())
        else:
            srcs.append(torch.from_numpy(f).cuda())
            outs.append(torch.zeros((T, th, tw, 3), dtype=torch.uint8, device="cuda"))
    return frames, srcs, outs


def _np(x):
    return x.cpu().numpy() if hasattr(x, "cpu") else x


@pytest.fixture(scope="module")
def refs(lib, synth):
    frames = [synth.clip(T, H, W, seed=s, cuts=(T // 2, T // 2)) for (T, H, W, tw, th, k, s) in SPEC]
    return [_alone(lib, f, tw, th, k) for f, (T, H, W, tw, th, k, s) in zip(frames, SPEC)]


def _run(srv, submitted, max_rounds=100000):
    done = {}
    for _ in range(max_rounds):
        srv.progress(wait=True)
        for t, st in srv.poll():
            done[t] = st
        if len(done) == len(submitted):
            return done
    raise AssertionError("the server did not finish")


def test_cancel_queued_job(lib, synth, refs):
    frames, srcs, outs = _jobs(lib, synth)
    fp = max(lib.scpl_job_footprint(None, lib.make_job(srcs[i], tw, th, k, outs[i]))
             for i, (T, H, W, tw, th, k, s) in enumerate(SPEC))
    srv = lib.Server(hbm_budget=fp + fp // 4)   # one job at a time
    tk = [srv.submit(srcs[i], tw, th, k, outs[i]) for i, (T, H, W, tw, th, k, s) in enumerate(SPEC)]
    srv.progress(wait=False)
    srv.cancel(tk[2])   # still queued behind the first
    done = _run(srv, tk)
    st = srv.stats()
    with pytest.raises(lib.SCPLError):
        srv.cancel(tk[0])       # already completed
    with pytest.raises(lib.SCPLError):
        srv.cancel(10 ** 9)     # unknown
    srv.close()
    assert done[tk[2]] == lib.SCPL_ECANCELED
    assert done[tk[0]] == lib.SCPL_OK and done[tk[1]] == lib.SCPL_OK
    assert st["cancelled"] == 1 and st["completed"] == 2 and st["failed"] == 0
    assert st["reserved_bytes"] == 0
    torch.cuda.synchronize()
    for i in (0, 1):
        assert np.array_equal(_np(outs[i]), refs[i]), i


@pytest.mark.parametrize("rounds", [0, 1, 2, 3, 5, 8, 13])
def test_cancel_admitted_job_at_any_stage(lib, synth, refs, rounds):
    """Cancel job 1 (host frames, two passes) after `rounds` scheduling rounds:
    it ends cancelled or, if it had already finished, OK and exact; the jobs
    beside it are exact; the server then carves a new job."""
    frames, srcs, outs = _jobs(lib, synth)
    srv = lib.Server()
    tk = [srv.submit(srcs[i], tw, th, k, outs[i]) for i, (T, H, W, tw, th, k, s) in enumerate(SPEC)]
    done = {}
    for _ in range(rounds):
        srv.progress(wait=False)
        for t, st in srv.poll():
            done[t] = st
    try:
        srv.cancel(tk[1])
        cancelled = True
    except lib.SCPLError:
        cancelled = False
    for t, st in _run(srv, [t for t in tk if t not in done]).items():
        done[t] = st
    st = srv.stats()
    assert st["reserved_bytes"] == 0
    torch.cuda.synchronize()
    for i in (0, 2):
        assert done[tk[i]] == lib.SCPL_OK
        assert np.array_equal(_np(outs[i]), refs[i]), i
    if cancelled:
        assert done[tk[1]] in (lib.SCPL_ECANCELED, lib.SCPL_OK)
    if done[tk[1]] == lib.SCPL_OK:
        assert np.array_equal(_np(outs[1]), refs[1])
    # still usable
    T, H, W, tw, th, k, s = SPEC[0]
    o = torch.zeros((T, th, tw, 3), dtype=torch.uint8, device="cuda")
    t = srv.submit(torch.from_numpy(frames[0]).cuda(), tw, th, k, o)
    assert _run(srv, [t])[t] == lib.SCPL_OK
    srv.close()
    assert np.array_equal(o.cpu().numpy(), refs[0])


def test_allocator_refusal_at_every_allocation(lib, synth, refs):
    """Refuse the n-th device allocation of a run, for every n: each job ends
    OK (exact) or SCPL_ENOMEM, nothing leaks, and the server stays usable."""
    srv = lib.Server()
    n_enomem = 0
    for skip in range(40):
        frames, srcs, outs = _jobs(lib, synth)
        srv.refuse_allocations(skip, 1)
        tk = [srv.submit(srcs[i], tw, th, k, outs[i])
              for i, (T, H, W, tw, th, k, s) in enumerate(SPEC)]
        done = _run(srv, tk)
        st = srv.stats()
        assert st["reserved_bytes"] == 0, skip
        torch.cuda.synchronize()
        for i, t in enumerate(tk):
            assert done[t] in (lib.SCPL_OK, lib.SCPL_ENOMEM), (skip, i, done[t])
            if done[t] == lib.SCPL_OK:
                assert np.array_equal(_np(outs[i]), refs[i]), (skip, i)
            else:
                n_enomem += 1
    srv.refuse_allocations(0, 0)
    srv.close()
    assert n_enomem >= 1   # a refusal with nothing else running fails its job


def test_allocator_refusing_everything_fails_jobs_alone(lib, synth, refs):
    frames, srcs, outs = _jobs(lib, synth)
    srv = lib.Server()
    srv.refuse_allocations(0, 1000)
    tk = [srv.submit(srcs[i], tw, th, k, outs[i]) for i, (T, H, W, tw, th, k, s) in enumerate(SPEC)]
    done = _run(srv, tk)
    assert all(done[t] == lib.SCPL_ENOMEM for t in tk), done
    assert srv.stats()["reserved_bytes"] == 0
    srv.refuse_allocations(0, 0)
    tk = [srv.submit(srcs[i], tw, th, k, outs[i]) for i, (T, H, W, tw, th, k, s) in enumerate(SPEC)]
    done = _run(srv, tk)
    srv.close()
    torch.cuda.synchronize()
    for i, t in enumerate(tk):
        assert done[t] == lib.SCPL_OK
        assert np.array_equal(_np(outs[i]), refs[i]), i


def test_job_larger_than_the_budget_fails_alone(lib, synth, refs):
    frames, srcs, outs = _jobs(lib, synth)
    fp = [lib.scpl_job_footprint(None, lib.make_job(srcs[i], tw, th, k, outs[i]))
          for i, (T, H, W, tw, th, k, s) in enumerate(SPEC)]
    big = torch.zeros((4, 720, 1280, 3), dtype=torch.uint8, device="cuda")
    big_out = torch.zeros((4, 720, 1000, 3), dtype=torch.uint8, device="cuda")
    srv = lib.Server(hbm_budget=2 * max(fp))
    tk = [srv.submit(big, 1000, 720, 8, big_out)]
    tk += [srv.submit(srcs[i], tw, th, k, outs[i]) for i, (T, H, W, tw, th, k, s) in enumerate(SPEC)]
    done = _run(srv, tk)
    srv.close()
    assert done[tk[0]] == lib.SCPL_ENOMEM
    torch.cuda.synchronize()
    for i, t in enumerate(tk[1:]):
        assert done[t] == lib.SCPL_OK
        assert np.array_equal(_np(outs[i]), refs[i]), i
