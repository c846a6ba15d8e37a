"""Randomised parity: seeded cases over sizes (from 1 row and 4 columns to
several tiles with ragged edges), every parameter of the method (k, the energy
weights, alpha, t_max, the maxval mode, the buffer on or off) and every DP
layout the library can pick (the default for the size, or a tuned layout).
Each GPU carve equals the oracle's byte for byte: frames, buffers and seams."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

LAYOUTS = [None, (32, 4, 4), (16, 4, 4), (16, 4, 2), (16, 8, 2), (0, 4, 4)]


def _cases(n=60, seed=0x5C9F):
    r = np.random.default_rng(seed)
    out = []
    for c in range(n):
        T = int(r.integers(1, 10))
        H = int(r.choice([1, 2, 3, int(r.integers(4, 40)), int(r.integers(40, 90))]))
        W = int(r.choice([4, 5, int(r.integers(6, 64)), int(r.integers(64, 300)), 513]))
        target = int(r.integers(2, W + 1))
        k = int(r.choice([1, 2, int(r.integers(3, 40)), 700]))
        wg, wm = [(1, 0), (1, 2), (2, 1), (0, 3), (3, 5)][int(r.integers(0, 5))]
        alpha = float(r.choice([0.0, 0.15, 0.2, 0.25, 1.0]))
        t_max = int(r.choice([1, 2, 3, 8, 128]))
        use_buffer = bool(r.integers(0, 4) > 0)
        if 255 * (8 * wg + wm) > 4095 and t_max > 64:
            t_max = 64   # keeps t_max * emax^2 below 2^32 (the library's overflow check)
        maxval_mode = int(r.integers(0, 2))
        layout = LAYOUTS[int(r.integers(0, len(LAYOUTS)))]
        rows = int(r.choice([1, 2, 4]))
        out.append((c, T, H, W, target, k, wg, wm, alpha, t_max, use_buffer, maxval_mode,
                    layout, rows, int(r.integers(0, 1 << 30))))
    return out


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1903_03180_gb300 import scpl
    scpl.scpl_tuning_clear()
    yield scpl
    scpl.scpl_tuning_clear()


@pytest.mark.parametrize("case", _cases(240), ids=lambda c: f"case{c[0]}")
def test_random_case_matches_oracle(orc, lib, case):
    from paper_1903_03180_gb300 import synth
    (_, T, H, W, target, k, wg, wm, alpha, t_max, use_buffer, maxval_mode, layout, rows,
     seed) = case
    f = synth.clip(T, H, W, seed=seed, cuts=(2, 4) if T >= 4 else None)
    if layout is not None:
        halo, warps, cols = layout
        lib.scpl_tuning_set(H, W, halo, rows, warps, cols)
    try:
        ref_out, ref_starts, ref_seams = orc.carve(f, target, k, wg=wg, wm=wm, alpha=alpha,
                                                   t_max=t_max, use_buffer=use_buffer,
                                                   maxval_mode=maxval_mode)
        r = lib.Retargeter(alpha=alpha, wg=wg, wm=wm, t_max=t_max, use_buffer=use_buffer,
                           maxval_mode=maxval_mode)
        out, starts, seams = r.carve(torch.from_numpy(f).cuda(), target, k, with_seams=True)
        torch.cuda.synchronize()
        r.close()
    finally:
        lib.scpl_tuning_clear()
    assert np.array_equal(starts, ref_starts)
    if W > target:
        assert np.array_equal(seams.cpu().numpy(), ref_seams)
    assert np.array_equal(out.cpu().numpy(), ref_out)


def _enlarge_cases(n=40, seed=0xE1A5):
    r = np.random.default_rng(seed)
    out = []
    for c in range(n):
        T = int(r.integers(1, 8))
        H = int(r.choice([1, 2, int(r.integers(3, 50))]))
        W = int(r.choice([4, 5, int(r.integers(6, 80)), int(r.integers(80, 300))]))
        target = int(r.integers(W, 2 * W - 1))
        k = int(r.choice([1, 3, int(r.integers(4, 33)), 700]))
        out.append((c, T, H, W, target, k, bool(r.integers(0, 3) > 0),
                    int(r.integers(0, 1 << 30))))
    return out


@pytest.mark.parametrize("case", _enlarge_cases(), ids=lambda c: f"enlarge{c[0]}")
def test_random_enlarge_matches_oracle(orc, lib, case):
    from paper_1903_03180_gb300 import synth
    _, T, H, W, target, k, use_buffer, seed = case
    f = synth.clip(T, H, W, seed=seed, cuts=(2, 3) if T >= 4 else None)
    ref, ref_starts = orc.enlarge(f, target, k, use_buffer=use_buffer)
    r = lib.Retargeter(use_buffer=use_buffer)
    out, starts = r.enlarge(torch.from_numpy(f).cuda(), target, k)
    torch.cuda.synchronize()
    r.close()
    assert np.array_equal(starts, ref_starts)
    assert np.array_equal(out.cpu().numpy(), ref)


def _job_mix(r, n):
    """n small jobs: sizes shared by some (so they group), width, height or both
    reduced, mixed k."""
    sizes = [(int(r.integers(2, 40)), int(r.integers(4, 120))) for _ in range(3)]
    jobs = []
    for j in range(n):
        H, W = sizes[int(r.integers(0, len(sizes)))]
        T = int(r.integers(1, 7))
        tw = int(r.integers(2, W + 1)) if r.integers(0, 3) else W
        th = int(r.integers(2, H + 1)) if r.integers(0, 3) else H
        k = int(r.choice([1, 2, int(r.integers(3, 20))]))
        jobs.append((T, H, W, tw, th, k, int(r.integers(0, 1 << 30))))
    return jobs


@pytest.mark.parametrize("seed", range(6))
def test_random_batch_matches_oracle(orc, lib, seed):
    from paper_1903_03180_gb300 import synth
    r = np.random.default_rng(0xBA7C + seed)
    spec = _job_mix(r, int(r.integers(3, 12)))
    frames = [synth.clip(T, H, W, seed=s, cuts=(2, 3) if T >= 4 else None)
              for (T, H, W, tw, th, k, s) in spec]
    outs = [torch.zeros((T, th, tw, 3), dtype=torch.uint8, device="cuda")
            for (T, H, W, tw, th, k, s) in spec]
    dev = [torch.from_numpy(f).cuda() for f in frames]
    jobs = [lib.make_job(dev[i], tw, th, k, outs[i]) for i, (T, H, W, tw, th, k, s)
            in enumerate(spec)]
    h = lib.scpl_create()
    res = lib.scpl_carve_batch(h, jobs)
    torch.cuda.synchronize()
    lib.scpl_destroy(h)
    for i, (T, H, W, tw, th, k, s) in enumerate(spec):
        ref, _ = orc.carve_job(frames[i], tw, th, k)
        assert res[i][0] == lib.SCPL_OK
        assert np.array_equal(outs[i].cpu().numpy(), ref), (i, spec[i])


@pytest.mark.parametrize("seed", range(4))
def test_random_server_order_and_cancels(orc, lib, seed):
    """Jobs submitted at random points between scheduling rounds, some
    cancelled: every job that completes OK equals the oracle, cancelled ones
    report SCPL_ECANCELED, and nothing stays reserved."""
    from paper_1903_03180_gb300 import synth
    r = np.random.default_rng(0x5E4 + seed)
    spec = _job_mix(r, 10)
    frames = [synth.clip(T, H, W, seed=s) for (T, H, W, tw, th, k, s) in spec]
    outs = [torch.zeros((T, th, tw, 3), dtype=torch.uint8, device="cuda")
            for (T, H, W, tw, th, k, s) in spec]
    dev = [torch.from_numpy(f).cuda() for f in frames]
    srv = lib.Server(hbm_budget=int(r.integers(1, 4)) * 8 * 1024 * 1024)
    tickets, done, cancelled = {}, {}, set()
    for i, (T, H, W, tw, th, k, s) in enumerate(spec):
        tickets[srv.submit(dev[i], tw, th, k, outs[i])] = i
        for _ in range(int(r.integers(0, 3))):
            srv.progress(wait=False)
            for t, st in srv.poll():
                done[tickets[t]] = st
        if r.integers(0, 5) == 0:
            victim = list(tickets)[int(r.integers(0, len(tickets)))]
            try:
                srv.cancel(victim)
                cancelled.add(tickets[victim])
            except lib.SCPLError:
                pass
    while len(done) < len(spec):
        srv.progress(wait=True)
        for t, st in srv.poll():
            done[tickets[t]] = st
    st = srv.stats()
    srv.close()
    assert st["reserved_bytes"] == 0
    torch.cuda.synchronize()
    for i, (T, H, W, tw, th, k, s) in enumerate(spec):
        if done[i] == lib.SCPL_ECANCELED:
            assert i in cancelled
            continue
        assert done[i] in (lib.SCPL_OK, lib.SCPL_ENOMEM), (i, done[i])
        if done[i] == lib.SCPL_OK:
            ref, _ = orc.carve_job(frames[i], tw, th, k)
            assert np.array_equal(outs[i].cpu().numpy(), ref), (i, spec[i])
