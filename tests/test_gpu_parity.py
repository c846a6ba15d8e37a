"""GPU parity: the CUDA library, called through its C ABI, against the CPU
oracle on the same seeded inputs.  Every output of the method is integer
(energies, buffer boundaries, seam columns, carved bytes), so the bar is
equality (tolerance 0)."""
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


def _carve_gpu(lib, frames, target, k, **params):
    r = lib.Retargeter(**params)
    out, starts, seams = r.carve(torch.from_numpy(frames).cuda(), target, k, with_seams=True)
    torch.cuda.synchronize()
    res = out.cpu().numpy(), starts, seams.cpu().numpy()
    r.close()
    return res


def _carve_both(orc, lib, frames, target, k, wg=1, wm=2, t_max=128, use_buffer=True,
                maxval_mode=0, alpha=0.2):
    ref = orc.carve(frames, target, k, wg=wg, wm=wm, alpha=alpha, t_max=t_max,
                    use_buffer=use_buffer, maxval_mode=maxval_mode)
    got = _carve_gpu(lib, frames, target, k, alpha=alpha, wg=wg, wm=wm, t_max=t_max,
                     use_buffer=use_buffer, maxval_mode=maxval_mode)
    return ref, got


def _assert_same(ref, got):
    ref_out, ref_starts, ref_seams = ref
    out, starts, seams = got
    assert np.array_equal(starts, ref_starts), (starts, ref_starts)
    assert seams.shape == ref_seams.shape
    for b in range(len(starts) - 1):
        assert np.array_equal(seams[b], ref_seams[b]), f"seams of buffer {b} differ"
    assert np.array_equal(out, ref_out)


# ------------------------------------------------------------------ energy
@pytest.mark.parametrize("T,H,W", [(1, 1, 1), (2, 1, 7), (3, 5, 1), (3, 17, 33), (4, 40, 130)])
def test_energy_random(orc, lib, T, H, W):
    r = np.random.default_rng(T * 1000 + H * 10 + W)
    f = r.integers(0, 256, (T, H, W, 3), dtype=np.uint8)
    for wg, wm in [(1, 0), (1, 2), (3, 5)]:
        h = lib.scpl_create(lib.Params(0.2, wg, wm, 128, 1, 0))
        e = torch.empty((T, H, W), dtype=torch.int32, device="cuda")
        lib.scpl_energy(h, torch.from_numpy(f).cuda(), e)
        torch.cuda.synchronize()
        lib.scpl_destroy(h)
        assert np.array_equal(e.cpu().numpy(), orc.energy(f, wg, wm))


def test_energy_clip(orc, lib, synth):
    f = synth.clip(5, 360, 640, seed=21)
    h = lib.scpl_create()
    e = torch.empty(f.shape[:3], dtype=torch.int32, device="cuda")
    lib.scpl_energy(h, torch.from_numpy(f).cuda(), e)
    torch.cuda.synchronize()
    lib.scpl_destroy(h)
    assert np.array_equal(e.cpu().numpy(), orc.energy(f))


# --------------------------------------------------------------------- scan
@pytest.mark.parametrize("T,H,W,seed,t_max", [(1, 8, 8, 1, 128), (10, 9, 70, 2, 4),
                                              (64, 360, 640, 0x5C9 ^ 2, 128),
                                              (40, 61, 97, 3, 16), (30, 24, 40, 4, 1)])
def test_scan(orc, lib, synth, T, H, W, seed, t_max):
    f = synth.clip(T, H, W, seed=seed, cuts=(5, 12) if T >= 30 else None)
    h = lib.scpl_create(lib.Params(0.2, 1, 2, t_max, 1, 0))
    starts = lib.scpl_scan(h, torch.from_numpy(f).cuda())
    lib.scpl_destroy(h)
    assert np.array_equal(starts, orc.scan(orc.energy(f), t_max=t_max))


def test_scan_maxval_theoretical(orc, lib, synth):
    f = synth.clip(20, 32, 48, seed=5, cuts=(4, 9))
    h = lib.scpl_create(lib.Params(0.05, 1, 2, 128, 1, 1))
    starts = lib.scpl_scan(h, torch.from_numpy(f).cuda())
    lib.scpl_destroy(h)
    assert np.array_equal(starts, orc.scan(orc.energy(f), alpha=0.05, maxval_mode=1,
                                           maxval_theory=255 * 10))


# ------------------------------------------------------- one SCPL iteration
@pytest.mark.parametrize("H,W,vmax,k", [(1, 1, 5, 1), (1, 9, 3, 4), (2, 2, 0, 2), (7, 3, 2, 3),
                                        (33, 31, 4, 8), (50, 1025, 9, 16), (64, 2049, 1, 32),
                                        (20, 700, 0, 700), (300, 1920, 2550, 32),
                                        (70, 5000, 40, 24), (40, 7000, 9, 16)])
def test_seams(orc, lib, H, W, vmax, k):
    r = np.random.default_rng(H * 7 + W)
    E = r.integers(0, vmax + 1, (H, W)).astype(np.int32)
    CE, L, d = orc.dp(E)
    ref_cols = orc.select(CE[-1], L[-1], k)
    h = lib.scpl_create()
    cols = torch.full((k, H), -1, dtype=torch.int16, device="cuda")
    ke = lib.scpl_seams(h, torch.from_numpy(E).cuda(), k, cols)
    lib.scpl_destroy(h)
    assert ke == len(ref_cols)
    got = cols.cpu().numpy()
    for s, c in enumerate(ref_cols):
        assert np.array_equal(got[s], orc.backtrack(d, int(c))), f"seam {s}"


# -------------------------------------------------------------------- carve
def test_carve_still_320x240(orc, lib, synth):
    """Single 320x240 frame, gradient energy only, 32 seams with k = 8."""
    f = synth.workload_still_320x240()
    ref, got = _carve_both(orc, lib, f, 288, 8, wg=1, wm=0, use_buffer=False)
    _assert_same(ref, got)


@pytest.mark.parametrize("T,H,W,target,k,t_max,seed", [
    (1, 1, 3, 2, 1, 128, 1),       # one row, narrowest
    (1, 5, 9, 9, 4, 128, 2),       # nothing to remove
    (2, 7, 40, 20, 64, 128, 3),    # k larger than the parents
    (6, 48, 80, 64, 4, 4, 4),      # several buffers
    (9, 33, 129, 100, 1, 3, 5),    # k = 1, ragged width
    (12, 70, 300, 210, 16, 128, 6),
    (5, 1, 600, 300, 32, 2, 7),    # H = 1: every column its own parent
])
def test_carve_small(orc, lib, synth, T, H, W, target, k, t_max, seed):
    f = synth.clip(T, H, W, seed=seed)
    ref, got = _carve_both(orc, lib, f, target, k, t_max=t_max)
    _assert_same(ref, got)


def test_carve_flat_frames_ties(orc, lib):
    """All-equal energy: every DP choice is a tie (lowest column wins)."""
    f = np.full((3, 20, 50, 3), 128, np.uint8)
    ref, got = _carve_both(orc, lib, f, 30, 8)
    _assert_same(ref, got)


def test_carve_raw_classic_per_frame(orc, lib, synth):
    f = synth.clip(4, 40, 64, seed=8)
    ref, got = _carve_both(orc, lib, f, 50, 1, use_buffer=False)
    _assert_same(ref, got)


def test_carve_clip_640x360(orc, lib, synth):
    """64-frame 640x360 clip, motion energy, buffer on, 160 seams, k = 16."""
    f = synth.workload_clip_640x360()
    ref, got = _carve_both(orc, lib, f, 480, 16)
    _assert_same(ref, got)


def test_carve_host_matches_device(orc, lib, synth):
    f = synth.clip(7, 50, 90, seed=9)
    out_d, starts_d, seams_d = _carve_gpu(lib, f, 70, 5)
    h = lib.scpl_create()
    out_h = np.empty((7, 50, 70, 3), np.uint8)
    seams_h = np.empty((7, 20, 50), np.int16)
    starts_h = lib.scpl_carve_host(h, f, 70, 5, out_h, seams_h)
    lib.scpl_destroy(h)
    assert np.array_equal(starts_h, starts_d)
    assert np.array_equal(out_h, out_d)
    assert np.array_equal(seams_h[: len(starts_h) - 1], seams_d)


def test_repeat_calls_identical(lib, synth):
    f = torch.from_numpy(synth.clip(10, 64, 100, seed=10)).cuda()
    r = lib.Retargeter()
    a = r.carve(f, 80, 8, with_seams=True)
    b = r.carve(f, 80, 8, with_seams=True)
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[2], b[2])
    assert np.array_equal(a[1], b[1])
    r.close()


def test_device_loop_follows_changing_calls(lib, synth):
    """One handle carves a sequence of clips whose size, k and seam output
    change from call to call, then repeats the first: the graph that loops
    over the iterations on the device is rebuilt whenever the workspace or
    the arguments change, and every result equals the same call on a
    profiled handle, whose iterations are launched from the host in chunks."""
    clips = [synth.clip(12, 40, 150, seed=31, cuts=(6, 9)),
             synth.clip(9, 56, 210, seed=32, cuts=(4, 7)),
             synth.clip(12, 40, 150, seed=33, cuts=(5, 8))]
    calls = [(0, 110, 8, False), (1, 140, 16, True), (0, 110, 8, True), (0, 110, 3, False),
             (2, 120, 8, False), (0, 110, 8, False)]
    r = lib.Retargeter()
    ref = lib.Retargeter()
    lib.scpl_set_profiling(ref.h, True)
    for ci, target, k, with_seams in calls:
        f = torch.from_numpy(clips[ci]).cuda()
        a = r.carve(f, target, k, with_seams=with_seams)
        b = ref.carve(f, target, k, with_seams=with_seams)
        torch.cuda.synchronize()
        assert torch.equal(a[0], b[0]), (ci, target, k, with_seams)
        assert np.array_equal(a[1], b[1])
        if with_seams:
            assert torch.equal(a[2], b[2])
    r.close()
    ref.close()


def test_launch_count_of_a_carve(lib, synth):
    """scpl_get_stats reports the kernels the last carve launched: with the
    iterations looping on the device, the scan, the initialisation, whole
    loop bodies (8 DP + 8 update launches and one condition kernel, up to the
    longest buffer's iterations) and the gather; profiled, the scan, the
    initialisation, the DP and update launches of the host's chunks and the
    gather."""
    f = torch.from_numpy(synth.clip(10, 40, 120, seed=41, cuts=(5, 8))).cuda()
    h = lib.scpl_create()
    out = torch.empty((10, 40, 80, 3), dtype=torch.uint8, device="cuda")
    lib.scpl_carve(h, f, 80, 4, out)
    torch.cuda.synchronize()
    st = lib.scpl_get_stats(h)
    bodies = max(1, -(-st["iterations_max"] // 8))
    assert st["launches"] == 3 + bodies * 17, st
    lib.scpl_set_profiling(h, True)
    lib.scpl_carve(h, f, 80, 4, out)
    st = lib.scpl_get_stats(h)
    assert st["launches"] == sum(k["launches"] for k in st["kernels"].values()), st
    lib.scpl_set_profiling(h, False)
    lib.scpl_destroy(h)


def test_errors(lib):
    h = lib.scpl_create()
    f = torch.zeros((1, 4, 4, 3), dtype=torch.uint8, device="cuda")
    out = torch.zeros((1, 4, 5, 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(lib.SCPLError):
        lib.scpl_carve(h, f, 5, 1, out)
    st = lib.load().scpl_carve(h, f.data_ptr(), 1, 4, 4, 5, 1, out.data_ptr(), None, None, None)
    assert st == lib.SCPL_EINVAL and "target_W" in lib.scpl_last_error(h)
    st = lib.load().scpl_carve(h, f.data_ptr(), 1, 4, 4, 3, 0, out.data_ptr(), None, None, None)
    assert st == lib.SCPL_EINVAL
    lib.scpl_destroy(h)
    # a huge height overflows the 32-bit cumulative energy
    h = lib.scpl_create(lib.Params(0.2, 1, 2, 128, 1, 0))
    big = torch.zeros((1, 1, 1, 3), dtype=torch.uint8, device="cuda")
    st = lib.load().scpl_scan(h, big.data_ptr(), 128, 65535, 1, None, None)
    assert st == lib.SCPL_EOVERFLOW
    lib.scpl_destroy(h)


# ------------------------------------------- full-size 1080p, sampled parity
@pytest.mark.slow
def test_carve_1080p_full_size_sampled(orc, lib, synth):
    """The 300-frame 1920x1080 workload in the same launch configuration the
    benchmark times: buffer boundaries compared with the oracle's scan, every
    buffer checked by the carving invariants (disjoint seams, output = input
    minus the seams' pixels), and the shortest buffer carved by the oracle
    and compared byte for byte."""
    f = synth.workload_clip_1080p()
    T, H, W = f.shape[:3]
    target, k = 1344, 32
    out, starts, seams = _carve_gpu(lib, f, target, k)
    e = orc.energy(f)
    assert np.array_equal(starts, orc.scan(e))
    del e
    for b in range(len(starts) - 1):
        sb = seams[b].astype(np.int64)
        srt = np.sort(sb, axis=0)
        assert (np.diff(srt, axis=0) > 0).all(), "seams overlap"
        for t in (starts[b], starts[b + 1] - 1):
            keep = np.ones((H, W), bool)
            keep[np.arange(H)[None, :].repeat(sb.shape[0], 0), sb] = False
            assert np.array_equal(out[t], f[t][keep].reshape(H, target, 3))
    b = int(np.argmin(np.diff(starts)))
    t0, t1 = starts[b], starts[b + 1]
    D = orc.motion(f[max(t0 - 1, 0):t1])[1 if t0 > 0 else 0:]
    ref_out, ref_seams, _ = orc.carve_buffer(f[t0:t1], D, target, k)
    assert np.array_equal(seams[b], ref_seams)
    assert np.array_equal(out[t0:t1], ref_out)


# ------------------------------------------------- 3840x2160 (serving sizes)
def test_seams_3840x2160(orc, lib):
    """The widest serving size: a 15-CTA cluster per buffer."""
    r = np.random.default_rng(2160)
    E = r.integers(0, 2551, (2160, 3840)).astype(np.int32)
    CE, L, d = orc.dp(E)
    ref_cols = orc.select(CE[-1], L[-1], 64)
    h = lib.scpl_create()
    cols = torch.full((64, 2160), -1, dtype=torch.int16, device="cuda")
    ke = lib.scpl_seams(h, torch.from_numpy(E).cuda(), 64, cols)
    lib.scpl_destroy(h)
    assert ke == len(ref_cols)
    got = cols.cpu().numpy()
    for s, c in enumerate(ref_cols):
        assert np.array_equal(got[s], orc.backtrack(d, int(c))), f"seam {s}"


def test_carve_3840x2160(orc, lib, synth):
    f = synth.clip(3, 2160, 3840, seed=61)
    ref, got = _carve_both(orc, lib, f, 3840 - 96, 64)
    _assert_same(ref, got)


# ------------------------------------ the integers behind every scan decision
def _oracle_A(orc, e, starts, t_max):
    """A_t of every frame from the oracle's energy and buffers: the sum over
    the buffer that was open when frame t arrived, frame t included."""
    T = e.shape[0]
    A = np.zeros(T, np.int64)
    bstart = {int(s): b for b, s in enumerate(starts[:-1])}
    for b in range(len(starts) - 1):
        s0, s1 = int(starts[b]), int(starts[b + 1])
        for t in range(s0, s1):
            lo = s0
            if t == s0 and b > 0 and (s0 - int(starts[b - 1])) < t_max:
                lo = int(starts[b - 1])   # frame t was tested against the previous buffer
            A[t] = orc.asde_sum(e[lo:t + 1])
    return A


@pytest.mark.parametrize("T,H,W,seed,t_max,cuts", [(40, 61, 300, 71, 128, (8, 14)),
                                                     (30, 200, 1000, 72, 7, (5, 9)),
                                                     (12, 1080, 1920, 73, 128, (5, 7)),
                                                     (6, 17, 5, 74, 2, None)])
def test_scan_stats_every_frame(orc, lib, synth, T, H, W, seed, t_max, cuts):
    f = synth.clip(T, H, W, seed=seed, cuts=cuts)
    e = orc.energy(f)
    h = lib.scpl_create(lib.Params(0.2, 1, 2, t_max, 1, 0))
    starts, A, M = lib.scpl_scan_stats(h, torch.from_numpy(f).cuda())
    lib.scpl_destroy(h)
    ref_starts = orc.scan(e, t_max=t_max)
    assert np.array_equal(starts, ref_starts)
    assert np.array_equal(M, e.reshape(T, -1).max(axis=1))
    assert np.array_equal(A, _oracle_A(orc, e, ref_starts, t_max))


def test_carve_more_buffers_than_kept_sums(orc, lib, synth):
    """t_max = 2 over 40 frames: 20 buffers, more than the scan keeps summed
    energy for, so k_energy_init sums the rest itself."""
    f = synth.clip(40, 30, 64, seed=75)
    ref, got = _carve_both(orc, lib, f, 50, 4, t_max=2)
    _assert_same(ref, got)


def test_carve_host_pipelined_matches_oracle(orc, lib, synth):
    """37 frames arrive in 5 chunks while the scan runs; buffers are gathered
    and sent back as each finishes.  Same bytes as the oracle."""
    f = synth.clip(37, 60, 130, seed=95, cuts=(6, 11))
    ref_out, ref_starts, ref_seams = orc.carve(f, 100, 8)
    h = lib.scpl_create()
    src = torch.from_numpy(f).pin_memory().numpy()
    out = torch.zeros((37, 60, 100, 3), dtype=torch.uint8).pin_memory().numpy()
    seams = np.zeros((37, 30, 60), np.int16)
    starts = lib.scpl_carve_host(h, src, 100, 8, out, seams)
    lib.scpl_destroy(h)
    assert np.array_equal(starts, ref_starts)
    assert np.array_equal(seams[: len(starts) - 1], ref_seams)
    assert np.array_equal(out, ref_out)


def test_carve_host_many_equals_each_clip_alone(lib):
    """Streamed host clips (two device slots, copies overlapping the
    kernels): every clip's result equals scpl_carve_host on that clip."""
    from paper_1903_03180_gb300 import synth
    T, H, W, tw, k = 20, 64, 112, 84, 8
    clips = [torch.from_numpy(synth.clip(T, H, W, seed=90 + i, cuts=(6, 12))).pin_memory().numpy()
             for i in range(5)]
    outs = [torch.zeros((T, H, tw, 3), dtype=torch.uint8).pin_memory().numpy() for _ in clips]
    h = lib.scpl_create()
    nbs = lib.scpl_carve_host_many(h, clips, tw, k, outs)
    refs = []
    for c in clips:
        o = np.zeros((T, H, tw, 3), np.uint8)
        refs.append((lib.scpl_carve_host(h, c, tw, k, o), o))
    lib.scpl_destroy(h)
    for i, (starts, ref) in enumerate(refs):
        assert nbs[i] == len(starts) - 1
        assert np.array_equal(outs[i], ref), i


def test_keff_log_matches_oracle(orc, lib):
    """The seams removed per iteration (Eq. 6: min(k, parents, remaining)),
    buffer by buffer, equal the oracle's."""
    from paper_1903_03180_gb300 import synth
    f = synth.clip(9, 40, 90, seed=95, cuts=(4, 5))
    r = lib.Retargeter()
    _, starts, _ = r.carve(torch.from_numpy(f).cuda(), 60, 6)
    log = lib.scpl_keff_log(r.h)
    r.close()
    D = orc.motion(f)
    assert len(log) == len(starts) - 1
    for b in range(len(starts) - 1):
        t0, t1 = starts[b], starts[b + 1]
        _, _, keff = orc.carve_buffer(f[t0:t1], D[t0:t1], 60, 6)
        assert list(log[b]) == list(keff), b
