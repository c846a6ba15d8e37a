"""Pins for the CPU oracle: each test checks it against something other than
itself -- closed forms, library routines, brute force, a textbook classic seam
carver, a hand-worked example, invariants that the paper's Sec. 3.1 argument
fixes.  No GPU is needed."""
from __future__ import annotations

import math
import os

import numpy as np
import pytest

from tests import textbook as tb

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- luma (R1)
def test_luma_grey_is_exact(orc):
    # the integer coefficients sum to 256, so a grey pixel keeps its value
    v = np.arange(256, dtype=np.uint8)
    rgb = np.stack([v, v, v], -1)[None]
    assert np.array_equal(orc.luma(rgb)[0], v)


def test_luma_within_one_of_float_bt601(orc):
    r = np.random.default_rng(0)
    rgb = r.integers(0, 256, (64, 97, 3), dtype=np.uint8)
    rgb[0, :8] = [[255, 0, 0], [0, 255, 0], [0, 0, 255], [255, 255, 0], [0, 255, 255],
                  [255, 0, 255], [255, 255, 255], [0, 0, 0]]
    y = orc.luma(rgb).astype(np.float64)
    assert np.max(np.abs(y - tb.luma_bt601_float(rgb))) <= 1.0


# ------------------------------------------------------------- Sobel (R2)
def test_sobel_closed_forms(orc):
    H, W = 7, 9
    assert not orc.sobel(np.full((H, W), 77, np.uint8)).any()
    ramp = np.tile(np.arange(W, dtype=np.uint8) * 3, (H, 1))
    G = orc.sobel(ramp)
    assert (G[:, 1:-1] == 8 * 3).all() and (G[:, 0] == 4 * 3).all() and (G[:, -1] == 4 * 3).all()
    G = orc.sobel(np.ascontiguousarray(ramp.T))
    assert (G[1:-1] == 24).all() and (G[0] == 12).all() and (G[-1] == 12).all()
    step = np.zeros((H, W), np.uint8)
    step[:, 4:] = 50
    G = orc.sobel(step)
    assert (G[:, 3] == 200).all() and (G[:, 4] == 200).all()
    assert not np.delete(G, [3, 4], axis=1).any()


def test_sobel_matches_scipy(orc):
    r = np.random.default_rng(1)
    for H, W in [(1, 1), (1, 5), (5, 1), (2, 2), (13, 31), (40, 17)]:
        Y = r.integers(0, 256, (H, W), dtype=np.uint8)
        assert np.array_equal(orc.sobel(Y), tb.sobel_scipy(Y))


# ------------------------------------------------------ motion energy (R3)
def test_motion_and_blend_hand_case(orc):
    f = np.zeros((3, 4, 6, 3), np.uint8)
    f[0], f[1], f[2] = 10, 30, 25
    assert np.array_equal(orc.motion(f)[:, 0, 0], [0, 20, 5])
    e = orc.energy(f, wg=1, wm=2)
    assert np.array_equal(e[:, 2, 3], [0, 40, 10])
    e = orc.energy(f, wg=1, wm=0)
    assert not e.any()


def test_energy_matches_scipy(orc):
    r = np.random.default_rng(2)
    f = r.integers(0, 256, (4, 11, 23, 3), dtype=np.uint8)
    for wg, wm in [(1, 0), (1, 2), (2, 3)]:
        ref = tb.energy_scipy(f, wg, wm, orc.luma)
        assert np.array_equal(orc.energy(f, wg, wm), ref)


# ------------------------------------------------ DP, labels, ties (R4-R5)
def _load_golden(name):
    blocks, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line[0].isalpha():
                cur = line
                blocks[cur] = []
            else:
                blocks[cur].append([int(x) for x in line.split()])
    return {k: np.array(v) for k, v in blocks.items()}


def test_dp_hand_worked_example(orc):
    g = _load_golden("dp_3x5.txt")
    CE, L, d = orc.dp(g["energy"])
    assert np.array_equal(CE, g["ce"])
    assert np.array_equal(L, g["labels"])
    assert np.array_equal(d, g["dir"])
    assert np.array_equal(orc.select(CE[-1], L[-1], 1), g["select_k1"][0])
    assert np.array_equal(orc.select(CE[-1], L[-1], 2), g["select_k2"][0])
    assert np.array_equal(orc.backtrack(d, 1), g["seam_from_1"][0])
    assert np.array_equal(orc.backtrack(d, 4), g["seam_from_4"][0])


@pytest.mark.parametrize("H,W,vmax,seed", [(1, 4, 3, 0), (2, 3, 2, 1), (4, 5, 3, 2), (5, 6, 2, 3),
                                          (5, 6, 9, 4), (3, 6, 0, 5), (5, 4, 1, 6)])
def test_dp_brute_force(orc, H, W, vmax, seed):
    """CE(H-1, j) is the least cost of all seams ending at j; the traced path is
    the lexicographically least (c_{H-2}, ..., c_0) among them; its row-0
    column is the label (Eq. 4, Eq. 5, lowest-column tie reading)."""
    r = np.random.default_rng(seed)
    E = r.integers(0, vmax + 1, (H, W)).astype(np.int32)
    CE, L, d = orc.dp(E)
    best = {}
    for path in tb.all_seams(H, W):
        cost = int(sum(E[i, c] for i, c in enumerate(path)))
        key = (cost, tuple(reversed(path[:-1])))
        j = path[-1]
        if j not in best or key < best[j][0]:
            best[j] = (key, path)
    for j in range(W):
        (cost, _), path = best[j]
        assert CE[-1, j] == cost
        assert L[-1, j] == path[0]
        assert tuple(orc.backtrack(d, j)) == path


def test_labels_non_decreasing_and_seams_disjoint(orc):
    """Sec. 3.1: paths never cross, so labels are sorted along every row and
    the traced seams of different parents share no pixel (Eq. 5)."""
    r = np.random.default_rng(7)
    for trial in range(20):
        H, W = int(r.integers(1, 40)), int(r.integers(1, 60))
        E = r.integers(0, int(r.integers(1, 50)), (H, W)).astype(np.int32)
        CE, L, d = orc.dp(E)
        assert (np.diff(L, axis=1) >= 0).all()
        cols = orc.select(CE[-1], L[-1], W)
        assert len(cols) == len(np.unique(L[-1]))
        paths = np.array([orc.backtrack(d, c) for c in cols])
        for i in range(H):
            assert len(np.unique(paths[:, i])) == len(cols)
        assert (np.abs(np.diff(paths, axis=1)) <= 1).all()


# --------------------------------------------------------- selection (R6)
def test_select_k1_is_global_argmin(orc):
    r = np.random.default_rng(8)
    for _ in range(30):
        H, W = int(r.integers(1, 20)), int(r.integers(1, 40))
        E = r.integers(0, 5, (H, W)).astype(np.int32)
        CE, L, _ = orc.dp(E)
        M, _ = tb.classic_dp(E)
        assert np.array_equal(CE, M)
        assert orc.select(CE[-1], L[-1], 1)[0] == int(np.argmin(M[-1]))


def test_select_per_parent_minimum(orc):
    r = np.random.default_rng(9)
    for _ in range(30):
        H, W = int(r.integers(1, 25)), int(r.integers(2, 50))
        E = r.integers(0, 4, (H, W)).astype(np.int32)
        CE, L, _ = orc.dp(E)
        cols = orc.select(CE[-1], L[-1], W)
        # every parent appears once, with the least (CE, column) of its children
        for c in cols:
            same = np.nonzero(L[-1] == L[-1, c])[0]
            assert c == same[np.lexsort((same, CE[-1, same]))][0]
        keys = [(CE[-1, c], c) for c in cols]
        assert keys == sorted(keys)
        for cap in range(1, len(cols) + 2):
            assert np.array_equal(orc.select(CE[-1], L[-1], cap), cols[:cap])


# ------------------------------------------- whole carve vs textbook SC (R9)
def test_k1_single_frame_equals_classic_seam_carving(orc):
    """With k = 1 and one frame, SCPL is classic Avidan-Shamir seam carving."""
    from paper_1903_03180_gb300 import synth
    f = synth.still_frame(36, 48, seed=11, n_rects=4)
    n = 12
    ref, ref_seams = tb.classic_seam_carve(f, n, lambda im: tb.sobel_scipy(orc.luma(im)))
    out, starts, seams = orc.carve(f[None], 48 - n, 1, wg=1, wm=0, use_buffer=False)
    assert np.array_equal(out[0], ref)
    assert np.array_equal(seams[0], ref_seams)


def test_k1_per_frame_raw_video_equals_classic(orc):
    from paper_1903_03180_gb300 import synth
    c = synth.clip(3, 24, 40, seed=12)
    out, starts, seams = orc.carve(c, 34, 1, wg=1, wm=0, use_buffer=False)
    assert np.array_equal(starts, [0, 1, 2, 3])
    for t in range(3):
        ref, _ = tb.classic_seam_carve(c[t], 6, lambda im: tb.sobel_scipy(orc.luma(im)))
        assert np.array_equal(out[t], ref)


def _check_carve_invariants(frames, out, starts, seams, target):
    T, H, W0 = frames.shape[:3]
    for b in range(len(starts) - 1):
        sb = seams[b]                                   # [W0-target, H] original columns
        for i in range(H):
            assert len(np.unique(sb[:, i])) == W0 - target   # disjoint, every row narrows
        for t in range(starts[b], starts[b + 1]):
            for i in range(H):
                keep = np.delete(frames[t, i], sb[:, i], axis=0)
                assert np.array_equal(out[t, i], keep)


def _current_columns(seams_b, H, W0):
    """Convert removal-order original columns into the column each pixel had
    at the time of its removal."""
    removed = [[] for _ in range(H)]
    cur = np.empty_like(seams_b)
    for s in range(seams_b.shape[0]):
        for i in range(H):
            o = int(seams_b[s, i])
            cur[s, i] = o - sum(1 for x in removed[i] if x < o)
        for i in range(H):
            removed[i].append(int(seams_b[s, i]))
    return cur


def test_multi_seam_invariants(orc):
    from paper_1903_03180_gb300 import synth
    c = synth.clip(6, 30, 52, seed=13)
    target = 36
    out, starts, seams = orc.carve(c, target, 5, wg=1, wm=2, t_max=4)
    assert starts[0] == 0 and starts[-1] == 6 and (np.diff(starts) <= 4).all()
    _check_carve_invariants(c, out, starts, seams, target)
    for b in range(len(starts) - 1):
        cur = _current_columns(seams[b], 30, 52)
        # every seam is 8-connected at the width it was removed at
        assert (np.abs(np.diff(cur, axis=1)) <= 1).all()


@pytest.mark.parametrize("seed", range(8))
def test_buffer_seam_is_least_costly_with_motion(orc, seed):
    """Brute force over every seam of a small multi-frame buffer (R8): the seam
    removed first has the least sum, along it, of every frame's energy
    wg*G_t + wm*D_t (the energies from `orc.energy`, pinned against scipy)."""
    r = np.random.default_rng(700 + seed)
    T, H, W = int(r.integers(2, 4)), int(r.integers(3, 6)), int(r.integers(4, 8))
    wg, wm = int(r.integers(0, 2)), int(r.integers(1, 4))
    f = r.integers(0, 256, (T, H, W, 3), dtype=np.uint8)
    _, seams, _ = orc.carve_buffer(f, orc.motion(f), W - 1, 1, wg=wg, wm=wm)
    E = orc.energy(f, wg, wm).sum(0)
    cost = lambda s: int(sum(E[i, c] for i, c in enumerate(s)))
    assert cost(seams[0]) == min(cost(s) for s in tb.all_seams(H, W))


def test_kbig_removes_one_seam_per_parent(orc):
    from paper_1903_03180_gb300 import synth
    f = synth.still_frame(20, 40, seed=14, n_rects=3)
    D = np.zeros((1, 20, 40), np.uint8)
    out, seams, keff = orc.carve_buffer(f[None], D, 30, 1000, wg=1, wm=0)
    E = orc.energy(f[None], 1, 0)[0]
    CE, L, d = orc.dp(E)
    assert keff[0] == min(len(np.unique(L[-1])), 10)
    assert keff.sum() == 10


# ----------------------------------------------------- buffer, ASDE (R7)
def test_isqrt_exact(orc):
    r = np.random.default_rng(15)
    xs = [0, 1, 2, 3, 4, 15, 16, 17, 2 ** 52 - 1, 2 ** 52, 2 ** 53 + 1, (2 ** 31 - 1) ** 2,
          (2 ** 31 - 1) ** 2 - 1, (10 ** 8) ** 2 + 10 ** 8]
    xs += [int(v) for v in r.integers(0, 2 ** 62, 200, dtype=np.int64)]
    for x in xs:
        assert orc.isqrt(x) == math.isqrt(x)


def test_threshold_is_eq9(orc):
    """Eq. 9 in its printed form equals the scaled threshold / (256*n*H*W)."""
    for n in range(1, 40):
        for M in [1, 255, 2550, 7777]:
            for alpha in [0.15, 0.2, 0.25]:
                mv = float(M)
                phi = alpha * math.sqrt(((mv - mv / n) ** 2 + (n - 1) * (mv / n) ** 2) / n)
                thr = orc.threshold(n, M, 6, 9, alpha)
                assert thr / (256 * n * 6 * 9) == pytest.approx(phi, rel=1e-12, abs=1e-12)


def test_asde_matches_numpy_std(orc):
    """A/(256*n*H*W) is Eq. 7 (mean of Eq. 8's population STD) up to the
    1/256 floor of each pixel's term."""
    r = np.random.default_rng(16)
    for n in [1, 2, 3, 7, 16]:
        e = r.integers(0, 2551, (n, 9, 13)).astype(np.int32)
        A = orc.asde_sum(e)
        asde = float(np.mean(np.std(e.astype(np.float64), axis=0)))
        approx = A / (256.0 * n * e.shape[1] * e.shape[2])
        assert asde - 1.0 / (256 * n) - 1e-9 <= approx <= asde + 1e-9


def test_fig4_worst_case_construction(orc):
    """Fig. 4: n-1 frames of the lowest energy then one of the highest.  Each
    pixel's STD is then M*sqrt(n-1)/n, so ASDE = phi(n)/alpha exactly."""
    H, W, M = 5, 7, 2550
    for n in range(2, 30):
        e = np.zeros((n, H, W), np.int32)
        e[-1] = M
        A = orc.asde_sum(e)
        assert A == H * W * math.isqrt(65536 * M * M * (n - 1))
        assert orc.exceeds(A, n, M, H, W, 0.2)
        assert not orc.exceeds(A, n, M, H, W, 1.0)     # floor never exceeds alpha = 1
        st = orc.scan(e, alpha=0.2)
        assert np.array_equal(st, [0, n - 1, n])           # the spike starts a new buffer


def test_constant_clip_fills_to_t_max(orc):
    e = np.full((70, 4, 6), 123, np.int32)
    assert np.array_equal(orc.scan(e, t_max=16), [0, 16, 32, 48, 64, 70])
    assert np.array_equal(orc.scan(e[:1], t_max=16), [0, 1])
    assert np.array_equal(orc.scan(e, t_max=1), np.arange(71))


def _scan_float_reference(e, alpha, t_max):
    """Sec. 3.2 with Eq. 7-9 in floating point as printed (np.std, Eq. 9's
    unsimplified form).  Returns the starts and the smallest relative margin."""
    T = e.shape[0]
    starts, start, margin = [], 0, np.inf
    buf = []
    for f in range(T):
        cand = buf + [e[f]]
        n = len(cand)
        if n >= 2:
            asde = float(np.mean(np.std(np.array(cand, np.float64), axis=0)))
            M = float(np.max(cand))
            phi = alpha * math.sqrt(((M - M / n) ** 2 + (n - 1) * (M / n) ** 2) / n)
            margin = min(margin, abs(asde - phi) / max(phi, 1e-9))
            if asde > phi:
                starts.append(start)
                start, buf = f, [e[f]]
                continue
        buf = cand
        if len(buf) == t_max:
            starts.append(start)
            start, buf = f + 1, []
    if buf:
        starts.append(start)
    return starts + [T], margin


def test_scan_matches_float_reading_of_eq7_9(orc):
    r = np.random.default_rng(17)
    checked = 0
    for trial in range(40):
        T, H, W = int(r.integers(2, 14)), int(r.integers(2, 8)), int(r.integers(2, 8))
        base = r.integers(0, 600, (H, W))
        jitter = int(r.integers(1, 400))
        e = np.stack([base + r.integers(0, jitter, (H, W)) * (r.random() < 0.3)
                      for _ in range(T)]).astype(np.int32)
        ref, margin = _scan_float_reference(e, 0.2, 6)
        if margin < 1e-3:
            continue
        assert list(orc.scan(e, alpha=0.2, t_max=6)) == ref
        checked += 1
    assert checked >= 20


def test_maxval_theoretical_mode(orc):
    # with M fixed at the theoretical maximum the bar is higher than with the
    # running maximum, so the spike of the Fig. 4 construction (M = 100) stays
    e = np.zeros((6, 3, 3), np.int32)
    e[-1] = 100
    assert np.array_equal(orc.scan(e, maxval_mode=0), [0, 5, 6])
    assert np.array_equal(orc.scan(e, maxval_mode=1, maxval_theory=2550), [0, 6])


def test_buffer_carves_same_seams_from_every_frame(orc):
    """Sec. 3.2: one seam set per buffer, applied to all of its frames."""
    from paper_1903_03180_gb300 import synth
    c = synth.clip(8, 24, 40, seed=18, pan=0, noise=0)
    out, starts, seams = orc.carve(c, 30, 4, t_max=8)
    _check_carve_invariants(c, out, starts, seams, 30)
    e = orc.energy(c)
    assert np.array_equal(starts, orc.scan(e, t_max=8))


def test_new_buffer_keeps_its_first_frames_maximum(orc):
    """After a flush the frame that starts the new buffer is part of it, so its
    maximum energy is the new buffer's maxval (Eq. 9's maxval over the buffer).
    Frames 0-2 are zero, frame 3 spikes to 2550 and starts buffer 2, frame 4
    drops to 2100: with maxval 2550 the drop (STD sum 450*H*W) stays under
    0.2*2550*H*W = 510*H*W, so frame 4 joins; a maxval of 2100 would flush it."""
    e = np.zeros((5, 3, 4), np.int32)
    e[3], e[4] = 2550, 2100
    assert np.array_equal(orc.scan(e, alpha=0.2), [0, 3, 5])


def test_new_buffer_does_not_inherit_the_closed_buffers_maximum(orc):
    """Eq. 9's maxval belongs to the open buffer: frame 0 peaks at 2550 and the
    zero frame 1 flushes it, so buffer 2 starts with maxval 0.  Frame 2 at 10
    spreads it by 10 per pixel (STD sum 10*H*W) against 0.2*10*H*W, so frame 2
    starts buffer 3; had the closed buffer's 2550 carried over (threshold
    510*H*W) it would have joined."""
    e = np.zeros((3, 3, 4), np.int32)
    e[0], e[2] = 2550, 10
    assert np.array_equal(orc.scan(e, alpha=0.2), [0, 1, 2, 3])


# ------------------------------------------------ C12: horizontal seams (Sec. 2)
def test_carve_job_height_is_classic_horizontal_seam_carving(orc):
    """k = 1, one frame, gradient energy: the job's height pass removes the
    same pixels as a horizontal seam carver written column by column."""
    from paper_1903_03180_gb300 import synth
    f = synth.clip(1, 18, 26, seed=31)
    out, starts = orc.carve_job(f, 26, 13, 1, wm=0, use_buffer=False)
    ref = tb.classic_horizontal_seam_carve(f[0], 5, lambda im: tb.sobel_scipy(orc.luma(im)))
    assert out.shape == (1, 13, 26, 3)
    assert np.array_equal(out[0], ref)
    assert list(starts) == [0, 1]


def test_carve_job_both_is_width_then_height(orc):
    """Both dimensions: classic vertical seams first, then horizontal ones."""
    from paper_1903_03180_gb300 import synth
    f = synth.clip(1, 16, 22, seed=32)
    efn = lambda im: tb.sobel_scipy(orc.luma(im))
    out, _ = orc.carve_job(f, 17, 12, 1, wm=0, use_buffer=False)
    mid, _ = tb.classic_seam_carve(f[0], 5, efn)
    ref = tb.classic_horizontal_seam_carve(mid, 4, efn)
    assert np.array_equal(out[0], ref)


def test_carve_job_width_only_is_carve(orc):
    from paper_1903_03180_gb300 import synth
    f = synth.clip(5, 20, 40, seed=33)
    out, starts = orc.carve_job(f, 30, 20, 4, t_max=3)
    ref, ref_starts, _ = orc.carve(f, 30, 4, t_max=3)
    assert np.array_equal(out, ref) and np.array_equal(starts, ref_starts)


# ------------------------------------ N4: blend sharpness (Sec. 4, Fig. 9 stand-in)
def _gray(Y):
    """RGB frame whose integer BT.601 luma is exactly Y (R = G = B)."""
    Y = np.asarray(Y, np.uint8)
    return np.repeat(Y[..., None], 3, axis=-1)


def test_blend_sharpness_step_edge_closed_form(orc):
    """One frame, a vertical step of height h at column c: with a replicate
    border the L1 Sobel gives 4h on the two columns next to the step and 0
    elsewhere (rows are identical, so Gy = 0): 8 h H in all."""
    H, W, c, h = 7, 12, 5, 10
    Y = np.zeros((H, W), np.uint8)
    Y[:, c:] = h
    num, den = orc.blend_sharpness(_gray(Y)[None], window=1)
    assert num == den == 8 * h * H


def test_blend_sharpness_static_frames_are_sharp(orc):
    """Identical frames: the blend is window x the frame and Sobel is linear."""
    from paper_1903_03180_gb300 import synth
    f = synth.still_frame(20, 30, seed=41)
    num, den = orc.blend_sharpness(np.repeat(f[None], 6, axis=0), window=4)
    assert num == den > 0


def test_blend_sharpness_complementary_frames_cancel(orc):
    """Gray frames alternating g and 255 - g: every blend of 4 is the constant
    510, so it has no gradient at all while each frame has."""
    r = np.random.default_rng(42)
    g = r.integers(0, 256, (9, 13), dtype=np.uint8)
    frames = np.stack([_gray(g), _gray(255 - g)] * 3)
    num, den = orc.blend_sharpness(frames, window=4)
    assert num == 0 and den > 0


def test_blend_sharpness_displaced_content_blurs(orc):
    """A frame and the same frame moved one column: the blend is blurred."""
    from paper_1903_03180_gb300 import synth
    f = synth.still_frame(24, 40, seed=43)
    moved = np.concatenate([f[:, :1], f[:, :-1]], axis=1)
    num, den = orc.blend_sharpness(np.stack([f, moved]), window=2)
    assert 0 < num < den


def test_blend_sharpness_short_clip_is_empty(orc):
    f = np.zeros((3, 4, 5, 3), np.uint8)
    assert orc.blend_sharpness(f, window=4) == (0, 0)


# ------------------------------------------------ N4: seam insertion (enlarging)
def _drop_inserted(out: np.ndarray, W: int, inserted_after: list) -> np.ndarray:
    """Remove, row by row, the pixel that follows each listed original column."""
    H = out.shape[0]
    rows = []
    for i in range(H):
        keep, p = [], 0
        for x in range(W):
            keep.append(p)
            p += 2 if x in inserted_after[i] else 1
        rows.append(out[i, keep])
    return np.stack(rows)


def test_enlarge_k1_inserts_the_classic_seams(orc):
    """k = 1, one frame, gradient energy: the inserted pixels follow exactly
    the first m seams of classic seam carving, each is the rounded mean of its
    neighbours, and dropping them gives the original frame back."""
    from paper_1903_03180_gb300 import synth
    f = synth.still_frame(16, 24, seed=51)
    m = 5
    out, starts = orc.enlarge(f[None], 24 + m, 1, wm=0, use_buffer=False)
    _, seams = tb.classic_seam_carve(f, m, lambda im: tb.sobel_scipy(orc.luma(im)))
    inserted = [set(int(s) for s in seams[:, i]) for i in range(16)]
    assert out.shape == (1, 16, 24 + m, 3)
    assert np.array_equal(_drop_inserted(out[0], 24, inserted), f)
    for i in range(16):
        p = 0
        for x in range(24):
            if x in inserted[i]:
                a = f[i, x].astype(int)
                b = f[i, min(x + 1, 23)].astype(int)
                assert np.array_equal(out[0, i, p + 1], (a + b + 1) >> 1)
                p += 2
            else:
                p += 1


def test_enlarge_shares_seams_within_a_buffer(orc):
    """Video: every frame of a buffer gets the same inserted columns (those
    that carving the clip removes from the buffer), and dropping them gives
    each frame back."""
    from paper_1903_03180_gb300 import synth
    f = synth.clip(6, 14, 20, seed=52, cuts=(3, 3))
    out, starts = orc.enlarge(f, 27, 4)
    _, cstarts, seams = orc.carve(f, 13, 4)
    assert np.array_equal(starts, cstarts)
    for b in range(len(starts) - 1):
        inserted = [set(int(s) for s in seams[b, :, i]) for i in range(14)]
        for t in range(starts[b], starts[b + 1]):
            assert np.array_equal(_drop_inserted(out[t], 20, inserted), f[t])


def test_enlarge_by_nothing_is_identity(orc):
    f = np.random.default_rng(53).integers(0, 256, (3, 5, 7, 3), dtype=np.uint8)
    out, starts = orc.enlarge(f, 7, 2)
    assert np.array_equal(out, f) and list(starts) == [0, 3]


# ------------------------------------------------------ N3: forward energy (R14)
def _inserted_luma(Y: np.ndarray, seam) -> int:
    """Luma differences between the pixels that become neighbours when `seam`
    (one column per row) is cut out of the luma frame Y: pairs that sit side by
    side, or one above the other, in the carved frame but did not in Y."""
    H, W = Y.shape
    orig = [[j for j in range(W) if j != seam[i]] for i in range(H)]
    total = 0
    for i in range(H):
        for c in range(W - 2):
            a, b = orig[i][c], orig[i][c + 1]
            if b - a != 1:
                total += abs(int(Y[i, b]) - int(Y[i, a]))
        if i > 0:
            for c in range(W - 1):
                a, b = orig[i - 1][c], orig[i][c]
                if a != b:
                    total += abs(int(Y[i - 1, a]) - int(Y[i, b]))
    return total


def _forward_cost(orc, f, seam, wg, wm, wf):
    """Backward energy of the buffer along the seam plus wf times the luma
    differences its removal creates in every frame."""
    E = orc.energy(f, wg, wm).sum(0)
    Y = [orc.luma(f[t]) for t in range(f.shape[0])]
    return (int(sum(E[i, c] for i, c in enumerate(seam))) +
            wf * sum(_inserted_luma(y, seam) for y in Y))


@pytest.mark.parametrize("seed", range(24))
def test_forward_seam_is_the_least_costly_of_all_seams(orc, seed):
    """Brute force over every seam of a tiny buffer: the seam the forward DP
    removes has the least backward energy plus wf times the differences its
    removal really creates.  Half the cases carry no backward energy, so the
    created differences alone decide; some use a coarse palette, which makes
    ties common."""
    r = np.random.default_rng(900 + seed)
    T, H, W = int(r.integers(1, 4)), int(r.integers(2, 6)), int(r.integers(3, 8))
    wg, wm, wf = int(r.integers(0, 3)), int(r.integers(0, 3)), int(r.integers(1, 4))
    if seed % 2 == 0:
        wg = wm = 0
    levels = np.array([0, 60, 200, 255], np.uint8) if seed % 3 == 0 else np.arange(256, dtype=np.uint8)
    f = levels[r.integers(0, len(levels), (T, H, W, 3))]
    _, seams, _ = orc.carve_buffer(f, orc.motion(f), W - 1, 1, wg=wg, wm=wm, wf=wf)
    best = min(_forward_cost(orc, f, s, wg, wm, wf) for s in tb.all_seams(H, W))
    assert _forward_cost(orc, f, seams[0], wg, wm, wf) == best


def test_forward_iterations_recompute_on_the_carved_frames(orc):
    """k = 1 over four iterations: each removed seam is the least costly of the
    frames as carved so far (brute force on the carved frames each time)."""
    r = np.random.default_rng(911)
    f = r.integers(0, 256, (2, 4, 7, 3), dtype=np.uint8)
    out, seams, keff = orc.carve_buffer(f, np.zeros((2, 4, 7), np.uint8), 3, 1, wg=1, wm=0, wf=2)
    assert list(keff) == [1, 1, 1, 1]
    cur = f.copy()
    orig = np.tile(np.arange(7), (4, 1))
    for s in range(4):
        W = cur.shape[2]
        seam = [int(np.nonzero(orig[i] == seams[s, i])[0][0]) for i in range(4)]
        best = min(_forward_cost(orc, cur, p, 1, 0, 2) for p in tb.all_seams(4, W))
        assert _forward_cost(orc, cur, seam, 1, 0, 2) == best
        keep = [[j for j in range(W) if j != seam[i]] for i in range(4)]
        cur = np.stack([np.stack([cur[t, i, keep[i]] for i in range(4)]) for t in range(2)])
        orig = np.stack([orig[i, keep[i]] for i in range(4)])
    assert np.array_equal(cur, out)


def test_forward_terms_of_a_ramp(orc):
    """Y = 3j: the horizontal term is 6 inside and 0 in the border columns, each
    diagonal move costs 3; with no backward energy the straight seam down the
    first column creates no new pair and is removed."""
    H, W = 5, 8
    ramp = np.tile((np.arange(W) * 3).astype(np.uint8), (H, 1))
    CU, A, B = orc.forward_terms(ramp)
    assert (CU[:, 1:-1] == 6).all() and not CU[:, [0, -1]].any()
    assert (A[1:, 1:] == 3).all() and (B[1:, :-1] == 3).all() and not A[0].any()
    f = np.stack([ramp] * 3, -1)[None]   # grey, so the luma is the ramp itself
    _, seams, _ = orc.carve_buffer(f, np.zeros((1, H, W), np.uint8), W - 1, 1, wg=0, wm=0, wf=1)
    assert (seams[0] == 0).all()


def test_forward_dp_with_zero_weight_is_the_plain_dp(orc):
    r = np.random.default_rng(912)
    E = r.integers(0, 50, (9, 13)).astype(np.int32)
    A, B = (r.integers(0, 255, (9, 13)).astype(np.int32) for _ in range(2))
    for x, y in zip(orc.dp_fwd(E, A, B, 0), orc.dp(E)):
        assert np.array_equal(x, y)


def test_forward_weight_shifts_seams_off_created_edges(orc):
    """One frame, no backward energy: a dark vertical bar two columns wide in
    a bright frame.  A seam through the bar joins bar and bright pixels, one
    beside it joins only bright ones; the forward cost sees the difference."""
    H, W = 6, 9
    img = np.full((H, W), 200, np.uint8)
    img[:, 3:5] = 20
    f = np.stack([img] * 3, -1)[None]
    _, seams, _ = orc.carve_buffer(f, np.zeros((1, H, W), np.uint8), W - 1, 1, wg=0, wm=0, wf=1)
    s = seams[0]
    assert _forward_cost(orc, f, s, 0, 0, 1) == 0
    assert not np.isin(s, [2, 3, 4, 5]).any()


# ------------------------------------- N4: insertion along the height (Sec. 2)
def _drop_inserted_rows(out: np.ndarray, H: int, inserted_after: list) -> np.ndarray:
    """Remove, column by column, the pixel that follows each listed original row."""
    return _drop_inserted(out.transpose(1, 0, 2), H, inserted_after).transpose(1, 0, 2)


def test_enlarge_job_height_inserts_the_classic_horizontal_seams(orc):
    """k = 1, one frame, gradient energy: the rows inserted into each column
    follow the horizontal seams of classic seam carving (found here as the
    vertical seams of the transposed frame, whose gradient is the transposed
    gradient), each new pixel is the rounded mean of the pixels above and
    below it, and dropping them gives the frame back."""
    from paper_1903_03180_gb300 import synth
    f = synth.still_frame(20, 15, seed=61)
    m = 4
    out = orc.enlarge_job(f[None], 15, 20 + m, 1, wm=0, use_buffer=False)
    assert out.shape == (1, 20 + m, 15, 3)
    ft = np.ascontiguousarray(f.transpose(1, 0, 2))
    _, seams = tb.classic_seam_carve(ft, m, lambda im: tb.sobel_scipy(orc.luma(im)))
    inserted = [set(int(s) for s in seams[:, j]) for j in range(15)]
    assert np.array_equal(_drop_inserted_rows(out[0], 20, inserted), f)
    for j in range(15):
        p = 0
        for x in range(20):
            if x in inserted[j]:
                a = f[x, j].astype(int)
                b = f[min(x + 1, 19), j].astype(int)
                assert np.array_equal(out[0, p + 1, j], (a + b + 1) >> 1)
                p += 2
            else:
                p += 1


def test_enlarge_job_both_drops_back_to_the_clip(orc):
    """Both dimensions on a multi-buffer clip: dropping the rows that the
    height stage inserted gives the width stage's result, and dropping the
    columns it inserted gives the clip back, frame by frame."""
    from paper_1903_03180_gb300 import synth
    f = synth.clip(6, 12, 18, seed=62, cuts=(3, 3))
    out = orc.enlarge_job(f, 23, 16, 3)
    mid, _ = orc.enlarge(f, 23, 3)
    assert np.array_equal(out, orc.enlarge_job(mid, 23, 16, 3))
    tr = np.ascontiguousarray(mid.transpose(0, 2, 1, 3))
    _, starts, seams = orc.carve(tr, 12 - 4, 3)
    _, wstarts, wseams = orc.carve(f, 18 - 5, 3)
    for b in range(len(starts) - 1):
        rows = [set(int(s) for s in seams[b, :, j]) for j in range(23)]
        for t in range(starts[b], starts[b + 1]):
            assert np.array_equal(_drop_inserted_rows(out[t], 12, rows), mid[t])
    for b in range(len(wstarts) - 1):
        cols = [set(int(s) for s in wseams[b, :, i]) for i in range(12)]
        for t in range(wstarts[b], wstarts[b + 1]):
            assert np.array_equal(_drop_inserted(mid[t], 18, cols), f[t])


def test_enlarge_job_identity_and_width_only(orc):
    f = np.random.default_rng(63).integers(0, 256, (3, 6, 9, 3), dtype=np.uint8)
    assert np.array_equal(orc.enlarge_job(f, 9, 6, 2), f)
    assert np.array_equal(orc.enlarge_job(f, 13, 6, 2), orc.enlarge(f, 13, 2)[0])


@pytest.mark.parametrize("wf", [1, 4])
def test_forward_multi_seam_invariants(orc, wf):
    """Forward terms with several seams an iteration on a multi-buffer clip:
    the removed pixels are disjoint and narrow every row, each seam is
    8-connected at the width it was removed at, and the output is the input
    minus the seams' pixels (the DP's moves cost more, the structure stays)."""
    from paper_1903_03180_gb300 import synth
    c = synth.clip(6, 26, 44, seed=913, cuts=(3, 3))
    target = 30
    out, starts, seams = orc.carve(c, target, 5, wf=wf, t_max=4)
    _check_carve_invariants(c, out, starts, seams, target)
    for b in range(len(starts) - 1):
        cur = _current_columns(seams[b], 26, 44)
        assert (np.abs(np.diff(cur, axis=1)) <= 1).all()


def test_forward_kbig_removes_one_seam_per_parent(orc):
    """The uncapped variant with forward terms: the first iteration removes one
    seam for every parent the forward DP's last row holds (capped by what is
    left to remove)."""
    from paper_1903_03180_gb300 import synth
    f = synth.still_frame(18, 36, seed=914, n_rects=3)
    D = np.zeros((1, 18, 36), np.uint8)
    out, seams, keff = orc.carve_buffer(f[None], D, 26, 1000, wg=1, wm=0, wf=2)
    Y = orc.luma(f)
    CU, A, B = orc.forward_terms(Y)
    E = orc.energy(f[None], 1, 0)[0] + 2 * CU
    CE, L, d = orc.dp_fwd(E, A, B, 2)
    assert keff[0] == min(len(np.unique(L[-1])), 10)
    assert keff.sum() == 10
