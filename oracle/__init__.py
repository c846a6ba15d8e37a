"""CPU oracle for SCPL video retargeting -- TEST INFRASTRUCTURE ONLY.

A plain single-threaded C statement of the method (``scpl_oracle.c``) with a
numpy/ctypes wrapper.  Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may load it.  The product library never
imports, links or calls anything here, and this module never imports the
product package.

Each wrapper names the passage of the paper (arXiv 1903.03180) it follows; the
readings taken where the paper is silent are listed at the top of the C file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "scpl_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

# Default parameters used across the tests and benchmarks (Sec. 3.2: alpha in
# [0.15, 0.25]; Sec. 3.3 weights are integers here).
ALPHA = 0.20
T_MAX = 128


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    P = ctypes.c_void_p
    i32, i64, dbl = ctypes.c_int, ctypes.c_int64, ctypes.c_double
    lib.orc_luma.argtypes = [P, i32, i32, P]
    lib.orc_sobel.argtypes = [P, i32, i32, P]
    lib.orc_motion.argtypes = [P, i32, i32, i32, P]
    lib.orc_energy.argtypes = [P, i32, i32, i32, i32, i32, P]
    lib.orc_dp.argtypes = [P, i32, i32, P, P, P]
    lib.orc_select.argtypes = [P, P, i32, i32, P]
    lib.orc_backtrack.argtypes = [P, i32, i32, i32, P]
    lib.orc_isqrt.argtypes = [ctypes.c_uint64]
    lib.orc_isqrt.restype = ctypes.c_uint64
    lib.orc_asde_sum.argtypes = [P, i32, i32, i32, P]
    lib.orc_threshold.argtypes = [i32, i64, i32, i32, dbl]
    lib.orc_threshold.restype = dbl
    lib.orc_exceeds.argtypes = [i64, i32, i64, i32, i32, dbl]
    lib.orc_scan.argtypes = [P, i32, i32, i32, dbl, i32, i32, i64, P, P]
    lib.orc_forward_terms.argtypes = [P, i32, i32, P, P, P]
    lib.orc_dp_fwd.argtypes = [P, P, P, i32, i32, i32, P, P, P]
    lib.orc_carve_buffer.argtypes = [P, P, i32, i32, i32, i32, i32, i32, i32, i32, P, P, P]
    lib.orc_carve.argtypes = [P, i32, i32, i32, i32, i32, i32, i32, i32, dbl, i32, i32, i32, P, P,
                              P, P]
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc):
    if rc != 0:
        raise RuntimeError(f"oracle error {rc}")


def luma(rgb: np.ndarray) -> np.ndarray:
    """Integer BT.601 luma of an [H,W,3] uint8 frame (Sec. 3.3 energy input)."""
    rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
    H, W = rgb.shape[:2]
    Y = np.empty((H, W), np.uint8)
    _check(_load().orc_luma(_ptr(rgb), H, W, _ptr(Y)))
    return Y


def sobel(Y: np.ndarray) -> np.ndarray:
    """|Gx|+|Gy| Sobel gradient with replicate border (Sec. 3.3)."""
    Y = np.ascontiguousarray(Y, dtype=np.uint8)
    H, W = Y.shape
    G = np.empty((H, W), np.int32)
    _check(_load().orc_sobel(_ptr(Y), H, W, _ptr(G)))
    return G


def motion(frames: np.ndarray) -> np.ndarray:
    """D_t = |Y_t - Y_{t-1}|, D_0 = 0 (Sec. 3.3).  frames [T,H,W,3]."""
    frames = np.ascontiguousarray(frames, dtype=np.uint8)
    T, H, W = frames.shape[:3]
    D = np.empty((T, H, W), np.uint8)
    _check(_load().orc_motion(_ptr(frames), T, H, W, _ptr(D)))
    return D


def energy(frames: np.ndarray, wg: int = 1, wm: int = 2) -> np.ndarray:
    """e_t = wg*Sobel(Y_t) + wm*D_t for every frame (Sec. 3.3).  [T,H,W] int32."""
    frames = np.ascontiguousarray(frames, dtype=np.uint8)
    T, H, W = frames.shape[:3]
    e = np.empty((T, H, W), np.int32)
    _check(_load().orc_energy(_ptr(frames), T, H, W, wg, wm, _ptr(e)))
    return e


def dp(E: np.ndarray):
    """Eq. 4 with parental labels: returns (CE int64, labels int32, dir uint8)."""
    E = np.ascontiguousarray(E, dtype=np.int32)
    H, W = E.shape
    CE = np.empty((H, W), np.int64)
    L = np.empty((H, W), np.int32)
    d = np.empty((H, W), np.uint8)
    _check(_load().orc_dp(_ptr(E), H, W, _ptr(CE), _ptr(L), _ptr(d)))
    return CE, L, d


def forward_terms(Y: np.ndarray):
    """Forward terms of one luma frame [H,W] (R14, after the forward energy of
    the related work, Sec. 2): (CU, A, B) int32, the luma differences a seam
    creates in its own row (CU), and between rows i-1 and i when it arrives
    from the upper left (A) or upper right (B)."""
    Y = np.ascontiguousarray(Y, dtype=np.uint8)
    H, W = Y.shape
    CU, A, B = (np.empty((H, W), np.int32) for _ in range(3))
    _check(_load().orc_forward_terms(_ptr(Y), H, W, _ptr(CU), _ptr(A), _ptr(B)))
    return CU, A, B


def dp_fwd(E: np.ndarray, A: np.ndarray, B: np.ndarray, wf: int):
    """Eq. 4 with parental labels where the diagonal moves cost wf*A (from the
    upper left) and wf*B (from the upper right) extra (R14).  E holds the
    per-pixel part.  Returns (CE int64, labels int32, dir uint8)."""
    E = np.ascontiguousarray(E, dtype=np.int32)
    A = np.ascontiguousarray(A, dtype=np.int32)
    B = np.ascontiguousarray(B, dtype=np.int32)
    H, W = E.shape
    CE = np.empty((H, W), np.int64)
    L = np.empty((H, W), np.int32)
    d = np.empty((H, W), np.uint8)
    _check(_load().orc_dp_fwd(_ptr(E), _ptr(A), _ptr(B), wf, H, W, _ptr(CE), _ptr(L), _ptr(d)))
    return CE, L, d


def select(ce_last: np.ndarray, lab_last: np.ndarray, cap: int) -> np.ndarray:
    """Eq. 6 per-parent argmin, then the `cap` lowest by (CE, column)."""
    ce_last = np.ascontiguousarray(ce_last, dtype=np.int64)
    lab_last = np.ascontiguousarray(lab_last, dtype=np.int32)
    W = ce_last.shape[0]
    cols = np.empty(max(W, 1), np.int32)
    n = _load().orc_select(_ptr(ce_last), _ptr(lab_last), W, cap, _ptr(cols))
    if n < 0:
        raise RuntimeError(f"oracle error {-n}")
    return cols[:n].copy()


def backtrack(d: np.ndarray, end_col: int) -> np.ndarray:
    """Follow the recorded indicators up from (H-1, end_col) (Sec. 3.1)."""
    d = np.ascontiguousarray(d, dtype=np.uint8)
    H, W = d.shape
    path = np.empty(H, np.int32)
    _check(_load().orc_backtrack(_ptr(d), H, W, end_col, _ptr(path)))
    return path


def isqrt(x: int) -> int:
    return int(_load().orc_isqrt(x))


def asde_sum(e: np.ndarray) -> int:
    """A = sum_ij floor(256*sqrt(n*S2 - S1^2)) over n maps [n,H,W] (Eq. 7-8)."""
    e = np.ascontiguousarray(e, dtype=np.int32)
    n, H, W = e.shape
    out = np.zeros(1, np.int64)
    _check(_load().orc_asde_sum(_ptr(e), n, H, W, _ptr(out)))
    return int(out[0])


def threshold(n: int, M: int, H: int, W: int, alpha: float = ALPHA) -> float:
    """256*alpha*M*sqrt(n-1)*H*W, the scaled phi(n) of Eq. 9."""
    return float(_load().orc_threshold(n, M, H, W, alpha))


def exceeds(A: int, n: int, M: int, H: int, W: int, alpha: float = ALPHA) -> bool:
    return bool(_load().orc_exceeds(A, n, M, H, W, alpha))


def scan(e: np.ndarray, alpha: float = ALPHA, t_max: int = T_MAX, maxval_mode: int = 0,
         maxval_theory: int = 0) -> np.ndarray:
    """Buffer boundaries of the dynamic spatiotemporal buffer (Sec. 3.2).

    Returns starts (int32, length n_buffers+1, last entry T)."""
    e = np.ascontiguousarray(e, dtype=np.int32)
    T, H, W = e.shape
    starts = np.empty(T + 1, np.int32)
    nb = np.zeros(1, np.int32)
    _check(_load().orc_scan(_ptr(e), T, H, W, alpha, t_max, maxval_mode, maxval_theory,
                            _ptr(starts), _ptr(nb)))
    return starts[: nb[0] + 1].copy()


def carve_buffer(frames: np.ndarray, D: np.ndarray, target: int, k: int, wg: int = 1,
                 wm: int = 2, wf: int = 0):
    """Carve one fixed buffer (Sec. 3.1/3.2; forward terms of weight wf, R14).
    Returns (out, seams, k_eff list)."""
    frames = np.ascontiguousarray(frames, dtype=np.uint8)
    D = np.ascontiguousarray(D, dtype=np.uint8)
    Tb, H, W0 = frames.shape[:3]
    out = np.empty((Tb, H, target, 3), np.uint8)
    seams = np.empty((max(W0 - target, 1), H), np.int16)
    keff = np.zeros(max(W0 - target, 1), np.int32)
    n = _load().orc_carve_buffer(_ptr(frames), _ptr(D), Tb, H, W0, target, k, wg, wm, wf,
                                 _ptr(out),
                                 _ptr(seams), _ptr(keff))
    if n < 0:
        raise RuntimeError(f"oracle error {-n}")
    return out, seams[: W0 - target].copy(), keff[:n].copy()


def carve(frames: np.ndarray, target: int, k: int, wg: int = 1, wm: int = 2,
          alpha: float = ALPHA, t_max: int = T_MAX, use_buffer: bool = True,
          maxval_mode: int = 0, wf: int = 0):
    """Whole clip: energy, buffer scan, per-buffer carving (with forward
    terms of weight wf in the seam cost when wf > 0, R14).

    Returns (out [T,H,target,3], starts [n_buffers+1], seams [n_buffers, W0-target, H])."""
    frames = np.ascontiguousarray(frames, dtype=np.uint8)
    T, H, W0 = frames.shape[:3]
    out = np.empty((T, H, target, 3), np.uint8)
    starts = np.empty(T + 1, np.int32)
    nb = np.zeros(1, np.int32)
    seams = np.empty((T, max(W0 - target, 1), H), np.int16)
    _check(_load().orc_carve(_ptr(frames), T, H, W0, target, k, wg, wm, wf, alpha, t_max,
                             int(use_buffer), maxval_mode, _ptr(out), _ptr(starts), _ptr(nb),
                             _ptr(seams)))
    n = int(nb[0])
    return out, starts[: n + 1].copy(), seams[:n, : W0 - target].copy()


def carve_job(frames: np.ndarray, target_W: int, target_H: int, k: int, wg: int = 1,
              wm: int = 2, alpha: float = ALPHA, t_max: int = T_MAX, use_buffer: bool = True,
              maxval_mode: int = 0, wf: int = 0):
    """A retarget job to target_H x target_W.  Seams are vertical or horizontal
    (Sec. 2).  The width is carved first with vertical seams (``carve``).  The
    height is then carved as vertical seams of the transposed result, with its
    own buffer scan, and transposed back.

    Returns (out [T,target_H,target_W,3], starts of the first pass)."""
    frames = np.ascontiguousarray(frames, dtype=np.uint8)
    T, H, W = frames.shape[:3]
    out, starts = frames, None
    kw = dict(wg=wg, wm=wm, alpha=alpha, t_max=t_max, use_buffer=use_buffer,
              maxval_mode=maxval_mode, wf=wf)
    if target_W < W:
        out, starts, _ = carve(out, target_W, k, **kw)
    if target_H < H:
        tr = np.ascontiguousarray(out.transpose(0, 2, 1, 3))
        o2, s2, _ = carve(tr, target_H, k, **kw)
        if starts is None:
            starts = s2
        out = np.ascontiguousarray(o2.transpose(0, 2, 1, 3))
    if starts is None:
        starts = np.array([0, T], np.int32)
    return out, starts


def blend_sharpness(frames: np.ndarray, window: int = 4) -> tuple[int, int]:
    """A numeric stand-in for Fig. 9 (Sec. 4): on a nearly static video, a
    blend of consecutive retargeted frames stays sharp when the same seams are
    removed from them and blurs when content moves between frames.

    For every run of `window` consecutive frames t .. t+window-1 (t = 0 ..
    T-window), the blend B is the sum of their integer BT.601 luma maps.  The
    numerator adds up the L1 Sobel magnitude |Gx| + |Gy| (3x3, replicate
    border) of B, and the denominator the same magnitude of each frame of the
    run.  Sobel is linear, so num <= den, with equality when the frames'
    gradients agree everywhere; num / den is the blend's sharpness.
    Returns (num, den) as exact integers."""
    frames = np.ascontiguousarray(frames, dtype=np.uint8)
    T = frames.shape[0]
    if T < window or window < 1:
        return 0, 0
    Y = np.stack([luma(f) for f in frames]).astype(np.int64)

    def mag(img):
        p = np.pad(img, 1, mode="edge")
        gx = (p[:-2, 2:] + 2 * p[1:-1, 2:] + p[2:, 2:]) - (p[:-2, :-2] + 2 * p[1:-1, :-2] + p[2:, :-2])
        gy = (p[2:, :-2] + 2 * p[2:, 1:-1] + p[2:, 2:]) - (p[:-2, :-2] + 2 * p[:-2, 1:-1] + p[:-2, 2:])
        return int(np.abs(gx).sum() + np.abs(gy).sum())

    per_frame = [mag(Y[t]) for t in range(T)]
    num = den = 0
    for t in range(T - window + 1):
        num += mag(Y[t:t + window].sum(axis=0))
        den += sum(per_frame[t:t + window])
    return num, den


def enlarge(frames: np.ndarray, target: int, k: int, wg: int = 1, wm: int = 2,
            alpha: float = ALPHA, t_max: int = T_MAX, use_buffer: bool = True,
            maxval_mode: int = 0, wf: int = 0):
    """Widen a clip by seam insertion (Sec. 2 retargets in both directions;
    the insertion rule is Avidan & Shamir's).  To add m = target - W columns,
    the clip is carved to W - m by SCPL (``carve``); the m seams removed from
    each spatiotemporal buffer, in original columns, are the ones inserted
    into every frame of that buffer.  Each row emits its original pixels in
    order and, after each seam pixel x, a new pixel that is the rounded mean
    (a + b + 1) >> 1, per channel, of pixel x and pixel x+1 (x itself at the
    last column).  m must be in [0, W-2].

    Returns (out [T,H,target,3], starts of the buffers)."""
    frames = np.ascontiguousarray(frames, dtype=np.uint8)
    T, H, W = frames.shape[:3]
    m = target - W
    if m < 0 or m > W - 2:
        raise ValueError("target must be in [W, 2W-2]")
    if m == 0:
        return frames.copy(), np.array([0, T], np.int32)
    _, starts, seams = carve(frames, W - m, k, wg=wg, wm=wm, alpha=alpha, t_max=t_max,
                             use_buffer=use_buffer, maxval_mode=maxval_mode, wf=wf)
    out = np.empty((T, H, target, 3), np.uint8)
    for b in range(len(starts) - 1):
        t0, t1 = int(starts[b]), int(starts[b + 1])
        for i in range(H):
            cols = set(int(c) for c in seams[b, :, i])
            left, right = [], []
            for x in range(W):
                left.append(x)
                right.append(x)
                if x in cols:
                    left.append(x)
                    right.append(min(x + 1, W - 1))
            a = frames[t0:t1, i, left].astype(np.int32)
            c = frames[t0:t1, i, right].astype(np.int32)
            out[t0:t1, i] = ((a + c + 1) >> 1).astype(np.uint8)
    return out, starts


def enlarge_job(frames: np.ndarray, target_W: int, target_H: int, k: int, wg: int = 1,
                wm: int = 2, alpha: float = ALPHA, t_max: int = T_MAX, use_buffer: bool = True,
                maxval_mode: int = 0, wf: int = 0):
    """Enlarge a clip to target_H x target_W (R12 in both directions; Sec. 2
    retargets along either axis).  The width grows first (``enlarge``); the
    height then grows as the width of the transposed result, its horizontal
    seams being the vertical seams of the transposed frames (R10), and the
    result is transposed back.  Each target lies in [size, 2*size - 2].

    Returns out [T,target_H,target_W,3]."""
    frames = np.ascontiguousarray(frames, dtype=np.uint8)
    T, H, W = frames.shape[:3]
    kw = dict(wg=wg, wm=wm, alpha=alpha, t_max=t_max, use_buffer=use_buffer,
              maxval_mode=maxval_mode, wf=wf)
    out = frames
    if target_W > W:
        out, _ = enlarge(out, target_W, k, **kw)
    if target_H > H:
        tr = np.ascontiguousarray(out.transpose(0, 2, 1, 3))
        o2, _ = enlarge(tr, target_H, k, **kw)
        out = np.ascontiguousarray(o2.transpose(0, 2, 1, 3))
    return out.copy() if out is frames else out
