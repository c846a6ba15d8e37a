"""Independent restatements used to pin the oracle (test-side only).

* ``sobel_scipy``: the Sobel L1 gradient through scipy.ndimage's correlate with
  the 'nearest' (replicate) border -- a library routine, not the oracle's loop.
* ``classic_seam_carve``: textbook Avidan-Shamir backward-energy seam carving,
  vectorised with numpy (one global-minimum seam per iteration, np.argmin's
  first-occurrence rule for ties).
* ``all_seams``: brute-force enumeration of every 8-connected vertical seam of a
  tiny energy map.
"""
from __future__ import annotations

import itertools

import numpy as np
from scipy import ndimage

SOBEL_X = np.array([[-1, 0, 1], [-2, 0, 2], [-1, 0, 1]], np.int64)
SOBEL_Y = SOBEL_X.T.copy()


def luma_bt601_float(rgb: np.ndarray) -> np.ndarray:
    rgb = rgb.astype(np.float64)
    return 0.299 * rgb[..., 0] + 0.587 * rgb[..., 1] + 0.114 * rgb[..., 2]


def sobel_scipy(Y: np.ndarray) -> np.ndarray:
    Y = Y.astype(np.int64)
    gx = ndimage.correlate(Y, SOBEL_X, mode="nearest")
    gy = ndimage.correlate(Y, SOBEL_Y, mode="nearest")
    return (np.abs(gx) + np.abs(gy)).astype(np.int64)


def energy_scipy(frames: np.ndarray, wg: int, wm: int, luma_fn) -> np.ndarray:
    """e_t = wg*|Sobel| + wm*|Y_t - Y_{t-1}| with the library Sobel."""
    Y = np.stack([luma_fn(f).astype(np.int64) for f in frames])
    D = np.zeros_like(Y)
    D[1:] = np.abs(Y[1:] - Y[:-1])
    return np.stack([wg * sobel_scipy(Y[t]) + wm * D[t] for t in range(len(Y))])


def classic_dp(E: np.ndarray):
    """Textbook cumulative energy M and backtrack pointers (absolute columns)."""
    H, W = E.shape
    M = E.astype(np.int64).copy()
    back = np.zeros((H, W), np.int64)
    cols = np.arange(W)
    inf = np.iinfo(np.int64).max // 4
    for i in range(1, H):
        prev = M[i - 1]
        left = np.concatenate([[inf], prev[:-1]])
        right = np.concatenate([prev[1:], [inf]])
        stack = np.stack([left, prev, right])
        idx = np.argmin(stack, axis=0)          # first occurrence: lowest column
        M[i] += stack[idx, cols]
        back[i] = cols + idx - 1
    return M, back


def classic_seam(E: np.ndarray) -> np.ndarray:
    M, back = classic_dp(E)
    H = E.shape[0]
    path = np.empty(H, np.int64)
    path[-1] = int(np.argmin(M[-1]))
    for i in range(H - 1, 0, -1):
        path[i - 1] = back[i, path[i]]
    return path


def classic_seam_carve(frame: np.ndarray, n_remove: int, energy_fn):
    """Remove n_remove seams one at a time (Avidan & Shamir).  energy_fn maps
    the current [H,W,3] frame to an [H,W] energy.  Returns (out, seams in
    original columns [n_remove, H])."""
    img = frame.copy()
    H, W = img.shape[:2]
    orig = np.tile(np.arange(W), (H, 1))
    seams = []
    for _ in range(n_remove):
        path = classic_seam(energy_fn(img))
        rows = np.arange(H)
        seams.append(orig[rows, path].copy())
        keep = np.ones(img.shape[:2], bool)
        keep[rows, path] = False
        Wn = img.shape[1] - 1
        img = img[keep].reshape(H, Wn, 3)
        orig = orig[keep].reshape(H, Wn)
    return img, np.array(seams, np.int64).reshape(n_remove, H)


def classic_horizontal_seam_carve(frame: np.ndarray, n_remove: int, energy_fn):
    """Horizontal seams written in their own orientation: the cumulative energy
    runs left to right over columns, M[i,j] = E[i,j] + min(M[i-1..i+1, j-1]),
    ties to the lowest row.  A seam has one pixel per column, and removing it
    moves the pixels below it up by one.  Returns the [H-n_remove, W, 3] frame."""
    img = frame.copy()
    for _ in range(n_remove):
        E = energy_fn(img).astype(np.int64)
        H, W = E.shape
        M = E.copy()
        back = np.zeros((H, W), np.int64)
        inf = np.iinfo(np.int64).max // 4
        for j in range(1, W):
            prev = M[:, j - 1]
            up = np.concatenate([[inf], prev[:-1]])
            down = np.concatenate([prev[1:], [inf]])
            stack = np.stack([up, prev, down])
            idx = np.argmin(stack, axis=0)
            M[:, j] += stack[idx, np.arange(H)]
            back[:, j] = np.arange(H) + idx - 1
        path = np.empty(W, np.int64)
        path[-1] = int(np.argmin(M[:, -1]))
        for j in range(W - 1, 0, -1):
            path[j - 1] = back[path[j], j]
        out = np.empty((H - 1, W, 3), img.dtype)
        for j in range(W):
            out[:, j] = np.delete(img[:, j], path[j], axis=0)
        img = out
    return img


def all_seams(H: int, W: int):
    """Every vertical 8-connected seam as a tuple of columns (row 0 .. H-1)."""
    for c0 in range(W):
        for steps in itertools.product((-1, 0, 1), repeat=H - 1):
            path = [c0]
            ok = True
            for s in steps:
                c = path[-1] + s
                if c < 0 or c >= W:
                    ok = False
                    break
                path.append(c)
            if ok:
                yield tuple(path)
