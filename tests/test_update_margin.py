"""The partial energy update recomputes only the pixels within one old column of
a removed pixel in rows i-1, i and i+1 (Sec. 3.1 seams move at most one column a
row).  This checks that claim on random removals, independently of the oracle
and of the CUDA path: every other pixel keeps its 3x3 Sobel gradient and its
three forward terms, and a narrower margin would miss changes."""
from __future__ import annotations

import numpy as np


def _sobel(Y: np.ndarray) -> np.ndarray:
    P = np.pad(Y.astype(np.int64), 1, mode="edge")
    gx = (P[:-2, 2:] + 2 * P[1:-1, 2:] + P[2:, 2:]) - (P[:-2, :-2] + 2 * P[1:-1, :-2] + P[2:, :-2])
    gy = (P[2:, :-2] + 2 * P[2:, 1:-1] + P[2:, 2:]) - (P[:-2, :-2] + 2 * P[:-2, 1:-1] + P[:-2, 2:])
    return np.abs(gx) + np.abs(gy)


def _forward(Y: np.ndarray):
    """Row term (0 in the border columns) and the two diagonal terms, from
    clamped neighbours."""
    Yi = Y.astype(np.int64)
    L = np.concatenate([Yi[:, :1], Yi[:, :-1]], 1)
    R = np.concatenate([Yi[:, 1:], Yi[:, -1:]], 1)
    U = np.concatenate([Yi[:1], Yi[:-1]], 0)
    CU = np.abs(R - L)
    CU[:, 0] = 0
    CU[:, -1] = 0
    return CU, np.abs(U - L), np.abs(U - R)


def _random_seams(rng, H: int, W: int, k: int) -> np.ndarray:
    """k disjoint, non-crossing, 8-connected seams: [H, k] ascending columns."""
    while True:
        S = np.zeros((H, k), np.int64)
        S[H - 1] = np.sort(rng.choice(W, k, replace=False))
        ok = True
        for i in range(H - 2, -1, -1):
            nxt = np.clip(S[i + 1] + rng.integers(-1, 2, k), 0, W - 1)
            for s in range(1, k):
                nxt[s] = max(nxt[s], nxt[s - 1] + 1)
            if nxt[-1] > W - 1 or (np.abs(nxt - S[i + 1]) > 1).any():
                ok = False
                break
            S[i] = nxt
        if ok:
            return S


def _count(margin: int, trials: int, seed: int):
    rng = np.random.default_rng(seed)
    kept = changed_outside = 0
    for _ in range(trials):
        H, W = int(rng.integers(1, 9)), int(rng.integers(4, 40))
        k = int(rng.integers(1, min(W - 2, 8) + 1))
        Y = rng.integers(0, 256, (H, W)).astype(np.uint8)
        S = _random_seams(rng, H, W, k)
        keep = np.ones((H, W), bool)
        keep[np.arange(H)[:, None], S] = False
        Yn = Y[keep].reshape(H, W - k)
        orig = np.tile(np.arange(W), (H, 1))[keep].reshape(H, W - k)
        old = (_sobel(Y),) + _forward(Y)
        new = (_sobel(Yn),) + _forward(Yn)
        for i in range(H):
            near = set()
            for a in (-1, 0, 1):
                near |= set(S[min(max(i + a, 0), H - 1)].tolist())
            for p in range(W - k):
                x = int(orig[i, p])
                if any(abs(x - c) <= margin for c in near):
                    continue
                kept += 1
                if any(o[i, x] != n[i, p] for o, n in zip(old, new)):
                    changed_outside += 1
    return kept, changed_outside


def test_one_column_margin_is_exact():
    kept, changed = _count(1, 400, seed=0x3A7)
    assert kept > 10000 and changed == 0


def test_a_narrower_margin_misses_changes():
    kept, changed = _count(0, 100, seed=0x3A8)
    assert changed > 0
