"""Seeded synthetic video for SCPL retargeting workloads.

Pure input generation: nothing here computes any part of the retargeting
method.  The paper's own clips are not available, so these generators stand in
for them with the same structure -- natural-looking frames with textured
regions, objects in motion, a panning camera and hard scene cuts -- at the
resolutions the workloads name.  All randomness comes from numpy's PCG64 seeded
with the given seed, so the same call returns the same bytes every time.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed & 0xFFFFFFFFFFFFFFFF))


def still_frame(H: int = 240, W: int = 320, seed: int = 1, n_rects: int = 12,
                noise: int = 8) -> np.ndarray:
    """One [H,W,3] uint8 frame: diagonal colour gradients, textured rectangles
    with stripe/checker patterns (period 2-8), uniform noise of +-`noise`."""
    r = _rng(seed)
    y, x = np.mgrid[0:H, 0:W]
    img = np.empty((H, W, 3), np.int16)
    img[..., 0] = 255 * (x + y) // max(W + H - 2, 1)
    img[..., 1] = 255 * x // max(W - 1, 1)
    img[..., 2] = 255 * y // max(H - 1, 1)
    for _ in range(n_rects):
        h = int(r.integers(16, 97))
        w = int(r.integers(16, 97))
        y0 = int(r.integers(-h // 2, max(H - h // 2, 1)))
        x0 = int(r.integers(-w // 2, max(W - w // 2, 1)))
        period = int(r.integers(2, 9))
        kind = int(r.integers(0, 4))
        c0 = r.integers(0, 256, 3)
        c1 = r.integers(0, 256, 3)
        ys, ye = max(y0, 0), min(y0 + h, H)
        xs, xe = max(x0, 0), min(x0 + w, W)
        if ys >= ye or xs >= xe:
            continue
        yy, xx = np.mgrid[ys:ye, xs:xe]
        if kind == 0:
            m = (xx // period) % 2
        elif kind == 1:
            m = (yy // period) % 2
        elif kind == 2:
            m = ((xx + yy) // period) % 2
        else:
            m = ((xx // period) + (yy // period)) % 2
        img[ys:ye, xs:xe] = np.where(m[..., None] == 1, c1, c0)
    img += r.integers(-noise, noise + 1, size=(H, W, 3), dtype=np.int16)
    return np.clip(img, 0, 255).astype(np.uint8)


def _background(r: np.random.Generator, H: int, Wext: int, scale: float) -> np.ndarray:
    """Sum of three seeded stripe/checker layers, [H, Wext, 3] int16."""
    y, x = np.mgrid[0:H, 0:Wext]
    bg = np.zeros((H, Wext, 3), np.int16)
    bg += r.integers(30, 90, 3).astype(np.int16)
    for _ in range(3):
        period = max(int(r.integers(8, 65) * scale), 2)
        kind = int(r.integers(0, 3))
        amp = r.integers(10, 51, 3).astype(np.int16)
        if kind == 0:
            m = (x // period) % 2
        elif kind == 1:
            m = (y // period) % 2
        else:
            m = ((x // period) + (y // period)) % 2
        bg += m.astype(np.int16)[..., None] * amp
    return bg


class _Scene:
    def __init__(self, r: np.random.Generator, H: int, W: int, length: int, pan: int,
                 scale: float, n_ellipses: int):
        self.H, self.W, self.pan = H, W, pan
        self.bg = _background(r, H, W + pan * length + 1, scale)
        self.ell = []
        for _ in range(n_ellipses):
            ry = float(r.integers(12, 61)) * scale
            rx = float(r.integers(12, 61)) * scale
            cy = float(r.uniform(0, H))
            cx = float(r.uniform(0, W))
            vy = float(r.uniform(-6, 6)) * scale
            vx = float(r.uniform(-6, 6)) * scale
            col = r.integers(0, 256, 3).astype(np.int16)
            self.ell.append([cy, cx, vy, vx, ry, rx, col])

    def frame(self, t: int) -> np.ndarray:
        H, W = self.H, self.W
        off = self.pan * t
        img = self.bg[:, off:off + W].copy()
        for e in self.ell:
            cy, cx, vy, vx, ry, rx, col = e
            y0, y1 = max(int(cy - ry), 0), min(int(cy + ry) + 1, H)
            x0, x1 = max(int(cx - rx), 0), min(int(cx + rx) + 1, W)
            if y0 < y1 and x0 < x1:
                yy, xx = np.ogrid[y0:y1, x0:x1]
                m = ((yy - cy) / ry) ** 2 + ((xx - cx) / rx) ** 2 <= 1.0
                img[y0:y1, x0:x1][m] = col
            # advance with reflection at the borders
            cy += vy
            cx += vx
            if cy < 0 or cy >= H:
                vy = -vy
                cy = min(max(cy, 0.0), H - 1.0)
            if cx < 0 or cx >= W:
                vx = -vx
                cx = min(max(cx, 0.0), W - 1.0)
            e[0], e[1], e[2], e[3] = cy, cx, vy, vx
        return img


def clip(T: int, H: int, W: int, seed: int, pan: int = 2, cuts: tuple | None = None,
         noise: int = 4, n_ellipses: int = 5) -> np.ndarray:
    """[T,H,W,3] uint8 clip: a textured background panning `pan` px/frame,
    `n_ellipses` moving ellipses of random colour and velocity (reflected at
    the borders) and uniform noise of +-`noise`.  With `cuts=(lo, hi)` the clip
    is split into scenes of seeded length U[lo, hi] with a new background and
    new ellipses after every cut.  Sizes of textures and objects scale with
    H/360."""
    r = _rng(seed)
    scale = max(H / 360.0, 0.25)
    out = np.empty((T, H, W, 3), np.uint8)
    # one pool of noise, sliced at a seeded offset per frame
    pool = r.integers(-noise, noise + 1, size=(H + 7, W + 61, 3), dtype=np.int16)
    t = 0
    while t < T:
        length = T - t if cuts is None else int(r.integers(cuts[0], cuts[1] + 1))
        length = min(length, T - t)
        sc = _Scene(r, H, W, length, pan, scale, n_ellipses)
        for s in range(length):
            img = sc.frame(s)
            oy, ox = int(r.integers(0, 8)), int(r.integers(0, 62))
            img += pool[oy:oy + H, ox:ox + W]
            np.clip(img, 0, 255, out=img)
            out[t + s] = img.astype(np.uint8)
        t += length
    return out


# ---- the named workloads ---------------------------------------------------

SEED_BASE = 0x5C9


def workload_still_320x240(seed: int = SEED_BASE ^ 1) -> np.ndarray:
    """Single 320x240 frame; carve 32 seams with k=8, gradient energy only."""
    return still_frame(240, 320, seed)[None]


def workload_clip_640x360(seed: int = SEED_BASE ^ 2, T: int = 64) -> np.ndarray:
    """64-frame 640x360 panning clip with 5 moving ellipses."""
    return clip(T, 360, 640, seed)


def workload_clip_1080p(seed: int = SEED_BASE ^ 3, T: int = 300) -> np.ndarray:
    """300-frame 1920x1080 clip with hard scene cuts every 60-120 frames."""
    return clip(T, 1080, 1920, seed, cuts=(60, 120))


BATCH_SIZES = ((240, 426), (360, 640), (720, 1280), (1080, 1920))
BATCH_ASPECTS = ("1:1", "4:3", "21:9")


def batch_spec(n_clips: int = 256, T: int = 32, seed: int = SEED_BASE ^ 4):
    """The batched workload's job list, without frames: for clip c a dict with
    its size (H, W drawn uniformly from BATCH_SIZES), target aspect (uniform
    over 1:1, 4:3, 21:9), target size and k, and the seed of its frames.
    1:1 and 4:3 keep the height and cut the width to round(H * aspect); 21:9
    keeps the width and cuts the height to round(W * 9 / 21) (horizontal
    seams).  k = 16 up to 640 columns wide, 32 above."""
    r = _rng(seed)
    out = []
    for c in range(n_clips):
        H, W = BATCH_SIZES[int(r.integers(0, len(BATCH_SIZES)))]
        aspect = BATCH_ASPECTS[int(r.integers(0, len(BATCH_ASPECTS)))]
        if aspect == "21:9":
            tw, th = W, int(round(W * 9 / 21))
        else:
            num, den = (1, 1) if aspect == "1:1" else (4, 3)
            tw, th = int(round(H * num / den)), H
        out.append({"clip": c, "T": T, "H": H, "W": W, "aspect": aspect, "target_W": tw,
                    "target_H": th, "k": 16 if W <= 640 else 32,
                    "seed": (seed * 1000003 + c) & 0xFFFFFFFF})
    return out


def batch_clip(spec: dict) -> np.ndarray:
    """Frames of one clip of the batched workload (one scene, no cuts)."""
    return clip(spec["T"], spec["H"], spec["W"], spec["seed"])


SERVE_SIZES = ((360, 640, 16), (720, 1280, 32), (1080, 1920, 32), (2160, 3840, 64))


def serve_jobs(n_jobs: int = 20, seed: int = SEED_BASE ^ 5):
    """A fixed list of served retarget jobs at the serving workload's sizes,
    without frames: for job j its size (H, W, k drawn uniformly from
    SERVE_SIZES), its length T ~ U[16, 128], its target width (a width
    reduction ~ U[10 %, 40 %], rounded) and the seed of its frames."""
    r = _rng(seed)
    out = []
    for j in range(n_jobs):
        H, W, k = SERVE_SIZES[int(r.integers(0, len(SERVE_SIZES)))]
        T = int(r.integers(16, 129))
        red = float(r.uniform(0.10, 0.40))
        out.append({"job": j, "T": T, "H": H, "W": W, "target_W": W - int(round(W * red)),
                    "target_H": H, "k": k, "seed": (seed * 1000003 + j) & 0xFFFFFFFF})
    return out


def serve_clip(spec: dict) -> np.ndarray:
    """Frames of one served job: a clip with scene cuts every 40-90 frames."""
    return clip(spec["T"], spec["H"], spec["W"], spec["seed"], cuts=(40, 90))
