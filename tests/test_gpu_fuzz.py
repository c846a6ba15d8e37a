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
