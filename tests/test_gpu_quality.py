"""Blend sharpness on the GPU (scpl_blend_sharpness): exact against the oracle,
and the paper's Fig. 9 observation measured: on a nearly static clip, frames
carved by SCPL with the spatiotemporal buffer blend into a sharper image than
frames carved one by one with classic seam carving."""
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


@pytest.mark.parametrize("T,H,W,window,seed", [(6, 9, 11, 4, 1), (10, 33, 70, 1, 2),
                                               (5, 17, 300, 5, 3), (7, 40, 257, 2, 4),
                                               (3, 8, 8, 4, 5), (4, 1, 1, 4, 6)])
def test_blend_sharpness_matches_oracle(orc, lib, T, H, W, window, seed):
    f = np.random.default_rng(seed).integers(0, 256, (T, H, W, 3), dtype=np.uint8)
    h = lib.scpl_create()
    got = lib.scpl_blend_sharpness(h, torch.from_numpy(f).cuda(), window)
    lib.scpl_destroy(h)
    assert got == orc.blend_sharpness(f, window)


def test_static_clip_scpl_blends_sharper_than_raw(orc, lib):
    from paper_1903_03180_gb300 import synth
    f = synth.clip(24, 90, 160, seed=71, pan=0, n_ellipses=0, noise=4)
    x = torch.from_numpy(f).cuda()
    scpl_r = lib.Retargeter(wg=1, wm=2)
    raw_r = lib.Retargeter(wg=1, wm=2, use_buffer=False)
    o_scpl, starts, _ = scpl_r.carve(x, 120, 8)
    o_raw, _, _ = raw_r.carve(x, 120, 1)
    h = scpl_r.h
    s = lib.scpl_blend_sharpness(h, o_scpl, 4)
    r = lib.scpl_blend_sharpness(h, o_raw, 4)
    torch.cuda.synchronize()
    scpl_r.close()
    raw_r.close()
    assert s == orc.blend_sharpness(o_scpl.cpu().numpy(), 4)
    assert r == orc.blend_sharpness(o_raw.cpu().numpy(), 4)
    assert len(starts) - 1 < 24          # SCPL found multi-frame buffers
    assert s[0] / s[1] > r[0] / r[1]     # and its blends are sharper
