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


# ------------------------------------------------------------ seam insertion
@pytest.mark.parametrize("T,H,W,target,k,seed,cuts", [(6, 14, 20, 27, 4, 81, (3, 3)),
                                                      (5, 33, 70, 120, 8, 82, None),
                                                      (4, 19, 257, 400, 16, 83, (2, 2)),
                                                      (3, 40, 64, 100, 32, 84, None)])
def test_enlarge_matches_oracle(orc, lib, T, H, W, target, k, seed, cuts):
    from paper_1903_03180_gb300 import synth
    f = synth.clip(T, H, W, seed=seed, cuts=cuts)
    r = lib.Retargeter()
    out, starts = r.enlarge(torch.from_numpy(f).cuda(), target, k)
    torch.cuda.synchronize()
    r.close()
    ref, ref_starts = orc.enlarge(f, target, k)
    assert np.array_equal(starts, ref_starts)
    assert np.array_equal(out.cpu().numpy(), ref)


def test_enlarge_still_k1(orc, lib):
    from paper_1903_03180_gb300 import synth
    f = synth.still_frame(30, 50, seed=85)[None]
    r = lib.Retargeter(wg=1, wm=0, use_buffer=False)
    out, _ = r.enlarge(torch.from_numpy(f).cuda(), 61, 1)
    torch.cuda.synchronize()
    r.close()
    ref, _ = orc.enlarge(f, 61, 1, wm=0, use_buffer=False)
    assert np.array_equal(out.cpu().numpy(), ref)


def test_enlarge_identity_and_limits(lib):
    f = torch.randint(0, 256, (2, 6, 9, 3), dtype=torch.uint8, device="cuda")
    r = lib.Retargeter()
    out, starts = r.enlarge(f, 9, 4)
    assert torch.equal(out, f) and list(starts) == [0, 2]
    with pytest.raises(lib.SCPLError):
        r.enlarge(f, 17, 4)   # more than 2W-2
    with pytest.raises(lib.SCPLError):
        r.enlarge(f, 8, 4)    # narrower: use scpl_carve
    r.close()


# ------------------------------------------------ insertion along both axes
@pytest.mark.parametrize("T,H,W,tw,th,k,seed,cuts", [(5, 14, 20, 20, 23, 4, 91, (2, 3)),
                                                     (4, 12, 18, 23, 16, 3, 92, (2, 2)),
                                                     (3, 33, 40, 60, 50, 8, 93, None),
                                                     (2, 9, 300, 300, 13, 16, 94, None)])
def test_enlarge_job_matches_oracle(orc, lib, T, H, W, tw, th, k, seed, cuts):
    from paper_1903_03180_gb300 import synth
    f = synth.clip(T, H, W, seed=seed, cuts=cuts)
    r = lib.Retargeter()
    out = r.enlarge_job(torch.from_numpy(f).cuda(), tw, th, k)
    torch.cuda.synchronize()
    r.close()
    assert np.array_equal(out.cpu().numpy(), orc.enlarge_job(f, tw, th, k))


def test_enlarge_job_limits(lib):
    f = torch.randint(0, 256, (2, 6, 9, 3), dtype=torch.uint8, device="cuda")
    r = lib.Retargeter()
    assert torch.equal(r.enlarge_job(f, 9, 6, 4), f)
    with pytest.raises(lib.SCPLError):
        r.enlarge_job(f, 9, 11, 4)   # more than 2H-2
    with pytest.raises(lib.SCPLError):
        r.enlarge_job(f, 9, 5, 4)    # shorter: carve instead
    r.close()
