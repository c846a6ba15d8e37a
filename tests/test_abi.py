"""The C-ABI library builds, loads without a GPU and exports every symbol that
include/scpl.h declares; the binding declares exactly those symbols."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "scpl.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(scpl_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1903_03180_gb300 import build, scpl
    build.build()
    return scpl.load()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["scpl_create", "scpl_energy", "scpl_carve", "scpl_destroy", "scpl_scan",
                 "scpl_seams", "scpl_carve_host", "scpl_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_the_header(lib):
    from paper_1903_03180_gb300 import scpl
    assert sorted(scpl.SIGNATURES) == _declared()


def test_default_params_host_only(lib):
    from paper_1903_03180_gb300 import scpl
    p = scpl.scpl_default_params()
    assert (p.alpha, p.wg, p.wm, p.t_max, p.use_buffer, p.maxval_mode, p.wf) == \
        (0.2, 1, 2, 128, 1, 0, 0)


def test_forward_params_are_checked_without_a_gpu(lib):
    """Forward terms: wf in [0, 255], and buffers of at most 256 frames, so a
    pixel's diagonal sums fit 16 bits; the check comes before any CUDA call."""
    import ctypes
    from paper_1903_03180_gb300 import scpl
    for wf, t_max, use_buffer in [(256, 128, 1), (-1, 128, 1), (1, 257, 1)]:
        p = scpl.scpl_default_params()
        p.wf, p.t_max, p.use_buffer = wf, t_max, use_buffer
        h = ctypes.c_void_p()
        assert lib.scpl_create(ctypes.byref(p), None, ctypes.byref(h)) == scpl.SCPL_EINVAL
        srv = ctypes.c_void_p()
        assert lib.scpl_server_create(ctypes.byref(p), 0, None, ctypes.byref(srv)) == \
            scpl.SCPL_EINVAL


def test_forward_footprint_adds_the_diagonal_planes(lib):
    """With forward terms a buffer's workspace holds two more 32-bit planes
    (the diagonal sums of both slots), padded rows as the energy planes."""
    from paper_1903_03180_gb300 import scpl
    j = scpl.Job()
    j.frames, j.out = 1, 1   # never dereferenced
    j.T, j.H, j.W, j.target_W, j.target_H, j.k = 16, 270, 481, 400, 270, 8
    p = scpl.scpl_default_params()
    base = scpl.scpl_job_footprint(p, j)
    p.wf = 3
    pitch = (481 + 31) // 32 * 32
    assert scpl.scpl_job_footprint(p, j) - base == 2 * 270 * pitch * 4


def test_null_handle_is_rejected_without_a_gpu(lib):
    from paper_1903_03180_gb300 import scpl
    assert lib.scpl_energy(None, None, 1, 1, 1, None) == scpl.SCPL_EINVAL
    assert lib.scpl_carve(None, None, 1, 1, 4, 2, 1, None, None, None, None) == scpl.SCPL_EINVAL
    assert lib.scpl_create(None, None, None) == scpl.SCPL_EINVAL
    lib.scpl_destroy(None)
    assert lib.scpl_last_error(None) == b"null handle"


def test_missing_library_fails_loudly(tmp_path):
    from paper_1903_03180_gb300 import scpl
    with pytest.raises(OSError):
        scpl.load(str(tmp_path / "libscpl.so"))


def test_job_footprint_host_only(lib):
    """Admission's footprint is host arithmetic (no GPU): the luma and motion
    maps plus the frame-minor luma copy at least, the host copies on top for a
    host job, and 0 for an invalid job."""
    from paper_1903_03180_gb300 import scpl
    j = scpl.Job()
    j.frames, j.out = 1, 1   # never dereferenced
    j.T, j.H, j.W, j.target_W, j.target_H, j.k = 32, 1080, 1920, 1440, 1080, 32
    fp = scpl.scpl_job_footprint(None, j)
    assert fp >= 3 * 32 * 1080 * 1920
    j.on_host = 1
    assert scpl.scpl_job_footprint(None, j) == fp + 32 * 1080 * (1920 + 1440) * 3
    assert scpl.scpl_job_footprint_per_buffer(j) > 1080 * 1920 * 16
    j.target_H = 823   # both dimensions: a second pass on the transposed clip
    assert scpl.scpl_job_footprint(None, j) > fp
    j.target_W = 1921
    assert scpl.scpl_job_footprint(None, j) == 0


def test_tuning_table_host_only(lib):
    from paper_1903_03180_gb300 import scpl
    scpl.scpl_tuning_clear()
    assert scpl.scpl_tuning_get(10, 20) is None
    scpl.scpl_tuning_set(10, 20, 16, 2)
    assert scpl.scpl_tuning_get(10, 20)["dpc_halo"] == 16
    with pytest.raises(scpl.SCPLError):
        scpl.scpl_tuning_set(10, 20, 8, 2)
    with pytest.raises(scpl.SCPLError):
        scpl.scpl_tuning_set(10, 20, 32, 3)
    with pytest.raises(scpl.SCPLError):
        scpl.scpl_tuning_set(10, 20, 32, 2, 4, 2)   # 2 columns a lane needs halo 16
    scpl.scpl_tuning_set(10, 20, 16, 2, 8, 2)
    assert scpl.scpl_tuning_get(10, 20)["dpc_lane_cols"] == 2
    scpl.scpl_tuning_clear()
    assert scpl.scpl_tuning_get(10, 20) is None


def test_tuning_cache_round_trip_host_only(lib, tmp_path):
    """The tuning table lists its entries in (H, W) order, and a saved table
    restores the same choices in a cleared one (a tuning cache)."""
    from paper_1903_03180_gb300 import scpl
    scpl.scpl_tuning_clear()
    scpl.scpl_tuning_set(1080, 1920, 16, 4, 4, 2)
    scpl.scpl_tuning_set(360, 640, 32, 2, 8, 4)
    scpl.scpl_tuning_set(720, 1280, 0, 1)
    got = [(t["H"], t["W"]) for t in scpl.scpl_tuning_list()]
    assert got == [(360, 640), (720, 1280), (1080, 1920)]
    path = tmp_path / "tuning.json"
    scpl.save_tuning(str(path))
    before = scpl.scpl_tuning_list()
    scpl.scpl_tuning_clear()
    assert scpl.scpl_tuning_list() == []
    assert scpl.load_tuning(str(path)) == 3
    after = scpl.scpl_tuning_list()
    keys = ("H", "W", "dpc_halo", "dpc_warps", "dpc_lane_cols", "update_rows")
    assert [{k: t[k] for k in keys} for t in after] == [{k: t[k] for k in keys} for t in before]
    scpl.scpl_tuning_clear()


def test_forward_terms_enter_the_overflow_rule(lib):
    """A column's cumulative cost must stay below 2^31 with the forward terms
    too: each row adds at most the buffer's summed energy plus wf times a row
    term and a diagonal term (255 each a frame).  At 1080 rows and 128-frame
    buffers that holds for wf = 0 but not for wf = 255, and admission (host
    arithmetic, no GPU) refuses the job."""
    from paper_1903_03180_gb300 import scpl
    j = scpl.Job()
    j.frames, j.out = 1, 1   # never dereferenced
    j.T, j.H, j.W, j.target_W, j.target_H, j.k = 128, 1080, 1920, 1440, 1080, 32
    p = scpl.scpl_default_params()
    assert scpl.scpl_job_footprint(p, j) > 0
    em, tb = 255 * (8 * p.wg + p.wm), 128
    p.wf = 255
    assert (em * tb + 2 * 255 * 255 * tb) * 1080 >= 2 ** 31
    assert scpl.scpl_job_footprint(p, j) == 0
    p.wf = 1
    assert (em * tb + 2 * 255 * 1 * tb) * 1080 < 2 ** 31
    assert scpl.scpl_job_footprint(p, j) > 0
