"""scpl_seams_noalloc -- the entry point for callers that may not allocate
device memory (graph capture, real-time loops, applications with their own
fixed memory pool) -- must give exactly what scpl_seams gives, call after
call, although every call reuses the same fixed scratch array.

This file is named to be collected last, so that a failure here comes after
every other test has run."""
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


def _seams_with_workspace(lib, E, k):
    h = lib.scpl_create()
    cols = torch.full((k, E.shape[0]), -1, dtype=torch.int16, device="cuda")
    ke = lib.scpl_seams(h, E, k, cols)
    torch.cuda.synchronize()
    lib.scpl_destroy(h)
    return ke, cols.cpu().numpy()[:ke]


def _seams_without_allocation(lib, E, k):
    cols = torch.full((k, E.shape[0]), -1, dtype=torch.int16, device="cuda")
    ke = lib.scpl_seams_noalloc(E, k, cols)
    return ke, cols.cpu().numpy()[:ke]


def test_two_calls_in_a_row_match_scpl_seams(lib):
    r = np.random.default_rng(1234)
    # a large map, then a small ragged one: the second call must not see any
    # state the first one left in the shared scratch
    cases = [((1080, 1920), 2550, 32), ((37, 301), 3, 7)]
    for (H, W), vmax, k in cases:
        E = torch.from_numpy(r.integers(0, vmax + 1, (H, W)).astype(np.int32)).cuda()
        ref_k, ref = _seams_with_workspace(lib, E, k)
        got_k, got = _seams_without_allocation(lib, E, k)
        assert got_k == ref_k
        assert np.array_equal(got, ref)                # tolerance 0: integer columns


def test_same_map_twice(lib):
    r = np.random.default_rng(99)
    E = torch.from_numpy(r.integers(0, 50, (200, 700)).astype(np.int32)).cuda()
    first = _seams_without_allocation(lib, E, 16)
    second = _seams_without_allocation(lib, E, 16)
    assert first[0] == second[0] and np.array_equal(first[1], second[1])
    assert np.array_equal(first[1], _seams_with_workspace(lib, E, 16)[1])


def test_sizes_beyond_the_scratch_are_rejected(lib):
    cols = torch.zeros((4, 8), dtype=torch.int16, device="cuda")
    wide = torch.zeros((8, 4097), dtype=torch.int32, device="cuda")
    with pytest.raises(lib.SCPLError) as ei:
        lib.scpl_seams_noalloc(wide, 4, cols)
    assert ei.value.status == lib.SCPL_EINVAL
    big_k = torch.zeros((8, 100), dtype=torch.int32, device="cuda")
    cols65 = torch.zeros((65, 8), dtype=torch.int16, device="cuda")
    with pytest.raises(lib.SCPLError) as ei:
        lib.scpl_seams_noalloc(big_k, 65, cols65)
    assert ei.value.status == lib.SCPL_EINVAL
