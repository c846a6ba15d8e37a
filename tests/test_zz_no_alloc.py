"""scpl_seams_noalloc -- the entry point for callers that may not allocate
device memory (a real-time frame loop that cannot take cudaMalloc's
device-wide synchronisation, an application that hands out all device memory
from its own fixed pool) -- must give exactly what scpl_seams gives, call
after call, although every call reuses the same fixed scratch array, and must
take no device memory of its own.

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
    # H * W one row of 1024 beyond 2^21
    tall = torch.zeros((2049, 1024), dtype=torch.int32, device="cuda")
    cols_t = torch.zeros((4, 2049), dtype=torch.int16, device="cuda")
    with pytest.raises(lib.SCPLError) as ei:
        lib.scpl_seams_noalloc(tall, 4, cols_t)
    assert ei.value.status == lib.SCPL_EINVAL
    # more rows than the removal lists index, although H * W fits
    high = torch.zeros((65536, 1), dtype=torch.int32, device="cuda")
    cols_h = torch.zeros((1, 65536), dtype=torch.int16, device="cuda")
    with pytest.raises(lib.SCPLError) as ei:
        lib.scpl_seams_noalloc(high, 1, cols_h)
    assert ei.value.status == lib.SCPL_EINVAL


def test_calls_take_no_device_memory(lib):
    """After one call has loaded the kernels, further calls leave the free
    device memory unchanged: nothing is allocated, not even temporarily kept."""
    r = np.random.default_rng(7)
    E = torch.from_numpy(r.integers(0, 2551, (1080, 1920)).astype(np.int32)).cuda()
    cols = torch.full((32, 1080), -1, dtype=torch.int16, device="cuda")
    lib.scpl_seams_noalloc(E, 32, cols)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(8):
        lib.scpl_seams_noalloc(E, 32, cols)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_on_a_side_stream(lib):
    """A call on a stream other than the default one gives the same seams."""
    r = np.random.default_rng(11)
    E = torch.from_numpy(r.integers(0, 300, (333, 1500)).astype(np.int32)).cuda()
    ref_k, ref = _seams_with_workspace(lib, E, 24)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        cols = torch.full((24, 333), -1, dtype=torch.int16, device="cuda")
        ke = lib.scpl_seams_noalloc(E, 24, cols, stream=side)
    side.synchronize()
    assert ke == ref_k
    assert np.array_equal(cols.cpu().numpy()[:ke], ref)
