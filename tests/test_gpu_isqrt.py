"""The exact integer square root of the buffer decision (Sec. 3.2, Eq. 7-8),
checked at its edges against Python's math.isqrt (tolerance 0).

The scan adds floor(sqrt(65536 Q)) per pixel, Q = n S2 - S1^2, with values up
to 2^51 (n = 128 frames of energies 0 and 2550).  The device routine starts
from a single-precision estimate and corrects it by one each way, so the
cases that could break it are the neighbours of perfect squares (s^2 - 1,
s^2, s^2 + 2s) where the estimate's rounding is widest, the top of the range,
and powers of two.  The last test runs the whole scan on a clip that reaches
that top: 128 buffered frames whose energy is 0 or 2550 in every pixel."""
from __future__ import annotations

import math

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


LIMIT = 1 << 53


def _device_isqrt(lib, xs):
    x = torch.tensor(np.array(xs, dtype=np.uint64).view(np.int64), device="cuda")
    r = torch.zeros(len(xs), dtype=torch.int32, device="cuda")
    lib.scpl_isqrt(x, r)
    torch.cuda.synchronize()
    return r.cpu().numpy().view(np.uint32).astype(np.int64)


def _check(lib, xs):
    xs = sorted({int(v) for v in xs if 0 <= v < LIMIT})
    got = _device_isqrt(lib, xs)
    want = np.array([math.isqrt(v) for v in xs], np.int64)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, [(xs[i], int(got[i]), int(want[i])) for i in bad[:10]]


def test_neighbours_of_squares(lib):
    top = math.isqrt(LIMIT - 1)                       # 94,906,265
    mid = math.isqrt(1 << 51)                          # about 2^25.5
    r = np.random.default_rng(53)
    roots = set(range(0, 4096)) | set(range(mid - 4096, mid + 4096)) | \
        set(range(top - 4096, top + 1)) | {1 << e for e in range(27)} | \
        {(1 << e) - 1 for e in range(1, 27)} | set(r.integers(1, top, 20000).tolist())
    xs = []
    for s in roots:
        xs += [s * s - 1, s * s, s * s + 1, s * s + s, s * s + 2 * s - 1, s * s + 2 * s]
    _check(lib, xs)


def test_powers_of_two_and_random(lib):
    xs = []
    for e in range(53):
        xs += [(1 << e) - 1, 1 << e, (1 << e) + 1]
    r = np.random.default_rng(7)
    xs += r.integers(0, LIMIT, 200000, dtype=np.int64).tolist()
    xs += r.integers(1 << 50, 1 << 52, 200000, dtype=np.int64).tolist()
    _check(lib, xs)


def test_every_spread_of_the_extreme_clip(lib):
    """65536 Q for every buffer length n <= 128 and every count m of frames
    at energy 2550 (the rest 0): Q = 2550^2 m (n - m), up to 2550^2 * 4096."""
    xs = []
    for n in range(1, 129):
        for m in range(n + 1):
            S1, S2 = 2550 * m, 2550 * 2550 * m
            xs.append((n * S2 - S1 * S1) << 16)
    # and any energies in [0, 2550]: the largest spread at n = 128 and its neighbours
    qmax = (128 * 64 * 2550 ** 2 - (64 * 2550) ** 2) << 16
    xs += [qmax - d for d in range(0, 1 << 17, 97)]
    _check(lib, xs)


def test_scan_at_the_top_of_the_range(orc, lib):
    """wg = 0, wm = 10: grey frames whose luma is 0 or 255 at random give
    motion energies of 0 or 2550.  With alpha far above any spread the buffer
    fills to t_max = 128, so 65536 Q reaches its maximum.  Every frame's A_t
    and maximum equal the oracle's."""
    T, H, W = 140, 24, 72
    r = np.random.default_rng(2550)
    y = (r.integers(0, 2, (T, H, W)) * 255).astype(np.uint8)
    f = np.repeat(y[..., None], 3, axis=3)
    e = orc.energy(f, 0, 10)
    assert e.max() == 2550
    alpha = 1e6
    h = lib.scpl_create(lib.Params(alpha, 0, 10, 128, 1, 0))
    starts, A, M = lib.scpl_scan_stats(h, torch.from_numpy(f).cuda())
    lib.scpl_destroy(h)
    ref_starts = orc.scan(e, alpha=alpha, t_max=128)
    assert list(ref_starts) == [0, 128, T]
    assert np.array_equal(starts, ref_starts)
    assert np.array_equal(M, e.reshape(T, -1).max(axis=1))
    ref_A = np.array([orc.asde_sum(e[(t // 128) * 128:t + 1]) for t in range(T)], np.int64)
    assert np.array_equal(A, ref_A)
