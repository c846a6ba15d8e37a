"""The buffer scan decides most frames from a bounded float sum of the
spread (Eq. 7-8) and sums a frame exactly only when the threshold of Eq. 9
falls inside that bound.  These clips put every decision inside it: the
construction of Fig. 4 (frames of energy 0, then one frame of energy M
everywhere) makes the spread of every later frame equal the threshold up to
the floor of Eq. 7-8 when alpha is near 1, so every such round is replayed
exactly.  The buffers must still equal the oracle's, and the exact A_t of
the diagnostics must be unchanged."""
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


def _step_clip(T, H, W, k, d):
    """Grey frames: luma 0 up to frame k-1, d from frame k on, so that with
    wg = 0, wm = 10 the energy is 10 d in every pixel of frame k and 0
    elsewhere."""
    y = np.zeros((T, H, W), np.uint8)
    y[k:] = d
    return np.repeat(y[..., None], 3, axis=3)


@pytest.mark.parametrize("alpha", [1.0, 1.0 - 1e-9, 1.0 - 1e-6, 1.0 - 1e-4, 0.999, 0.5])
@pytest.mark.parametrize("k,d", [(3, 7), (10, 155), (21, 255)])
def test_near_threshold_decisions_match_the_oracle(orc, lib, alpha, k, d):
    T, H, W = 48, 24, 72
    f = _step_clip(T, H, W, k, d)
    e = orc.energy(f, 0, 10)
    ref = orc.scan(e, alpha=alpha, t_max=128)
    h = lib.scpl_create(lib.Params(alpha, 0, 10, 128, 1, 0))
    got = lib.scpl_scan(h, torch.from_numpy(f).cuda())
    starts_s, A, M = lib.scpl_scan_stats(h, torch.from_numpy(f).cuda())
    lib.scpl_destroy(h)
    assert np.array_equal(got, ref)
    assert np.array_equal(starts_s, ref)
    assert np.array_equal(M, e.reshape(T, -1).max(axis=1))


def test_random_clips_decide_as_the_oracle(orc, lib):
    """Ordinary clips at many alphas and buffer caps: the bounded sums decide
    almost every frame, and the buffers equal the oracle's."""
    from paper_1903_03180_gb300 import synth
    for case in range(8):
        r = np.random.default_rng(3100 + case)
        T, H, W = int(r.integers(20, 70)), int(r.integers(8, 90)), int(r.integers(16, 300))
        alpha = float(r.choice([0.02, 0.1, 0.2, 0.35, 0.8]))
        t_max = int(r.choice([5, 16, 128]))
        f = synth.clip(T, H, W, seed=3200 + case, cuts=(4, 15))
        h = lib.scpl_create(lib.Params(alpha, 1, 2, t_max, 1, 0))
        got = lib.scpl_scan(h, torch.from_numpy(f).cuda())
        lib.scpl_destroy(h)
        ref = orc.scan(orc.energy(f), alpha=alpha, t_max=t_max)
        assert np.array_equal(got, ref), (case, got, ref)
