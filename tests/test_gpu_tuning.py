"""Autotuning: every kernel choice the tuner can make (cluster DP with halo
depth 16 or 32, 4 or 8 warps a CTA, 4 or 2 columns a lane; the single-CTA DP;
1/2/4 update rows) gives the oracle's result bit for bit; the tuner measures
and records a choice."""
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
    scpl.scpl_tuning_clear()
    yield scpl
    scpl.scpl_tuning_clear()   # the table is process-wide


@pytest.fixture(scope="module")
def synth():
    from paper_1903_03180_gb300 import synth as s
    return s


# (halo, update rows, warps a CTA, columns a lane)
CHOICES = [(32, 4, 4, 4), (32, 1, 8, 4), (16, 2, 4, 4), (16, 4, 8, 4), (16, 2, 8, 2),
           (16, 1, 4, 2), (0, 1, 4, 4), (0, 4, 4, 4)]


@pytest.mark.parametrize("halo,rows,warps,cols", CHOICES)
@pytest.mark.parametrize("T,H,W,target,k,seed", [(6, 70, 300, 220, 16, 81),
                                                 (4, 50, 1000, 900, 32, 82),
                                                 (3, 37, 131, 100, 8, 83)])
def test_every_choice_is_exact(orc, lib, synth, halo, rows, warps, cols, T, H, W, target, k,
                               seed):
    lib.scpl_tuning_set(H, W, halo, rows, warps, cols)
    f = synth.clip(T, H, W, seed=seed, cuts=(2, 3))
    ref_out, ref_starts, ref_seams = orc.carve(f, target, k)
    r = lib.Retargeter()
    out, starts, seams = r.carve(torch.from_numpy(f).cuda(), target, k, with_seams=True)
    torch.cuda.synchronize()
    r.close()
    lib.scpl_tuning_clear()
    assert np.array_equal(starts, ref_starts)
    assert np.array_equal(seams.cpu().numpy(), ref_seams)
    assert np.array_equal(out.cpu().numpy(), ref_out)


def test_tune_measures_and_records(lib):
    h = lib.scpl_create()
    t = lib.scpl_tune(h, 1080, 1920, 32)
    lib.scpl_destroy(h)
    assert all(t["dp_us"][k] > 0 for k in ("r32w4", "r16w4", "r32w8", "r16w8", "r16w4v2",
                                           "r16w8v2"))
    assert t["dpc_lane_cols"] in (2, 4)
    assert all(v > 0 for v in t["update_us"].values())
    assert t["dpc_halo"] in (0, 16, 32) and t["update_rows"] in (1, 2, 4)
    rec = lib.scpl_tuning_get(1080, 1920)
    assert rec["dpc_halo"] == t["dpc_halo"] and rec["update_rows"] == t["update_rows"]
    lib.scpl_tuning_clear()


def test_autotuned_batch_is_exact(orc, lib, synth):
    spec = [(5, 48, 90, 70, 48, 4, 91), (4, 48, 90, 90, 30, 8, 92)]
    frames = [synth.clip(T, H, W, seed=s) for (T, H, W, tw, th, k, s) in spec]
    outs = [torch.zeros((T, th, tw, 3), dtype=torch.uint8, device="cuda")
            for (T, H, W, tw, th, k, s) in spec]
    dev = [torch.from_numpy(x).cuda() for x in frames]
    jobs = [lib.make_job(dev[i], tw, th, k, outs[i]) for i, (T, H, W, tw, th, k, s)
            in enumerate(spec)]
    h = lib.scpl_create()
    lib.scpl_set_autotune(h, True)
    lib.scpl_carve_batch(h, jobs)
    torch.cuda.synchronize()
    lib.scpl_destroy(h)
    assert lib.scpl_tuning_get(48, 90) is not None      # width pass size
    assert lib.scpl_tuning_get(90, 48) is not None      # height pass (transposed) size
    for i, (T, H, W, tw, th, k, s) in enumerate(spec):
        ref, _ = orc.carve_job(frames[i], tw, th, k)
        assert np.array_equal(outs[i].cpu().numpy(), ref)
    lib.scpl_tuning_clear()
