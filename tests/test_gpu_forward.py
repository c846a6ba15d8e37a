"""Forward terms in the seam cost (params.wf > 0): every entry point that
carves equals the oracle's forward-energy carving byte for byte -- frames,
buffer starts and seams -- on single- and multi-buffer clips, ragged widths,
k from 1 to every parent, the wide-frame DP layout, the host-memory path, the
batch engine, the server and seam insertion."""
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


def _carve(lib, f, target, k, **kw):
    r = lib.Retargeter(**kw)
    out, starts, seams = r.carve(torch.from_numpy(f).cuda(), target, k, with_seams=True)
    torch.cuda.synchronize()
    r.close()
    return out.cpu().numpy(), starts, seams.cpu().numpy()


@pytest.mark.parametrize("T,H,W,target,k,wf,seed,cuts", [
    (6, 9, 11, 7, 2, 1, 1, (3, 3)),
    (5, 33, 70, 50, 8, 2, 2, (2, 3)),
    (4, 19, 257, 200, 16, 1, 3, None),
    (3, 40, 64, 40, 700, 3, 4, None),
    (2, 1, 5, 3, 1, 1, 5, None),
    (1, 7, 4, 2, 1, 2, 6, None),
    (8, 24, 130, 66, 4, 1, 7, (4, 4)),
])
def test_forward_carve_matches_oracle(orc, lib, T, H, W, target, k, wf, seed, cuts):
    from paper_1903_03180_gb300 import synth
    f = synth.clip(T, H, W, seed=seed, cuts=cuts)
    out, starts, seams = _carve(lib, f, target, k, wf=wf)
    ref, ref_starts, ref_seams = orc.carve(f, target, k, wf=wf)
    assert np.array_equal(starts, ref_starts)
    assert np.array_equal(seams, ref_seams)
    assert np.array_equal(out, ref)


def test_forward_changes_the_seams(orc, lib):
    """The weight matters: on the same clip wf = 2 removes other seams than
    the backward energy alone (so the parity above is not parity of the
    backward path)."""
    from paper_1903_03180_gb300 import synth
    f = synth.clip(4, 30, 80, seed=11)
    _, _, s0 = _carve(lib, f, 60, 4)
    _, _, s2 = _carve(lib, f, 60, 4, wf=2)
    assert not np.array_equal(s0, s2)
    assert np.array_equal(s2, orc.carve(f, 60, 4, wf=2)[2])


def test_forward_per_frame_and_gradient_only(orc, lib):
    from paper_1903_03180_gb300 import synth
    f = synth.clip(5, 21, 90, seed=12, cuts=(2, 2))
    out, starts, seams = _carve(lib, f, 70, 1, wf=1, use_buffer=False, wm=0)
    ref, ref_starts, ref_seams = orc.carve(f, 70, 1, wf=1, use_buffer=False, wm=0)
    assert np.array_equal(starts, ref_starts) and np.array_equal(out, ref)
    assert np.array_equal(seams, ref_seams)


def test_forward_second_cluster_layout(orc, lib):
    """2049 to 4096 columns: too wide for the 2-column-lane cluster, so the
    forward terms go through the 32-deep-halo, 4-column-lane layout."""
    from paper_1903_03180_gb300 import synth
    f = synth.clip(2, 6, 3000, seed=15)
    out, starts, seams = _carve(lib, f, 2990, 4, wf=2)
    ref, ref_starts, ref_seams = orc.carve(f, 2990, 4, wf=2)
    assert np.array_equal(starts, ref_starts) and np.array_equal(out, ref)
    assert np.array_equal(seams, ref_seams)


def test_forward_wide_frame_layout(orc, lib):
    """More than 4096 columns: the single-CTA DP's 8-column lanes."""
    from paper_1903_03180_gb300 import synth
    f = synth.clip(2, 3, 4500, seed=13)
    out, starts, seams = _carve(lib, f, 4488, 4, wf=1)
    ref, ref_starts, ref_seams = orc.carve(f, 4488, 4, wf=1)
    assert np.array_equal(starts, ref_starts) and np.array_equal(out, ref)
    assert np.array_equal(seams, ref_seams)


def test_forward_long_buffer(orc, lib):
    """A static clip of 200 frames in one buffer: the diagonal sums grow to
    255 * 200 and stay exact."""
    f = np.zeros((200, 10, 24, 3), np.uint8)
    f[:, :, ::2] = 255   # columns alternate black and white in every frame
    f[:, 3:6, 5:9] = 30
    out, starts, seams = _carve(lib, f, 20, 2, wf=1, t_max=256)
    ref, ref_starts, ref_seams = orc.carve(f, 20, 2, wf=1, t_max=256)
    assert list(starts) == list(ref_starts) == [0, 200]
    assert np.array_equal(out, ref) and np.array_equal(seams, ref_seams)


def test_forward_host_path(orc, lib):
    from paper_1903_03180_gb300 import synth
    f = synth.clip(12, 17, 60, seed=14, cuts=(4, 4))
    r = lib.Retargeter(wf=2)
    out = np.zeros((12, 17, 45, 3), np.uint8)
    starts = lib.scpl_carve_host(r.h, f, 45, 3, out)
    r.close()
    ref, ref_starts, _ = orc.carve(f, 45, 3, wf=2)
    assert np.array_equal(starts, ref_starts) and np.array_equal(out, ref)


def test_forward_batch_engine(orc, lib):
    """Width, height and both through one scpl_carve_batch call."""
    from paper_1903_03180_gb300 import synth
    spec = [(5, 20, 40, 30, 20, 3), (4, 20, 40, 40, 14, 2), (6, 20, 40, 33, 16, 4),
            (3, 12, 30, 20, 12, 1)]
    frames = [synth.clip(T, H, W, seed=20 + i) for i, (T, H, W, tw, th, k) in enumerate(spec)]
    outs = [torch.zeros((T, th, tw, 3), dtype=torch.uint8, device="cuda")
            for (T, H, W, tw, th, k) in spec]
    dev = [torch.from_numpy(f).cuda() for f in frames]
    jobs = [lib.make_job(dev[i], tw, th, k, outs[i]) for i, (T, H, W, tw, th, k) in enumerate(spec)]
    p = lib.scpl_default_params()
    p.wf = 2
    h = lib.scpl_create(p)
    res = lib.scpl_carve_batch(h, jobs)
    torch.cuda.synchronize()
    lib.scpl_destroy(h)
    for i, (T, H, W, tw, th, k) in enumerate(spec):
        assert res[i][0] == lib.SCPL_OK
        ref, _ = orc.carve_job(frames[i], tw, th, k, wf=2)
        assert np.array_equal(outs[i].cpu().numpy(), ref), i


def test_forward_server(orc, lib):
    from paper_1903_03180_gb300 import synth
    p = lib.scpl_default_params()
    p.wf = 1
    srv = lib.Server(p)
    f = [synth.clip(4, 16, 36, seed=30), synth.clip(3, 16, 36, seed=31)]
    outs = [torch.zeros((4, 16, 28, 3), dtype=torch.uint8, device="cuda"),
            torch.zeros((3, 12, 36, 3), dtype=torch.uint8, device="cuda")]
    t0 = srv.submit(torch.from_numpy(f[0]).cuda(), 28, 16, 3, outs[0])
    t1 = srv.submit(torch.from_numpy(f[1]).cuda(), 36, 12, 2, outs[1])
    srv.drain()
    done = dict(srv.poll())
    srv.close()
    torch.cuda.synchronize()
    assert done[t0] == lib.SCPL_OK and done[t1] == lib.SCPL_OK
    assert np.array_equal(outs[0].cpu().numpy(), orc.carve_job(f[0], 28, 16, 3, wf=1)[0])
    assert np.array_equal(outs[1].cpu().numpy(), orc.carve_job(f[1], 36, 12, 2, wf=1)[0])


def test_forward_enlarge(orc, lib):
    from paper_1903_03180_gb300 import synth
    f = synth.clip(5, 14, 30, seed=40, cuts=(2, 3))
    r = lib.Retargeter(wf=2)
    out, starts = r.enlarge(torch.from_numpy(f).cuda(), 41, 4)
    torch.cuda.synchronize()
    r.close()
    ref, ref_starts = orc.enlarge(f, 41, 4, wf=2)
    assert np.array_equal(starts, ref_starts) and np.array_equal(out.cpu().numpy(), ref)


def _fwd_cases(n=40, seed=0xF0E):
    r = np.random.default_rng(seed)
    out = []
    for c in range(n):
        T = int(r.integers(1, 8))
        H = int(r.choice([1, 2, int(r.integers(3, 40)), int(r.integers(40, 70))]))
        W = int(r.choice([4, 5, int(r.integers(6, 64)), int(r.integers(64, 260))]))
        out.append((c, T, H, W, int(r.integers(2, W + 1)),
                    int(r.choice([1, 2, int(r.integers(3, 30)), 700])),
                    int(r.choice([1, 2, 5, 255])), int(r.integers(0, 3)),
                    bool(r.integers(0, 4) > 0), int(r.integers(0, 1 << 30))))
    return out


@pytest.mark.parametrize("case", _fwd_cases(), ids=lambda c: f"fwd{c[0]}")
def test_forward_random_case(orc, lib, case):
    from paper_1903_03180_gb300 import synth
    _, T, H, W, target, k, wf, wm, use_buffer, seed = case
    f = synth.clip(T, H, W, seed=seed, cuts=(2, 3) if T >= 4 else None)
    kw = dict(wf=wf, wm=wm, wg=1, use_buffer=use_buffer)
    out, starts, seams = _carve(lib, f, target, k, **kw)
    ref, ref_starts, ref_seams = orc.carve(f, target, k, **kw)
    assert np.array_equal(starts, ref_starts)
    if W > target:
        assert np.array_equal(seams, ref_seams)
    assert np.array_equal(out, ref)
