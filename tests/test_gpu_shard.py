"""scpl_carve_buffer, the GPU half of buffer-level sharding (a clip's fixed
buffers carved on different GPUs after one scan, Sec. 3.2): one buffer carved
on its own, given the clip's frame before it, is byte for byte that buffer of
the whole clip's carve.  Checked against the oracle's digests of the 300-frame
1080p clip (every buffer), against oracle.carve_buffer on small random clips,
and through shard.carve_clip_by_buffers on one rank."""
from __future__ import annotations

import hashlib
import json
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1903_03180_gb300 import scpl
    return scpl


def _sha(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def _carve_buffer(lib, h, fb, prev, target, k, with_seams=True):
    T, H, W, _ = fb.shape
    out = torch.empty((T, H, target, 3), dtype=torch.uint8, device="cuda")
    seams = torch.full((1, W - target, H), -1, dtype=torch.int16, device="cuda") \
        if with_seams else None
    lib.scpl_carve_buffer(h, fb, target, k, out, prev, seams)
    torch.cuda.synchronize()
    return out.cpu().numpy(), None if seams is None else seams.cpu().numpy()[0]


def test_every_buffer_of_the_1080p_clip_alone(lib):
    from paper_1903_03180_gb300 import synth
    with open(os.path.join(GOLDEN, "clip_1080p_300f.json")) as fh:
        g = json.load(fh)
    frames = torch.from_numpy(synth.workload_clip_1080p()).cuda()
    h = lib.scpl_create()
    for b, gb in enumerate(g["buffers"]):
        t0, t1 = gb["t0"], gb["t1"]
        prev = frames[t0 - 1] if t0 > 0 else None
        out, seams = _carve_buffer(lib, h, frames[t0:t1], prev, g["target"], g["k"])
        assert _sha(seams.astype("<i2")) == gb["seams_sha256"], f"seams of buffer {b}"
        assert _sha(out) == gb["out_sha256"], f"frames of buffer {b}"
        assert [int(x) for x in lib.scpl_keff_log(h)[0]] == gb["k_eff"]
    lib.scpl_destroy(h)


@pytest.mark.parametrize("case", range(12))
def test_random_buffers_against_the_oracle(orc, lib, case):
    from paper_1903_03180_gb300 import synth
    r = np.random.default_rng(700 + case)
    T = int(r.integers(2, 30))
    H, W = int(r.integers(3, 70)), int(r.integers(5, 300))
    target = int(r.integers(2, W + 1))
    k = int(r.choice([1, 3, 8, 32, 1000]))
    wg, wm, wf = [(1, 2, 0), (1, 0, 0), (2, 5, 0), (1, 2, 1)][case % 4]
    f = synth.clip(T + 1, H, W, seed=900 + case)
    first = case % 3 == 0          # a buffer that starts its clip: no frame before it
    fb = f[:T] if first else f[1:]
    D = orc.motion(fb) if first else orc.motion(f)[1:]
    ref_out, ref_seams, ref_keff = orc.carve_buffer(fb, D, target, k, wg=wg, wm=wm, wf=wf)
    h = lib.scpl_create(lib.Params(0.2, wg, wm, 128, 1, 0, wf))
    dev = torch.from_numpy(f).cuda()
    out, seams = _carve_buffer(lib, h, dev[:T] if first else dev[1:], None if first else dev[0],
                               target, k)
    keff = lib.scpl_keff_log(h)[0] if W > target else []
    lib.scpl_destroy(h)
    assert np.array_equal(seams[:W - target], ref_seams)
    assert np.array_equal(out, ref_out)
    assert [int(x) for x in keff] == [int(x) for x in ref_keff]


def test_more_frames_than_a_buffer_holds(lib):
    h = lib.scpl_create(lib.Params(0.2, 1, 2, 4, 1, 0))
    f = torch.zeros((5, 8, 16, 3), dtype=torch.uint8, device="cuda")
    out = torch.zeros((5, 8, 12, 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(lib.SCPLError) as ei:
        lib.scpl_carve_buffer(h, f, 12, 2, out)
    assert ei.value.status == lib.SCPL_EINVAL
    lib.scpl_carve_buffer(h, f[:4].contiguous(), 12, 2, out[:4])   # t_max frames are fine
    lib.scpl_destroy(h)


def test_sharded_orchestration_on_one_rank(orc, lib):
    """shard.carve_clip_by_buffers with the GPU carving every buffer (a
    one-rank group): the clip equals the oracle's carve."""
    import torch.distributed as dist
    from paper_1903_03180_gb300 import shard, synth
    f = synth.clip(40, 36, 90, seed=77, cuts=(6, 12))
    ref_out, ref_starts, _ = orc.carve(f, 70, 8)
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        h = lib.scpl_create()

        def scan(fr):
            return lib.scpl_scan(h, fr)

        def carve(fb, prev, target, k):
            out = torch.empty((fb.shape[0], fb.shape[1], target, 3), dtype=torch.uint8,
                              device="cuda")
            lib.scpl_carve_buffer(h, fb, target, k, out, prev)
            return out

        out, starts, mine = shard.carve_clip_by_buffers(torch.from_numpy(f).cuda(), 70, 8, scan,
                                                        carve)
        torch.cuda.synchronize()
        lib.scpl_destroy(h)
    finally:
        dist.destroy_process_group()
    assert list(starts) == list(ref_starts) and mine == list(range(len(starts) - 1))
    assert np.array_equal(out.cpu().numpy(), ref_out)
