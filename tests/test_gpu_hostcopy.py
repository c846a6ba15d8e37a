"""scpl_copy, the host/device transfer of the host-memory entry points: every
byte arrives, in both directions, for sizes around the 16-byte body and
offsets that share or do not share their place within 16 bytes (the second
kind goes through the copy engines), and from pageable memory."""
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


SIZES = [0, 1, 15, 16, 17, 255, 4096 + 3, 1 << 20, (1 << 24) + 11]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("off_h,off_d", [(0, 0), (5, 5), (3, 0), (0, 12)])
def test_both_directions(lib, n, off_h, off_d):
    r = np.random.default_rng(n * 7 + off_h * 3 + off_d)
    host = torch.empty(n + 32, dtype=torch.uint8).pin_memory()
    host.copy_(torch.from_numpy(r.integers(0, 256, n + 32, dtype=np.uint8)))
    dev = torch.full((n + 32,), 0xA5, dtype=torch.uint8, device="cuda")
    lib.scpl_copy(dev[off_d:off_d + n], host[off_h:off_h + n])
    torch.cuda.synchronize()
    got = dev.cpu()
    assert torch.equal(got[off_d:off_d + n], host[off_h:off_h + n])
    assert (got[:off_d] == 0xA5).all() and (got[off_d + n:] == 0xA5).all()   # nothing else written
    back = torch.zeros(n + 32, dtype=torch.uint8).pin_memory()
    lib.scpl_copy(back[off_h:off_h + n], dev[off_d:off_d + n])
    torch.cuda.synchronize()
    assert torch.equal(back[off_h:off_h + n], host[off_h:off_h + n])
    assert (back[:off_h] == 0).all() and (back[off_h + n:] == 0).all()


def test_pageable_host_memory(lib):
    src = np.arange(1 << 16, dtype=np.uint32).view(np.uint8)
    dev = torch.zeros(src.size, dtype=torch.uint8, device="cuda")
    lib.scpl_copy(dev, src)
    torch.cuda.synchronize()
    assert np.array_equal(dev.cpu().numpy(), src)


def test_side_stream_and_frames(lib):
    """A clip's worth of frames up and back on a stream of its own."""
    from paper_1903_03180_gb300 import synth
    f = synth.clip(8, 270, 480, seed=5)
    host = torch.from_numpy(f).pin_memory()
    dev = torch.empty(f.shape, dtype=torch.uint8, device="cuda")
    back = torch.zeros(f.shape, dtype=torch.uint8).pin_memory()
    s = torch.cuda.Stream()
    lib.scpl_copy(dev, host, stream=s)
    lib.scpl_copy(back, dev, stream=s)
    s.synchronize()
    assert np.array_equal(back.numpy(), f)
