"""Full-size parity on the GPU: the headline 1080p clip, the 256-clip batch and
a list of served jobs, each at the size and in the launch configuration the
benchmark uses, against SHA-256 digests of the oracle's outputs.

The digests in tests/golden/*.json were written by tests/golden/make_digests.py,
which calls only the CPU oracle (and the seeded input generator).  Every
output of the method is an integer, so the bar is equality: the same seams,
buffer starts and carved bytes (tolerance 0).  A digest covers each buffer's
seams and carved frames, so a failure names the buffer."""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import json
import multiprocessing as mp
import os

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


def _golden(name: str) -> dict:
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        pytest.skip(f"{name} has not been written (tests/golden/make_digests.py)")
    with open(path) as fh:
        return json.load(fh)


def _sha(a) -> str:
    if isinstance(a, torch.Tensor):
        a = a.cpu().numpy()
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def _generate(fn, specs):
    """Frames of every spec, generated in parallel processes (spawned, so that
    no CUDA state is forked)."""
    with cf.ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 4),
                                mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(fn, specs))


def _check_buffers(g_buffers, out, seams=None):
    for b, gb in enumerate(g_buffers):
        t0, t1 = gb["t0"], gb["t1"]
        if seams is not None:
            assert _sha(seams[b].astype("<i2")) == gb["seams_sha256"], f"seams of buffer {b}"
        assert _sha(out[t0:t1]) == gb["out_sha256"], f"frames of buffer {b} ({t0}..{t1})"


# ------------------------------------------------- 300-frame 1920x1080 clip
def test_clip_1080p_300f_every_buffer(lib):
    """The headline clip through scpl_carve, as the benchmark times it (no
    seam output) and with the seams requested: every buffer's seams and
    frames, the starts and every iteration's k_eff equal the oracle's."""
    from paper_1903_03180_gb300 import synth
    g = _golden("clip_1080p_300f.json")
    f = synth.workload_clip_1080p()
    frames = torch.from_numpy(f).cuda()
    T, H, W = f.shape[:3]
    r = lib.Retargeter(alpha=g["alpha"], wg=g["wg"], wm=g["wm"], t_max=g["t_max"])
    out = torch.empty((T, H, g["target"], 3), dtype=torch.uint8, device="cuda")
    starts = lib.scpl_carve(r.h, frames, g["target"], g["k"], out)
    torch.cuda.synchronize()
    assert [int(x) for x in starts] == g["starts"]
    out_np = out.cpu().numpy()
    _check_buffers(g["buffers"], out_np)
    assert _sha(out_np) == g["out_sha256"]
    keff = lib.scpl_keff_log(r.h)
    for b, gb in enumerate(g["buffers"]):
        assert [int(x) for x in keff[b]] == gb["k_eff"], f"k_eff of buffer {b}"
    out2, starts2, seams = r.carve(frames, g["target"], g["k"], with_seams=True)
    torch.cuda.synchronize()
    assert [int(x) for x in starts2] == g["starts"]
    _check_buffers(g["buffers"], out2.cpu().numpy(), seams.cpu().numpy())
    r.close()


def test_clip_1080p_300f_host_streamed(lib):
    """The end-to-end path the benchmark times: two clips streamed from
    page-locked host memory through scpl_carve_host_many (uploads, scans,
    carving and copies back overlapping), then one scpl_carve_host call.
    Every clip equals the oracle's."""
    from paper_1903_03180_gb300 import synth
    g = _golden("clip_1080p_300f.json")
    f = synth.workload_clip_1080p()
    T, H, W = f.shape[:3]
    src = torch.from_numpy(f).pin_memory().numpy()
    outs = [torch.zeros((T, H, g["target"], 3), dtype=torch.uint8).pin_memory().numpy()
            for _ in range(2)]
    h = lib.scpl_create()
    nbs = lib.scpl_carve_host_many(h, [src, src], g["target"], g["k"], outs)
    assert nbs == [len(g["starts"]) - 1] * 2
    for o in outs:
        _check_buffers(g["buffers"], o)
    outs[0][:] = 0
    starts = lib.scpl_carve_host(h, src, g["target"], g["k"], outs[0])
    lib.scpl_destroy(h)
    assert [int(x) for x in starts] == g["starts"]
    assert _sha(outs[0]) == g["out_sha256"]


# ------------------------------------------------- 256 clips x 32 frames
def test_batch_256x32_every_clip(lib):
    """The whole batched workload in one scpl_carve_batch call, autotuned as
    the benchmark runs it: every clip's buffer starts (first pass) and
    output equal the oracle's carve_job."""
    from paper_1903_03180_gb300 import synth
    g = _golden("batch_256x32.json")
    specs = synth.batch_spec()
    assert [(s["H"], s["W"], s["target_W"], s["target_H"], s["k"], s["seed"]) for s in specs] == \
        [(c["H"], c["W"], c["target_W"], c["target_H"], c["k"], c["seed"]) for c in g["clips"]]
    dev, outs, starts, jobs = [], [], [], []
    for sp, f in zip(specs, _generate(synth.batch_clip, specs)):
        dev.append(torch.from_numpy(f).cuda())
        outs.append(torch.zeros((sp["T"], sp["target_H"], sp["target_W"], 3),
                                dtype=torch.uint8, device="cuda"))
        starts.append(np.full(sp["T"] + 1, -1, np.int32))
        jobs.append(lib.make_job(dev[-1], sp["target_W"], sp["target_H"], sp["k"], outs[-1],
                                 starts[-1]))
    h = lib.scpl_create()
    lib.scpl_set_autotune(h, True)
    res = lib.scpl_carve_batch(h, jobs)
    torch.cuda.synchronize()
    lib.scpl_destroy(h)
    bad = []
    for c, (gc, (st, nb)) in enumerate(zip(g["clips"], res)):
        assert st == lib.SCPL_OK
        if [int(x) for x in starts[c][:nb + 1]] != gc["starts"]:
            bad.append((c, "starts"))
        elif _sha(outs[c]) != gc["out_sha256"]:
            bad.append((c, "frames"))
    assert not bad, bad


# --------------------------------------------------------- served jobs
def test_served_jobs_every_buffer(lib):
    """Twenty served jobs (640x360 to 3840x2160, 16-128 frames, 10-40 %
    narrower) submitted from page-locked host memory one scheduling round
    apart, so that each joins while the earlier ones are on the GPU: every
    job's starts, and every buffer's frames, equal the oracle's."""
    from paper_1903_03180_gb300 import synth
    g = _golden("serve_jobs20.json")
    specs = synth.serve_jobs()
    assert [(s["T"], s["H"], s["W"], s["target_W"], s["k"], s["seed"]) for s in specs] == \
        [(j["T"], j["H"], j["W"], j["target_W"], j["k"], j["seed"]) for j in g["jobs"]]
    srcs, outs, starts = [], [], []
    for sp, f in zip(specs, _generate(synth.serve_clip, specs)):
        srcs.append(torch.from_numpy(f).pin_memory().numpy())
        outs.append(torch.zeros((sp["T"], sp["H"], sp["target_W"], 3),
                                dtype=torch.uint8).pin_memory().numpy())
        starts.append(np.full(sp["T"] + 1, -1, np.int32))
    srv = lib.Server()
    tickets = {}
    max_active = 0
    for j, sp in enumerate(specs):
        tickets[srv.submit(srcs[j], sp["target_W"], sp["H"], sp["k"], outs[j], starts[j])] = j
        a, _ = srv.progress(wait=False)
        max_active = max(max_active, a)
    done = {}
    while len(done) < len(specs):
        a, _ = srv.progress(wait=True)
        max_active = max(max_active, a)
        for t, st in srv.poll():
            done[tickets[t]] = st
    srv.close()
    assert all(st == lib.SCPL_OK for st in done.values()), done
    assert max_active >= 2
    for j, gj in enumerate(g["jobs"]):
        nb = len(gj["starts"]) - 1
        assert [int(x) for x in starts[j][:nb + 1]] == gj["starts"], f"starts of job {j}"
        for b, gb in enumerate(gj["buffers"]):
            assert _sha(outs[j][gb["t0"]:gb["t1"]]) == gb["out_sha256"], \
                f"frames of job {j}, buffer {b}"
