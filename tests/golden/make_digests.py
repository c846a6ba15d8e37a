#!/usr/bin/env python3
"""Writes the SHA-256 digests of the full-size workloads, computed by the CPU
oracle alone (test infrastructure: it imports ``oracle`` and the seeded input
generator ``synth`` and nothing of the CUDA library).

The GPU tests (``tests/test_gpu_golden.py``) carve the same seeded inputs
through the C ABI and compare the digests of their outputs with these.

  python tests/golden/make_digests.py clip_1080p_300f [--procs N]
  python tests/golden/make_digests.py batch_256x32    [--procs N]
  python tests/golden/make_digests.py serve_jobs20    [--procs N]

What each file holds:
- clip_1080p_300f.json: the 300-frame 1920x1080 clip with scene cuts (576
  seams, k = 32, wg = 1, wm = 2, alpha = 0.2, t_max = 128).  The buffer starts
  of the scan (Sec. 3.2, Eq. 7-9) and, per buffer, the digests of its seams
  (int16 [W - target][H], original columns, removal order) and of its carved
  frames (uint8 [T_b][H][target][3]); also the digest of the whole output.
- batch_256x32.json: the 256 clips of 32 frames of mixed size and target
  aspect; per clip the starts of its first pass and the digest of its output
  (uint8 [T][target_H][target_W][3]), carved by ``oracle.carve_job``
  (horizontal seams by transposition).
- serve_jobs20.json: 20 served jobs drawn by ``synth.serve_jobs`` (360p to
  3840x2160, 16-128 frames, 10-40 % narrower); per job its starts and, per
  buffer, the digests of its seams and of its carved frames.

A clip's buffers are carved independently once the scan has fixed them
(Sec. 3.2: the same seams are removed from every frame of a buffer, computed
from that buffer's frames alone), so the script carves them in separate
processes.  Buffer b's motion term needs the frame before it (D_t uses Y_{t-1},
with D = 0 only for the clip's first frame); ``motion`` of the slice that
starts one frame earlier gives exactly the rows ``oracle.carve`` uses.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CLIP = dict(target=1344, k=32, wg=1, wm=2, alpha=0.2, t_max=128)


def sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


# ------------------------------------------------------------ 1080p clip
def _clip_buffer(task):
    import oracle
    from paper_1903_03180_gb300 import synth
    b, t0, t1 = task
    f = synth.workload_clip_1080p()
    D = oracle.motion(f[max(t0 - 1, 0):t1])[1 if t0 > 0 else 0:]
    t = time.time()
    out, seams, keff = oracle.carve_buffer(f[t0:t1], D, CLIP["target"], CLIP["k"],
                                           wg=CLIP["wg"], wm=CLIP["wm"])
    return b, out, seams, keff, time.time() - t


def clip_1080p(procs: int) -> dict:
    import oracle
    from paper_1903_03180_gb300 import synth
    f = synth.workload_clip_1080p()
    T, H, W = f.shape[:3]
    starts = oracle.scan(oracle.energy(f, CLIP["wg"], CLIP["wm"]), alpha=CLIP["alpha"],
                         t_max=CLIP["t_max"])
    del f
    tasks = [(b, int(starts[b]), int(starts[b + 1])) for b in range(len(starts) - 1)]
    outs = {}
    with mp.get_context("spawn").Pool(min(procs, len(tasks))) as pool:
        for b, out, seams, keff, dt in pool.imap_unordered(_clip_buffer, tasks):
            outs[b] = (out, seams, keff)
            print(f"buffer {b}: {out.shape[0]} frames, {len(keff)} iterations, {dt:.0f} s",
                  flush=True)
    whole = np.concatenate([outs[b][0] for b in range(len(tasks))])
    return {
        "workload": "clip_1080p_300f",
        "source": "synth.workload_clip_1080p()",
        "T": T, "H": H, "W": W, **CLIP,
        "starts": [int(x) for x in starts],
        "buffers": [{"t0": t0, "t1": t1, "iterations": int(len(outs[b][2])),
                     "k_eff": [int(x) for x in outs[b][2]],
                     "seams_sha256": sha(outs[b][1].astype("<i2")),
                     "out_sha256": sha(outs[b][0])} for b, t0, t1 in tasks],
        "out_sha256": sha(whole),
    }


# ------------------------------------------------------- batched clips
def _batch_clip(spec):
    import oracle
    from paper_1903_03180_gb300 import synth
    f = synth.batch_clip(spec)
    t = time.time()
    out, starts = oracle.carve_job(f, spec["target_W"], spec["target_H"], spec["k"])
    return spec["clip"], [int(x) for x in starts], sha(out), time.time() - t


def batch(procs: int) -> dict:
    from paper_1903_03180_gb300 import synth
    specs = synth.batch_spec()
    res = {}
    with mp.get_context("spawn").Pool(procs) as pool:
        for c, starts, digest, dt in pool.imap_unordered(_batch_clip, specs):
            res[c] = (starts, digest)
            print(f"clip {c} ({len(res)}/{len(specs)}): {dt:.0f} s", flush=True)
    return {
        "workload": "batch_256x32",
        "source": "synth.batch_spec(), synth.batch_clip(spec)",
        "params": "wg = 1, wm = 2, alpha = 0.2, t_max = 128, buffer on",
        "clips": [{**{k: sp[k] for k in ("clip", "T", "H", "W", "target_W", "target_H", "k",
                                         "seed")},
                   "starts": res[sp["clip"]][0], "out_sha256": res[sp["clip"]][1]}
                  for sp in specs],
    }


# -------------------------------------------------------- served jobs
def _serve_scan(spec):
    import oracle
    from paper_1903_03180_gb300 import synth
    f = synth.serve_clip(spec)
    starts = oracle.scan(oracle.energy(f, CLIP["wg"], CLIP["wm"]), alpha=CLIP["alpha"],
                         t_max=CLIP["t_max"])
    return spec["job"], [int(x) for x in starts]


def _serve_buffer(task):
    import oracle
    from paper_1903_03180_gb300 import synth
    spec, b, t0, t1 = task
    f = synth.serve_clip(spec)[max(t0 - 1, 0):t1].copy()
    D = oracle.motion(f)[1 if t0 > 0 else 0:]
    t = time.time()
    out, seams, keff = oracle.carve_buffer(f[1 if t0 > 0 else 0:], D, spec["target_W"],
                                           spec["k"], wg=CLIP["wg"], wm=CLIP["wm"])
    return spec["job"], b, sha(out), sha(seams.astype("<i2")), len(keff), time.time() - t


def serve(procs: int) -> dict:
    """Every served job narrows the width only (target_H = H), so ``carve_job``
    is ``carve``: the scan, then each buffer carved on its own."""
    from paper_1903_03180_gb300 import synth
    specs = synth.serve_jobs()
    assert all(sp["target_H"] == sp["H"] for sp in specs)
    starts = {}
    with mp.get_context("spawn").Pool(procs) as pool:
        for j, st in pool.imap_unordered(_serve_scan, specs):
            starts[j] = st
            print(f"job {j}: buffers {st}", flush=True)
        tasks = [(sp, b, starts[sp["job"]][b], starts[sp["job"]][b + 1])
                 for sp in specs for b in range(len(starts[sp["job"]]) - 1)]
        # the largest buffers first, so that none of them finishes last
        tasks.sort(key=lambda t: -(t[3] - t[2]) * t[0]["H"] * t[0]["W"] *
                   (t[0]["W"] - t[0]["target_W"]))
        res = {}
        for j, b, od, sd, it, dt in pool.imap_unordered(_serve_buffer, tasks):
            res[(j, b)] = (od, sd, it)
            print(f"job {j} buffer {b} ({len(res)}/{len(tasks)}): {it} iterations, {dt:.0f} s",
                  flush=True)
    return {
        "workload": "serve_jobs20",
        "source": "synth.serve_jobs(), synth.serve_clip(spec)",
        "params": "wg = 1, wm = 2, alpha = 0.2, t_max = 128, buffer on",
        "jobs": [{**{k: sp[k] for k in ("job", "T", "H", "W", "target_W", "target_H", "k",
                                        "seed")},
                  "starts": starts[sp["job"]],
                  "buffers": [{"t0": starts[sp["job"]][b], "t1": starts[sp["job"]][b + 1],
                               "iterations": res[(sp["job"], b)][2],
                               "seams_sha256": res[(sp["job"], b)][1],
                               "out_sha256": res[(sp["job"], b)][0]}
                              for b in range(len(starts[sp["job"]]) - 1)]}
                 for sp in specs],
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["clip_1080p_300f", "batch_256x32", "serve_jobs20"])
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 4)
    args = ap.parse_args()
    t = time.time()
    fn = {"clip_1080p_300f": clip_1080p, "batch_256x32": batch, "serve_jobs20": serve}
    doc = fn[args.what](args.procs)
    doc["generated_by"] = "tests/golden/make_digests.py (oracle only)"
    path = os.path.join(HERE, args.what + ".json")
    with open(path, "w") as fh:
        json.dump(doc, fh, indent=1)
        fh.write("\n")
    print(f"wrote {path} in {time.time() - t:.0f} s")


if __name__ == "__main__":
    main()
