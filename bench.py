#!/usr/bin/env python3
"""Benchmark: 1080p video retargeting throughput of libscpl on GB300.

One step = one scpl_carve of the 300-frame 1920x1080 clip (scene cuts every
60-120 frames, motion-aware energy, spatiotemporal buffer on, width reduced by
30 % = 576 seams, k = 32): energy, buffer scan, SCPL iterations of every
buffer and the colour gather, inputs resident in HBM.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

--impl reference times the CPU oracle (C, one process per host core, each
carving its own sub-clip) on a bounded sample of the same workload; that is
this project's reference arm.  --compare-raw adds the paper's comparison with
raw seam carving (classic, frame by frame) on the GPU and in the oracle.  Under torchrun
every rank carves its own clip (weak scaling, no collective on the data
path); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "1080p frames/s retargeted (bit-exact vs oracle), % of HBM roofline; p50/p99"
UNIT = "frames/s"

WORKLOADS = {
    # name: (T, H, W, target_W, k, generator kwargs, energy weights (wg, wm), use_buffer)
    "clip_1080p_300f": (300, 1080, 1920, 1344, 32, dict(cuts=(60, 120)), (1, 2), True),
    "clip_360p_64f": (64, 360, 640, 480, 16, dict(), (1, 2), True),
    "still_240p": (1, 240, 320, 288, 8, None, (1, 0), False),
}
SEEDS = {"clip_1080p_300f": 0x5C9 ^ 3, "clip_360p_64f": 0x5C9 ^ 2, "still_240p": 0x5C9 ^ 1}

# dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture of k_dpc<16,4,2>
# (16.7 MB for 2 buffers x 1080 rows x ~1900 columns, profiles/k_dpc_clip_1080p_128f.md)
# per carved pixel; the roofline's traffic scales it by the pixels a launch carves.
DP_DRAM_BYTES_PER_PX = 4.1


def make_frames(name: str, rank: int = 0, frames: int = 0) -> np.ndarray:
    from paper_1903_03180_gb300 import synth
    T, H, W, _, _, gen, _, _ = WORKLOADS[name]
    if frames:
        T = min(T, frames)
    seed = SEEDS[name] + 7919 * rank
    if gen is None:
        return synth.still_frame(H, W, seed)[None]
    return synth.clip(T, H, W, seed, **gen)


def peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return {"hbm_gbs": float(p["hbm_gbs"]), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [l.strip().split(",") for l in self.file.read().splitlines() if l.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_baseline(name: str, frames: np.ndarray, n_frames: int, wf: int = 0) -> dict:
    """The oracle as it stands (single thread) on the first `n_frames` frames
    of the workload: energy, buffer scan and carving of that sub-clip."""
    import oracle
    T, H, W, target, k, _, (wg, wm), use_buffer = WORKLOADS[name]
    sub = np.ascontiguousarray(frames[:n_frames])
    t0 = time.perf_counter()
    oracle.carve(sub, target, k, wg=wg, wm=wm, use_buffer=use_buffer, wf=wf)
    dt = time.perf_counter() - t0
    return {"value": round(len(sub) / dt, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {len(sub)} frames of {name} carved as one clip by the "
                      f"single-threaded C oracle ({dt:.1f} s)"}


def _oracle_warm(_):
    import oracle
    oracle._load()
    return os.getpid()


def _oracle_carve(task):
    """One process of the all-cores oracle run: carve frames [a, b) of the
    memory-mapped workload as a clip of its own; returns the seconds taken."""
    path, a, b, target, k, wg, wm, use_buffer, wf = task
    import oracle
    sub = np.ascontiguousarray(np.load(path, mmap_mode="r")[a:b])
    t0 = time.perf_counter()
    oracle.carve(sub, target, k, wg=wg, wm=wm, use_buffer=use_buffer, wf=wf)
    return time.perf_counter() - t0


class OraclePool:
    """The oracle on every host core: `procs` spawned processes, each carving
    an independent sub-clip of the workload (clips are independent units of
    the method, so this is the oracle as it stands, run side by side)."""

    def __init__(self, name: str, frames: np.ndarray, procs: int = 0, wf: int = 0):
        import multiprocessing as mp
        import oracle
        oracle.build()
        self.name = name
        self.wf = wf
        self.T = frames.shape[0]
        self.procs = procs or os.cpu_count() or 1
        self.dir = tempfile.mkdtemp(prefix="scpl_oracle_")
        self.path = os.path.join(self.dir, "frames.npy")
        np.save(self.path, frames)
        self.pool = mp.get_context("spawn").Pool(self.procs)
        self.pool.map(_oracle_warm, range(self.procs))

    def run(self, n: int) -> dict:
        T, H, W, target, k, _, (wg, wm), use_buffer = WORKLOADS[self.name]
        n = max(1, min(n, self.T))
        span = max(self.T - n + 1, 1)
        tasks = [(self.path, (p * n) % span, (p * n) % span + n, target, k, wg, wm, use_buffer,
                  self.wf) for p in range(self.procs)]
        t0 = time.perf_counter()
        per = self.pool.map(_oracle_carve, tasks, chunksize=1)
        wall = time.perf_counter() - t0
        return {"frames": n * self.procs, "wall_s": wall, "max_proc_s": max(per)}

    def close(self):
        self.pool.close()
        self.pool.join()
        os.unlink(self.path)
        os.rmdir(self.dir)


def _oracle_batch_job(task):
    """One process of the batched workload's oracle run: the first n frames
    of one job (its own size, targets and k) carved by the oracle."""
    spec, n = task
    import oracle

    from paper_1903_03180_gb300 import synth
    sub = np.ascontiguousarray(synth.batch_clip(spec)[:n])
    t0 = time.perf_counter()
    oracle.carve_job(sub, spec["target_W"], spec["target_H"], spec["k"])
    return time.perf_counter() - t0, len(sub)


def cpu_baseline_batch(specs: list, n_frames: int) -> dict:
    """The oracle on every host core for the batched workload: process p
    carves the first n_frames frames of job p."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    procs = min(os.cpu_count() or 1, len(specs))
    with mp.get_context("spawn").Pool(procs) as pool:
        pool.map(_oracle_warm, range(procs))
        t0 = time.perf_counter()
        per = pool.map(_oracle_batch_job, [(specs[p], n_frames) for p in range(procs)],
                       chunksize=1)
        wall = time.perf_counter() - t0
    frames = sum(n for _, n in per)
    busy = sum(t for t, _ in per)
    sizes = sorted({f"{sp['W']}x{sp['H']}" for sp in specs[:procs]})
    return {"value": round(frames / wall, 4), "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"{procs} processes (one per host core), process p carving the first "
                      f"{n_frames} frames of job p ({', '.join(sizes)}) with the C oracle "
                      f"({wall:.1f} s wall)",
            "one_core_value": round(frames / busy, 4),
            "one_core_note": "frames / summed per-process seconds, measured while all cores ran"}


def cpu_baseline_all_cores(name: str, frames: np.ndarray, n_frames: int, wf: int = 0) -> dict:
    pool = OraclePool(name, frames, wf=wf)
    try:
        r = pool.run(n_frames)
    finally:
        pool.close()
    return {"value": round(r["frames"] / r["wall_s"], 4), "unit": UNIT, "cores": pool.procs,
            "kind": "oracle",
            "sample": f"{pool.procs} processes (one per host core), each carving its own "
                      f"{n_frames}-frame sub-clip of {name} as a clip with the C oracle "
                      f"({r['wall_s']:.1f} s wall)"}


def run_reference(args) -> None:
    ws, rank, _ = _dist()
    if rank != 0:
        return
    name = args.workload
    frames = make_frames(name)
    n = args.ref_frames
    pool = OraclePool(name, frames, args.ref_procs, wf=args.wf)
    try:
        for _ in range(args.warmup):
            pool.run(n)
        t_all = time.perf_counter()
        done = 0
        for _ in range(args.steps):
            done += pool.run(n)["frames"]
        total = time.perf_counter() - t_all
    finally:
        pool.close()
    value = done / total
    sample = (f"each step: {pool.procs} processes (one per host core), each carving its own "
              f"{n}-frame sub-clip of {name} (energy, buffer scan, carving) with the C oracle")
    line = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1000 * total / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": name, "frames_per_step": n * pool.procs, "wf": args.wf},
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": pool.procs,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def raw_comparison(frames, frames_np, name: str, scpl_ms: float, cpu_frames: int,
                   cpu_scpl: dict | None) -> dict:
    """The paper's comparison of SCPL with raw seam carving (classic seam
    carving frame by frame: k = 1, no buffer, the same energy) on this
    hardware: the same clip carved both ways through the same kernels, and
    the oracle both ways on a sample."""
    import torch

    from paper_1903_03180_gb300 import scpl
    T, H, W, target, k, _, (wg, wm), use_buffer = WORKLOADS[name]
    raw = scpl.Retargeter(wg=wg, wm=wm, use_buffer=False, stream=torch.cuda.current_stream())
    out = torch.empty((frames.shape[0], H, target, 3), dtype=torch.uint8, device="cuda")
    scpl.scpl_carve(raw.h, frames, target, 1, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    scpl.scpl_carve(raw.h, frames, target, 1, out)
    e1.record()
    torch.cuda.synchronize()
    raw_ms = e0.elapsed_time(e1)
    raw.close()
    res = {"what": "raw = classic seam carving per frame (k = 1, no buffer, same energy)",
           "gpu_scpl_ms_per_clip": round(scpl_ms, 3), "gpu_raw_ms_per_clip": round(raw_ms, 3),
           "gpu_reduction": round(1.0 - scpl_ms / raw_ms, 4)}
    import oracle
    sub = np.ascontiguousarray(frames_np[:cpu_frames])
    t0 = time.perf_counter()
    oracle.carve(sub, target, 1, wg=wg, wm=wm, use_buffer=False)
    raw_s = (time.perf_counter() - t0) / len(sub)
    res["cpu_raw_s_per_frame"] = round(raw_s, 3)
    res["cpu_sample"] = f"first {len(sub)} frames, single-threaded C oracle"
    if cpu_scpl:
        scpl_s = 1.0 / cpu_scpl["value"]
        res["cpu_scpl_s_per_frame"] = round(scpl_s, 3)
        res["cpu_reduction"] = round(1.0 - scpl_s / raw_s, 4)
    return res


def run_native(args) -> None:
    import torch

    from paper_1903_03180_gb300 import scpl

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    name = args.workload
    T, H, W, target, k, _, (wg, wm), use_buffer = WORKLOADS[name]
    frames_np = make_frames(name, rank, args.frames)
    T = frames_np.shape[0]
    frames = torch.from_numpy(frames_np).cuda()
    out = torch.empty((T, H, target, 3), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    r = scpl.Retargeter(wg=wg, wm=wm, use_buffer=use_buffer, stream=stream, wf=args.wf)
    h = r.h

    for _ in range(max(args.warmup, 0)):
        starts = scpl.scpl_carve(h, frames, target, k, out)
    torch.cuda.synchronize()

    gpu_id = "0"
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        gpu_id = str(local)
    clocks = ClockSampler(gpu_id)
    clocks.start()
    time.sleep(0.3)

    # timed region: whole steps only (events between launches would cost ~6 %
    # and serialise the programmatic launch of each DP after its update)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev[0].record(stream)
    for s in range(args.steps):
        starts = scpl.scpl_carve(h, frames, target, k, out)
        ev[s + 1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    # kernel launches of the timed region: every call launches the same ones
    # (the carving iterations run as a graph that loops on the device)
    timed_launches = int(scpl.scpl_get_stats(h)["launches"]) * args.steps
    # per-kernel region: the same number of steps with every launch bracketed
    # by CUDA events on its stream, for the roofline of each kernel
    scpl.scpl_set_profiling(h, True)
    pev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    pev[0].record(stream)
    for s in range(args.steps):
        scpl.scpl_carve(h, frames, target, k, out)
    pev[1].record(stream)
    torch.cuda.synchronize()
    prof_ms = pev[0].elapsed_time(pev[1]) / args.steps
    stats = scpl.scpl_get_stats(h)
    keff = np.concatenate(scpl.scpl_keff_log(h) or [np.zeros(0, np.int32)])
    scpl.scpl_set_profiling(h, False)
    total_ms = ev[0].elapsed_time(ev[-1])
    if dist:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = T * ws * args.steps / (total_ms / 1000.0)

    # dominant kernel and its roofline
    pk = peaks()
    kern = stats["kernels"]
    dom = max(kern, key=lambda n: kern[n]["ms"])
    d = kern[dom]
    avg_ms = d["ms"] / max(d["launches"], 1)
    bytes_per_launch = d["bytes"] / max(d["launches"], 1)
    achieved = bytes_per_launch / (avg_ms / 1000.0) / 1e9
    traffic = None
    # DRAM bytes per carved pixel of one ncu capture of the plain k_dpc, scaled
    # (the forward-energy DP was not captured)
    if dom == "k_dp" and args.wf == 0:
        # carved_px covers the last clip; the launches cover every profiled step
        traffic = round(DP_DRAM_BYTES_PER_PX * stats["carved_px"] * args.steps /
                        max(d["launches"], 1))
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": pk["hbm_gbs"],
                "unit": "GB/s", "frac": round(achieved / pk["hbm_gbs"], 4), "traffic": traffic,
                "kernel": dom, "peak_source": pk["source"],
                "avg_launch_ms": round(avg_ms, 4),
                "alg_bytes_per_launch": round(bytes_per_launch),
                "timing": "per-launch CUDA events over %d steps right after the timed region "
                          "(%.3f ms a step with the events)" % (args.steps, prof_ms)}
    total_kernel_ms = sum(v["ms"] for v in kern.values())
    all_bytes = sum(v["bytes"] for v in kern.values())
    per_kernel = {n: {"launches_per_step": v["launches"] / args.steps,
                      "ms_per_step": round(v["ms"] / args.steps, 4),
                      "share": round(v["ms"] / total_kernel_ms, 4) if total_kernel_ms else None,
                      "GB_per_step": round(v["bytes"] / args.steps / 1e9, 4)}
                  for n, v in kern.items()}
    launches = int(sum(v["launches"] for v in kern.values()))

    # end to end through the host-memory entry points, pinned buffers: the
    # steps' clips streamed through scpl_carve_host_many (each clip's copies up
    # and back inside the timed region), and one scpl_carve_host call per clip
    e2e = e2e_single = None
    if not args.no_e2e:
        hin = torch.from_numpy(frames_np).pin_memory()
        houts = [torch.empty((T, H, target, 3), dtype=torch.uint8).pin_memory() for _ in range(2)]
        hin_np, hout_np = hin.numpy(), [o.numpy() for o in houts]

        def timed_host(fn, reps=1):
            """Wall time of fn() (host memory in and out, synchronised), after
            one untimed call; the median of `reps` timed calls, max over ranks."""
            fn()
            torch.cuda.synchronize()
            times = []
            for _ in range(reps):
                if dist:
                    dist.barrier()
                t0 = time.perf_counter()
                fn()
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                if dist:
                    t = torch.tensor([dt], device="cuda")
                    dist.all_reduce(t, op=dist.ReduceOp.MAX)
                    dt = float(t.item())
                times.append(dt)
            return float(np.median(times)), times

        # the machine's host<->device copy rates right now (page-locked, one
        # stream each way): the library's link copy (scpl_copy), which the
        # host paths use, and the copy engines (torch's copy_) for context
        dtmp = torch.empty_like(frames)
        otmp = torch.empty((T, H, target, 3), dtype=torch.uint8, device="cuda")

        def rate(fn, nbytes):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            return nbytes / (time.perf_counter() - t0) / 1e9

        def copy_rates():
            return {
                "link_h2d_gbs": round(rate(lambda: scpl.scpl_copy(dtmp, hin), hin.nbytes), 1),
                "link_d2h_gbs": round(rate(lambda: scpl.scpl_copy(houts[0], otmp),
                                           houts[0].nbytes), 1),
                "engine_h2d_gbs": round(rate(lambda: dtmp.copy_(hin, non_blocking=True),
                                             hin.nbytes), 1),
                "engine_d2h_gbs": round(rate(lambda: houts[0].copy_(otmp, non_blocking=True),
                                             houts[0].nbytes), 1)}

        copy_bw = copy_rates()
        ck = ClockSampler(gpu_id)
        ck.start()
        time.sleep(0.3)
        n_clips = max(args.steps, 2)
        dt, reps = timed_host(lambda: scpl.scpl_carve_host_many(
            h, [hin_np] * n_clips, target, k, [hout_np[i % 2] for i in range(n_clips)]),
            reps=args.e2e_reps)
        e2e_clk = ck.stop()
        dt_one, _ = timed_host(lambda: scpl.scpl_carve_host_many(h, [hin_np], target, k,
                                                                 [hout_np[0]]), reps=3)
        copy_bw_after = copy_rates()
        del dtmp, otmp
        steady_ms = (dt - dt_one) / (n_clips - 1) * 1e3
        dev_ms = total_ms / args.steps
        copies_ms = (hin.nbytes / copy_bw["link_h2d_gbs"] +
                     houts[0].nbytes / copy_bw["link_d2h_gbs"]) / 1e6
        e2e = {"value": round(T * ws * n_clips / dt, 2), "unit": UNIT,
               "h2d_bytes_per_step": int(frames_np.nbytes),
               "d2h_bytes_per_step": int(hout_np[0].nbytes),
               "api": "scpl_carve_host_many: %d clips streamed from page-locked host memory "
                      "through two device slots, uploads and copies back by scpl_copy "
                      "overlapping the kernels" % n_clips,
               "repetitions_s": [round(x, 4) for x in reps],
               "statistic": "median of %d timed calls after one untimed call" % len(reps),
               "one_clip_ms": round(dt_one * 1e3, 2),
               "steady_clip_ms": round(steady_ms, 2),
               "device_resident_clip_ms": round(dev_ms, 2),
               "copies_alone_ms": round(copies_ms, 2),
               "copies_hidden": round((dev_ms + copies_ms - steady_ms) / copies_ms, 3),
               "clocks": e2e_clk,
               "copy_bandwidth": copy_bw, "copy_bandwidth_after": copy_bw_after}
        dt1, _ = timed_host(lambda: [scpl.scpl_carve_host(h, hin_np, target, k, hout_np[0])
                                     for _ in range(args.steps)])
        e2e_single = {"value": round(T * ws * args.steps / dt1, 2), "unit": UNIT,
                      "api": "scpl_carve_host, one call per clip"}

    # the batched and served workloads, briefly, so that this line records
    # them too: one timed batched step of all 256 clips against the same jobs
    # one clip per call, and a short Poisson sweep through the server
    summaries = None
    if rank == 0 and ws == 1 and not args.no_summaries:
        b = measure_batch(256, steps=2, warmup=1)
        rates = [float(x) for x in args.summary_rates.split(",")]
        sv = measure_serve(rates, args.summary_duration, args.max_requests, args.out_buffers)
        summaries = {
            "batch_256x32": {
                "frames_per_s": round(b["value"], 1),
                "ms_per_step": round(sum(b["step_ms"]) / len(b["step_ms"]), 2),
                "one_clip_at_a_time_frames_per_s": round(b["one"], 1),
                "batched_over_one_at_a_time": round(b["value"] / b["one"], 3),
                "identical_output": b["identical"],
                "gpu_launches_per_step": int(b["engine"]["kernel_launches"]),
                "steps": len(b["step_ms"]), "clocks": b["clocks"],
                "what": "256 device-resident clips of 32 frames (426x240 to 1920x1080, "
                        "1:1/4:3/21:9 targets) in one scpl_carve_batch per step, against "
                        "the same jobs one call per clip"},
            "serve_poisson": {
                "sweep": [{"rate_per_s": x["rate_per_s"], "requests": x["requests"],
                           "failed": x["failed"], "frames_per_s": round(x["frames_per_s"], 1),
                           "p50_ms": None if x["p50_ms"] is None else round(x["p50_ms"], 2),
                           "p99_ms": None if x["p99_ms"] is None else round(x["p99_ms"], 2)}
                          for x in sv["results"]],
                "duration_s_per_rate": args.summary_duration,
                "what": "Poisson arrivals of page-locked host jobs (16-128 frames, 640x360 to "
                        "3840x2160, 10-40 % narrower) through one server; latency from "
                        "arrival to the result in host memory"}}

    cpu = cpu1 = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu1 = cpu_baseline(name, frames_np, args.cpu_frames, args.wf)
        cpu = cpu_baseline_all_cores(name, frames_np, args.cpu_frames, args.wf)
    raw = None
    if rank == 0 and args.compare_raw:
        raw = raw_comparison(frames, frames_np, name, total_ms / args.steps,
                             args.raw_cpu_frames, cpu1)

    if rank == 0:
        algo_gb = all_bytes / args.steps / 1e9
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": name if not args.frames else f"{name}[:{T}]", "T": T, "H": H, "W": W, "target_W": target, "k": k,
                       "seams": W - target, "wg": wg, "wm": wm, "wf": args.wf, "alpha": 0.2,
                       "use_buffer": use_buffer, "buffers": stats["n_buffers"],
                       "mean_buffer_frames": round(T / max(stats["n_buffers"], 1), 2),
                       "iterations_max": stats["iterations_max"],
                       "iterations_total": stats["iterations_total"],
                       "keff_mean": round(float(keff.mean()), 2) if keff.size else None,
                       "keff_histogram": {lbl: int(((keff >= lo) & (keff <= hi)).sum())
                                          for lbl, lo, hi in (("1", 1, 1), ("2-4", 2, 4),
                                                              ("5-8", 5, 8), ("9-16", 9, 16),
                                                              ("17-32", 17, 32),
                                                              (">32", 33, 1 << 30))},
                       "l2": "no flush: the clip (%.2f GB) and its luma are larger than the "
                             "129 MB L2" % (frames_np.nbytes / 1e9),
                       "parallelism": f"replicas{ws}"},
            "latency_ms": {"p50": round(float(np.percentile(step_ms, 50)), 3),
                           "p99": round(float(np.percentile(step_ms, 99)), 3),
                           "what": "one clip, device-resident"},
            "roofline": roofline,
            "hbm_fraction_whole_step": round(algo_gb / (total_ms / args.steps / 1000) /
                                             pk["hbm_gbs"], 4),
            "kernels": per_kernel,
            "kernels_region": "per-launch CUDA events over the %d steps after the timed region, "
                              "with the carving iterations launched from the host in chunks "
                              "(%d launches); the timed region runs them as a graph that "
                              "loops on the device" % (args.steps, launches),
            "gpu_launches": timed_launches,
            "clocks": clk,
            "e2e": e2e,
            "e2e_single_clip": e2e_single,
            "cpu_baseline": cpu,
            "cpu_baseline_1core": cpu1,
        }
        if summaries:
            line["workload_summaries"] = summaries
        if raw:
            line["raw_sc"] = raw
        print(json.dumps(line), flush=True)
    r.close()
    if dist:
        dist.destroy_process_group()


BATCH_METRIC = "frames/s retargeted, 256 clips x 32 frames of mixed size and target (batched)"
SERVE_METRIC = "frames/s and p50/p99 latency of served retarget jobs (Poisson arrivals)"


def _event_ms(fn):
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def _generate(fn, specs) -> list:
    """Frames of every spec, generated by spawned processes (no CUDA state is
    forked)."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 4)) as pool:
        return pool.map(fn, specs, chunksize=2)


def measure_batch(n_clips: int, steps: int, warmup: int, cpu_frames: int = 0) -> dict:
    """The batched workload: every clip device-resident, one scpl_carve_batch
    per step; then the same jobs one clip per call, outputs compared."""
    import torch

    from paper_1903_03180_gb300 import scpl, synth
    torch.cuda.set_device(0)
    specs = synth.batch_spec(n_clips=n_clips)
    t_gen = time.perf_counter()
    dev, outs, outs1 = [], [], []
    for sp, f in zip(specs, _generate(synth.batch_clip, specs)):
        dev.append(torch.from_numpy(f).cuda())
        shape = (sp["T"], sp["target_H"], sp["target_W"], 3)
        outs.append(torch.zeros(shape, dtype=torch.uint8, device="cuda"))
        outs1.append(torch.zeros(shape, dtype=torch.uint8, device="cuda"))
    t_gen = time.perf_counter() - t_gen
    jobs = [scpl.make_job(dev[i], sp["target_W"], sp["target_H"], sp["k"], outs[i])
            for i, sp in enumerate(specs)]
    jobs1 = [scpl.make_job(dev[i], sp["target_W"], sp["target_H"], sp["k"], outs1[i])
             for i, sp in enumerate(specs)]
    frames = sum(sp["T"] for sp in specs)
    h = scpl.scpl_create()
    scpl.scpl_set_autotune(h, True)   # every size is tuned once, during the warm-up
    for _ in range(max(warmup, 1)):
        scpl.scpl_carve_batch(h, jobs)
    st0 = scpl.scpl_batch_stats(h)
    clocks = ClockSampler("0")
    clocks.start()
    time.sleep(0.3)
    step_ms = [_event_ms(lambda: scpl.scpl_carve_batch(h, jobs)) for _ in range(steps)]
    clk = clocks.stop()
    st1 = scpl.scpl_batch_stats(h)
    # one clip per call through the same engine and kernels
    one_ms = _event_ms(lambda: [scpl.scpl_carve_batch(h, [j]) for j in jobs1])
    identical = all(torch.equal(a, b) for a, b in zip(outs, outs1))
    tuning = {f"{hh}x{w}": scpl.scpl_tuning_get(hh, w) for hh, w in
              sorted({(sp["H"], sp["W"]) for sp in specs} |
                     {(sp["W"] if sp["target_H"] < sp["H"] else sp["H"],
                       sp["H"] if sp["target_H"] < sp["H"] else sp["W"]) for sp in specs})}
    scpl.scpl_destroy(h)
    in_gb = sum(d.numel() for d in dev) / 1e9
    del dev, outs, outs1, jobs, jobs1
    torch.cuda.empty_cache()
    cpu = cpu_baseline_batch(specs, cpu_frames) if cpu_frames else None
    total = sum(step_ms)
    steps = max(steps, 1)
    value = frames * steps / (total / 1000.0)
    one = frames / (one_ms / 1000.0)
    return {"value": value, "frames": frames, "clips": len(specs), "step_ms": step_ms,
            "one_ms": one_ms, "one": one, "identical": bool(identical), "clocks": clk,
            "t_gen": t_gen, "in_gb": in_gb, "tuning": tuning, "cpu": cpu,
            "engine": {k: (st1[k] - st0[k]) / steps for k in
                       ("scan_waves", "groups", "chunks", "kernel_launches")}}


def run_batch(args) -> None:
    from paper_1903_03180_gb300 import synth
    m = measure_batch(args.clips, args.steps, args.warmup,
                      0 if args.no_cpu_baseline else args.batch_cpu_frames)
    steps = max(args.steps, 1)
    line = {"metric": BATCH_METRIC, "value": round(m["value"], 2), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(sum(m["step_ms"]) / steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"batch_{args.clips}x32", "clips": m["clips"],
                       "frames": m["frames"], "sizes": [f"{w}x{hh}" for hh, w in synth.BATCH_SIZES],
                       "aspects": list(synth.BATCH_ASPECTS), "wg": 1, "wm": 2,
                       "l2": "no flush: %.1f GB of clips, far above the 129 MB L2" % m["in_gb"],
                       "generation_s": round(m["t_gen"], 1)},
            "latency_ms": {"p50": round(float(np.percentile(m["step_ms"], 50)), 3),
                           "p99": round(float(np.percentile(m["step_ms"], 99)), 3),
                           "what": "one batched step (all clips)"},
            "one_clip_at_a_time": {"value": round(m["one"], 2), "unit": UNIT,
                                   "ms": round(m["one_ms"], 3),
                                   "what": "the same jobs, one scpl_carve_batch call per clip"},
            "batched_over_one_at_a_time": round(m["value"] / m["one"], 3),
            "identical_output": m["identical"],
            "engine_per_step": m["engine"],
            "tuning": m["tuning"],
            "gpu_launches": int(m["engine"]["kernel_launches"]),
            "clocks": m["clocks"],
            "cpu_baseline": m["cpu"]}
    print(json.dumps(line), flush=True)


STILLS_METRIC = "still-image retargeting time: SCPL (every parent's seam per iteration) vs seam carving"


def run_stills(args) -> None:
    """The paper's two image experiments (Sec. 4, Figs. 6-7) on synthetic
    stills: recursive carving to 0.8 of the previous width per loop, and direct
    carving to several width ratios, each by SCPL with an uncapped k (every
    parent's lowest seam per iteration, Eq. 6) and by classic seam carving
    (k = 1), with the gradient energy alone.  Times are CUDA-event medians of
    3 carves after a warm-up, on the GPU; the oracle repeats both at 640x480."""
    import torch

    from paper_1903_03180_gb300 import scpl, synth
    torch.cuda.set_device(0)
    r = scpl.Retargeter(wg=1, wm=0, use_buffer=False)
    UNCAPPED = 1 << 20

    def gpu_ms(img, target, k):
        x = torch.from_numpy(img[None]).cuda()
        out = torch.empty((1, img.shape[0], target, 3), dtype=torch.uint8, device="cuda")
        scpl.scpl_carve(r.h, x, target, k, out)
        ts = []
        for _ in range(3):
            ts.append(_event_ms(lambda: scpl.scpl_carve(r.h, x, target, k, out)))
        return float(np.median(ts)), out[0].cpu().numpy()

    def experiments(img, time_fn, loops=5, ratios=(0.9, 0.8, 0.7, 0.6, 0.5)):
        H, W = img.shape[:2]
        rec, cur = [], {"scpl": img, "sc": img}
        for i in range(loops):
            row = {"loop": i + 1}
            for name, k in (("scpl", UNCAPPED), ("sc", 1)):
                w = cur[name].shape[1]
                tgt = max(2, int(round(0.8 * w)))
                t, out = time_fn(cur[name], tgt, k)
                row[name + "_ms"] = round(t, 3)
                row["width"] = f"{w}->{tgt}"
                cur[name] = out
            row["reduction"] = round(1.0 - row["scpl_ms"] / row["sc_ms"], 4)
            rec.append(row)
        direct = []
        for ratio in ratios:
            tgt = max(2, int(round(ratio * W)))
            row = {"ratio": ratio, "width": f"{W}->{tgt}"}
            for name, k in (("scpl", UNCAPPED), ("sc", 1)):
                row[name + "_ms"] = round(time_fn(img, tgt, k)[0], 3)
            row["reduction"] = round(1.0 - row["scpl_ms"] / row["sc_ms"], 4)
            direct.append(row)
        return {"recursive": rec, "direct": direct}

    sizes = [(480, 640), (1080, 1920), (2160, 3840)]
    gpu = {}
    for H, W in sizes:
        img = synth.still_frame(H, W, seed=0x5C9 ^ 6 ^ (H * 7919 + W))
        gpu[f"{W}x{H}"] = experiments(img, gpu_ms)
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()

        def cpu_ms(img, target, k):
            t0 = time.perf_counter()
            out, _, _ = oracle.carve(img[None], target, k, wg=1, wm=0, use_buffer=False)
            return (time.perf_counter() - t0) * 1e3, out[0]

        img = synth.still_frame(480, 640, seed=0x5C9 ^ 6 ^ (480 * 7919 + 640))
        cpu = {"640x480": experiments(img, cpu_ms, loops=3, ratios=(0.9, 0.7, 0.5)),
               "cores": 1, "kind": "oracle"}
    reds = [row["reduction"] for v in gpu.values() for row in v["direct"]]
    line = {"metric": STILLS_METRIC, "value": round(100 * float(np.mean(reds)), 2),
            "unit": "% less time (mean over the direct ratios and sizes)", "n_gpus": 1,
            "higher_is_better": True, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "stills", "sizes": [f"{w}x{h}" for h, w in sizes],
                       "energy": "gradient only (wg = 1, wm = 0)", "scpl_k": "uncapped",
                       "sc_k": 1},
            "gpu": gpu, "cpu": cpu}
    print(json.dumps(line), flush=True)
    r.close()


CONSISTENCY_METRIC = "sharpness of 4-frame blends of a retargeted static clip (Fig. 9 stand-in)"


def run_consistency(args) -> None:
    """Fig. 9 of the paper, measured: a nearly static 64-frame 1920x1080 clip
    (no pan, no moving objects, noise of +-2) carved by 30 % with SCPL
    and the spatiotemporal buffer, and with raw seam carving frame by frame.
    The blend sharpness (num / den of scpl_blend_sharpness over every run of 4
    consecutive frames) is 1 for perfectly static content."""
    import torch

    from paper_1903_03180_gb300 import scpl, synth
    torch.cuda.set_device(0)
    T, H, W, target = 64, 1080, 1920, 1344
    f = synth.clip(T, H, W, seed=0x5C9 ^ 7, pan=0, n_ellipses=0, noise=2)
    x = torch.from_numpy(f).cuda()
    rs = scpl.Retargeter(wg=1, wm=2)
    rr = scpl.Retargeter(wg=1, wm=2, use_buffer=False)
    o_s, starts, _ = rs.carve(x, target, 32)
    ms_s = _event_ms(lambda: rs.carve(x, target, 32))
    o_r, _, _ = rr.carve(x, target, 1)
    ms_r = _event_ms(lambda: rr.carve(x, target, 1))

    def ratio(frames):
        n, d = scpl.scpl_blend_sharpness(rs.h, frames, 4)
        return round(n / d, 5) if d else None

    line = {"metric": CONSISTENCY_METRIC, "value": ratio(o_s), "unit": "num / den",
            "higher_is_better": True, "n_gpus": 1, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "static_1080p_64f", "T": T, "H": H, "W": W,
                       "target_W": target, "blend_window": 4},
            "input": ratio(x), "scpl": {"value": ratio(o_s), "k": 32, "buffers": len(starts) - 1,
                                        "ms_per_clip": round(ms_s, 3)},
            "raw_seam_carving": {"value": ratio(o_r), "k": 1, "buffers": T,
                                 "ms_per_clip": round(ms_r, 3)}}
    print(json.dumps(line), flush=True)
    rs.close()
    rr.close()


def _serve_source(i):
    """The 128-frame source clip of serving size i (cuts every 40-90 frames)."""
    from paper_1903_03180_gb300 import synth
    H, W, _ = SERVE_SIZES[i]
    return synth.clip(128, H, W, seed=(0x5C9 ^ 5) * 1000003 + i, cuts=(40, 90))


SERVE_SIZES = [(360, 640, 16), (720, 1280, 32), (1080, 1920, 32), (2160, 3840, 64)]


def measure_serve(rates: list, duration: float, max_requests: int, out_buffers: int) -> dict:
    """Serving: Poisson arrivals of host-memory jobs (16-128 frames, 360p to
    2160p, 10-40 % narrower) through one server, rates swept."""
    import torch

    from paper_1903_03180_gb300 import scpl, serve
    torch.cuda.set_device(0)
    sizes = SERVE_SIZES
    t_gen = time.perf_counter()
    # one 128-frame source clip per size, page-locked
    pool = [torch.from_numpy(f).pin_memory().numpy()
            for f in _generate(_serve_source, list(range(len(sizes))))]
    t_gen = time.perf_counter() - t_gen
    # page-locked output buffers, allocated before timing: out_buffers per
    # size, each big enough for 128 frames at full width
    t_pin = time.perf_counter()
    free_out = {i: [torch.empty(128 * H * W * 3, dtype=torch.uint8).pin_memory().numpy()
                    for _ in range(out_buffers)] for i, (H, W, k) in enumerate(sizes)}
    t_pin = time.perf_counter() - t_pin

    def get_out(si, T, H, tw):
        lst = free_out[si]
        if not lst:
            return None, None
        buf = lst.pop()
        return buf, buf[: T * H * tw * 3].reshape(T, H, tw, 3)

    results = []
    srv = scpl.Server()
    # tune the four sizes before the sweep (what a server does at start-up)
    th = scpl.scpl_create()
    tuning = {f"{W}x{H}": scpl.scpl_tune(th, H, W, k) for H, W, k in sizes}
    scpl.scpl_destroy(th)
    for ri, rate in enumerate(rates):
        r = np.random.default_rng(1000 + ri)
        arrivals = serve.poisson_arrivals(rate, duration, seed=2000 + ri,
                                          max_requests=max_requests)
        reqs = []
        for _ in arrivals:
            si = int(r.integers(0, len(sizes)))
            T = int(r.integers(16, 129))
            red = float(r.uniform(0.10, 0.40))
            reqs.append((si, T, red))
        held = {}

        def make(i):
            si, T, red = reqs[i]
            H, W, k = sizes[si]
            tw = W - int(round(W * red))
            buf, out = get_out(si, T, H, tw)
            if buf is None:
                return None   # waits for a buffer of its size
            held[i] = (si, buf)
            return serve.Request(pool[si][:T], tw, H, k, out)

        def done(i, st):
            si, buf = held.pop(i)
            free_out[si].append(buf)

        res = serve.run(srv, make, arrivals, on_complete=done)
        res["rate_per_s"] = rate
        results.append(res)
    st = srv.stats()
    srv.close()
    return {"results": results, "server": st, "tuning": tuning, "t_gen": t_gen, "t_pin": t_pin}


def run_serve(args) -> None:
    rates = [float(x) for x in args.rates.split(",")]
    m = measure_serve(rates, args.duration, args.max_requests, args.out_buffers)
    results, st, tuning = m["results"], m["server"], m["tuning"]
    best = max(results, key=lambda x: x["frames_per_s"])
    line = {"metric": SERVE_METRIC, "value": round(best["frames_per_s"], 2), "unit": UNIT,
            "n_gpus": 1, "steps": len(rates), "warmup": 0, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "serve_poisson", "sizes": [f"{w}x{h}" for h, w, _ in SERVE_SIZES],
                       "frames": "U[16,128]", "width_reduction": "U[10%,40%]",
                       "k": "16/32/32/64 by size", "duration_s_per_rate": args.duration,
                       "max_requests_per_rate": args.max_requests,
                       "source_clips": "one seeded 128-frame clip per size, requests take its "
                                       "first T frames (page-locked host memory)",
                       "output_buffers_per_size": args.out_buffers,
                       "generation_s": round(m["t_gen"], 1), "pinning_s": round(m["t_pin"], 1)},
            "latency_ms": {"p50": round(best["p50_ms"], 2), "p99": round(best["p99_ms"], 2),
                           "what": "arrival to result in host memory, at the best rate"},
            "sweep": [{k: (round(v, 3) if isinstance(v, float) else v) for k, v in x.items()}
                      for x in results],
            "server": {k: st[k] for k in ("submitted", "completed", "failed", "scan_waves",
                                          "groups", "chunks", "graphs_built",
                                          "kernel_launches", "peak_reserved_bytes",
                                          "budget_bytes")},
            "tuning": {k: {"dpc_halo": v["dpc_halo"], "update_rows": v["update_rows"]}
                       for k, v in tuning.items()},
            "gpu_launches": int(st["kernel_launches"])}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batch", "serve", "stills",
                                                                "consistency"],
                    default="clip_1080p_300f")
    ap.add_argument("--clips", type=int, default=256, help="batch: clips")
    ap.add_argument("--rates", default="5,10,20,50,100,200", help="serve: arrivals per s")
    ap.add_argument("--duration", type=float, default=2.0, help="serve: seconds per rate")
    ap.add_argument("--max-requests", type=int, default=120, help="serve: cap per rate")
    ap.add_argument("--out-buffers", type=int, default=6,
                    help="serve: page-locked output buffers per size (requests in flight)")
    ap.add_argument("--ref-frames", type=int, default=8,
                    help="frames each oracle process carves per reference step")
    ap.add_argument("--ref-procs", type=int, default=0,
                    help="oracle processes of the reference arm (0: one per host core)")
    ap.add_argument("--compare-raw", action="store_true",
                    help="also carve the clip as raw seam carving (k = 1, no buffer)")
    ap.add_argument("--raw-cpu-frames", type=int, default=1,
                    help="frames the oracle carves as raw seam carving for --compare-raw")
    ap.add_argument("--cpu-frames", type=int, default=16,
                    help="frames of the workload the oracle carves for cpu_baseline")
    ap.add_argument("--batch-cpu-frames", type=int, default=4,
                    help="batch: frames of each job the oracle carves for cpu_baseline")
    ap.add_argument("--frames", type=int, default=0,
                    help="carve only the first N frames of the workload (smaller profiling case)")
    ap.add_argument("--wf", type=int, default=0,
                    help="weight of the forward terms in the seam cost (0: the paper's "
                         "backward energy)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-summaries", action="store_true",
                    help="skip the short batch and serving measurements of the default run")
    ap.add_argument("--summary-rates", default="20,100",
                    help="arrival rates of the default run's serving summary")
    ap.add_argument("--summary-duration", type=float, default=2.0,
                    help="seconds per rate of the default run's serving summary")
    ap.add_argument("--e2e-reps", type=int, default=3,
                    help="timed repetitions of the end-to-end call (the median is reported)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "stills":
        run_stills(args)
    elif args.workload == "consistency":
        run_consistency(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
