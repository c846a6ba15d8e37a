#!/usr/bin/env python3
"""Benchmark: 1080p video retargeting throughput of libscpl on GB300.

One step = one scpl_carve of the 300-frame 1920x1080 clip (scene cuts every
60-120 frames, motion-aware energy, spatiotemporal buffer on, width reduced by
30 % = 576 seams, k = 32): energy, buffer scan, SCPL iterations of every
buffer and the colour gather, inputs resident in HBM.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

--impl reference times the CPU oracle (single-threaded C) on a bounded sample
of the same workload; that is this project's reference arm.  Under torchrun
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


def cpu_baseline(name: str, frames: np.ndarray, n_frames: int) -> dict:
    """The oracle as it stands (single thread) on the first `n_frames` frames
    of the workload: energy, buffer scan and carving of that sub-clip."""
    import oracle
    T, H, W, target, k, _, (wg, wm), use_buffer = WORKLOADS[name]
    sub = np.ascontiguousarray(frames[:n_frames])
    t0 = time.perf_counter()
    oracle.carve(sub, target, k, wg=wg, wm=wm, use_buffer=use_buffer)
    dt = time.perf_counter() - t0
    return {"value": round(len(sub) / dt, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {len(sub)} frames of {name} carved as one clip by the "
                      f"single-threaded C oracle ({dt:.1f} s)"}


def run_reference(args) -> None:
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    oracle.build()
    name = args.workload
    frames = make_frames(name)
    n = args.ref_frames
    for _ in range(args.warmup):
        cpu_baseline(name, frames, n)
    vals = []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        cpu_baseline(name, frames, n)
        vals.append(time.perf_counter() - t0)
    total = time.perf_counter() - t_all
    value = n * args.steps / total
    sample = (f"each step: first {n} frames of {name} (energy, buffer scan, carving) by the "
              f"single-threaded C oracle")
    line = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1000 * total / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": name, "frames_per_step": n},
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": 1,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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
    r = scpl.Retargeter(wg=wg, wm=wm, use_buffer=use_buffer, stream=stream)
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

    scpl.scpl_set_profiling(h, True)
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
    stats = scpl.scpl_get_stats(h)
    scpl.scpl_set_profiling(h, False)
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
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
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": pk["hbm_gbs"],
                "unit": "GB/s", "frac": round(achieved / pk["hbm_gbs"], 4), "traffic": None,
                "kernel": dom, "peak_source": pk["source"],
                "avg_launch_ms": round(avg_ms, 4),
                "alg_bytes_per_launch": round(bytes_per_launch)}
    total_kernel_ms = sum(v["ms"] for v in kern.values())
    all_bytes = sum(v["bytes"] for v in kern.values())
    per_kernel = {n: {"launches_per_step": v["launches"] / args.steps,
                      "ms_per_step": round(v["ms"] / args.steps, 4),
                      "share": round(v["ms"] / total_kernel_ms, 4) if total_kernel_ms else None,
                      "GB_per_step": round(v["bytes"] / args.steps / 1e9, 4)}
                  for n, v in kern.items()}
    launches = int(sum(v["launches"] for v in kern.values()))

    # end to end through the host-memory entry point, pinned buffers
    e2e = None
    if not args.no_e2e:
        hin = torch.from_numpy(frames_np).pin_memory()
        hout = torch.empty((T, H, target, 3), dtype=torch.uint8).pin_memory()
        hin_np, hout_np = hin.numpy(), hout.numpy()
        scpl.scpl_carve_host(h, hin_np, target, k, hout_np)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            scpl.scpl_carve_host(h, hin_np, target, k, hout_np)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if dist:
            t = torch.tensor([dt], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        e2e = {"value": round(T * ws * args.steps / dt, 2), "unit": UNIT,
               "h2d_bytes_per_step": int(frames_np.nbytes),
               "d2h_bytes_per_step": int(hout_np.nbytes)}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(name, frames_np, args.cpu_frames)

    if rank == 0:
        algo_gb = all_bytes / args.steps / 1e9
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": name if not args.frames else f"{name}[:{T}]", "T": T, "H": H, "W": W, "target_W": target, "k": k,
                       "seams": W - target, "wg": wg, "wm": wm, "alpha": 0.2,
                       "use_buffer": use_buffer, "buffers": stats["n_buffers"],
                       "mean_buffer_frames": round(T / max(stats["n_buffers"], 1), 2),
                       "iterations_max": stats["iterations_max"],
                       "iterations_total": stats["iterations_total"],
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
            "gpu_launches": launches,
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    r.close()
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="clip_1080p_300f")
    ap.add_argument("--ref-frames", type=int, default=8,
                    help="frames of the workload the oracle carves per reference step")
    ap.add_argument("--cpu-frames", type=int, default=16,
                    help="frames of the workload the oracle carves for cpu_baseline")
    ap.add_argument("--frames", type=int, default=0,
                    help="carve only the first N frames of the workload (smaller profiling case)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
