"""Serving: a request loop over the native server (scpl_server_*).

Requests arrive by a seeded Poisson process and are submitted as they
arrive.  The server admits them by device-memory footprint and runs them
beside the jobs already on the GPU (continuous batching).  The loop records
each request's latency, from arrival to completion with the result back in
host memory.  Everything the GPU does happens in libscpl; this module only
times arrivals and hands over buffers.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np

from . import scpl


@dataclass
class Request:
    frames: np.ndarray     # [T,H,W,3] uint8, host (page-locked for overlap)
    target_W: int
    target_H: int
    k: int
    out: np.ndarray        # [T,target_H,target_W,3] uint8, host


def poisson_arrivals(rate: float, duration: float, seed: int, max_requests: int = 0):
    """Arrival times (seconds from start) of a Poisson process of `rate` per
    second over `duration` seconds, optionally capped at max_requests."""
    r = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += float(r.exponential(1.0 / rate))
        if t >= duration or (max_requests and len(out) >= max_requests):
            return out
        out.append(t)


def run(server: scpl.Server, make_request, arrivals: list[float], idle_sleep: float = 2e-4,
        on_complete=None) -> dict:
    """Submit request i at arrivals[i] and drive the server until every
    request has completed; return throughput and latency figures.
    make_request(i) returns a Request, or None while it has no output buffer
    for it (the request then waits, in arrival order, with its latency clock
    running).  on_complete(i, status) is called for each completion, e.g. to
    recycle buffers."""
    from collections import deque
    n = len(arrivals)
    pending: dict[int, tuple[int, float, int]] = {}
    waiting: deque[int] = deque()
    lat = np.zeros(n)
    status = np.zeros(n, np.int32)
    frames_done = 0
    i = 0
    t0 = time.perf_counter()
    while i < n or pending or waiting:
        now = time.perf_counter() - t0
        did = False
        while i < n and arrivals[i] <= now:
            waiting.append(i)
            i += 1
        while waiting:
            j = waiting[0]
            req = make_request(j)
            if req is None:
                break
            waiting.popleft()
            tk = server.submit(req.frames, req.target_W, req.target_H, req.k, req.out)
            pending[tk] = (j, arrivals[j], req.frames.shape[0])
            did = True
        server.progress(wait=False)
        done = server.poll()
        t_done = time.perf_counter() - t0
        for tk, st in done:
            j, a, T = pending.pop(tk)
            lat[j] = t_done - a
            status[j] = st
            if st == scpl.SCPL_OK:
                frames_done += T
            if on_complete is not None:
                on_complete(j, st)
            did = True
        if not did:
            if i < n and not pending and not waiting:
                time.sleep(max(0.0, min(arrivals[i] - now, 0.01)))
            else:
                time.sleep(idle_sleep)
    elapsed = time.perf_counter() - t0
    ok = status == scpl.SCPL_OK
    return {"requests": n, "failed": int((~ok).sum()), "frames": int(frames_done),
            "elapsed_s": elapsed,
            "frames_per_s": frames_done / elapsed if elapsed > 0 else 0.0,
            "p50_ms": float(np.percentile(lat[ok], 50) * 1e3) if ok.any() else None,
            "p99_ms": float(np.percentile(lat[ok], 99) * 1e3) if ok.any() else None,
            "mean_ms": float(lat[ok].mean() * 1e3) if ok.any() else None}
