"""The golden digest files (tests/golden/*.json, written from the oracle by
tests/golden/make_digests.py) describe exactly the inputs the seeded
generator draws today, and are internally consistent.  CPU only."""
from __future__ import annotations

import json
import os

import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        pytest.skip(f"{name} has not been written")
    with open(path) as fh:
        return json.load(fh)


def _buffers_cover(starts, buffers, T):
    assert starts[0] == 0 and starts[-1] == T
    assert all(a < b for a, b in zip(starts, starts[1:]))
    assert [(b["t0"], b["t1"]) for b in buffers] == list(zip(starts, starts[1:]))


def test_clip_1080p_golden():
    g = _load("clip_1080p_300f.json")
    assert (g["T"], g["H"], g["W"], g["target"], g["k"]) == (300, 1080, 1920, 1344, 32)
    _buffers_cover(g["starts"], g["buffers"], g["T"])
    for b in g["buffers"]:
        # every iteration removes k_eff >= 1 seams, at most k; together the
        # W - target seams (Sec. 3.1: the loop runs until the target width)
        assert len(b["k_eff"]) == b["iterations"]
        assert all(1 <= x <= g["k"] for x in b["k_eff"])
        assert sum(b["k_eff"]) == g["W"] - g["target"]
        assert len(b["seams_sha256"]) == len(b["out_sha256"]) == 64
    # the scan's buffers never exceed t_max frames (Sec. 3.2 cap)
    assert max(b["t1"] - b["t0"] for b in g["buffers"]) <= g["t_max"]


def test_batch_golden_matches_the_generator():
    from paper_1903_03180_gb300 import synth
    g = _load("batch_256x32.json")
    specs = synth.batch_spec()
    assert len(g["clips"]) == len(specs) == 256
    for c, sp in zip(g["clips"], specs):
        for key in ("clip", "T", "H", "W", "target_W", "target_H", "k", "seed"):
            assert c[key] == sp[key], (c["clip"], key)
        assert c["starts"][0] == 0 and c["starts"][-1] == c["T"]


def test_serve_golden_matches_the_generator():
    from paper_1903_03180_gb300 import synth
    g = _load("serve_jobs20.json")
    specs = synth.serve_jobs()
    assert len(g["jobs"]) == len(specs) == 20
    for j, sp in zip(g["jobs"], specs):
        for key in ("job", "T", "H", "W", "target_W", "target_H", "k", "seed"):
            assert j[key] == sp[key], (j["job"], key)
        _buffers_cover(j["starts"], j["buffers"], j["T"])
        for b in j["buffers"]:
            assert b["iterations"] >= (j["W"] - j["target_W"] + j["k"] - 1) // j["k"]
