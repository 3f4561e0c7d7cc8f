"""Host-side logic of bench.py (no GPU): the time-to-accuracy reading of an iterate history,
the cost-model fit behind the oracle ladder, and the traffic lookup that is tied to the
profiled kernel source."""
import json
import math

import numpy as np

import bench


def test_first_crossing_takes_the_first_iterate_within_target():
    bh = np.array([1.0, -2.0, 2.0])  # norm 3
    hist = np.stack([bh + np.array([0.3, 0.0, 0.0]),     # rel. error 0.1
                     bh + np.array([0.0, 2.7e-8, 0.0]),  # 9e-9: the first within 1e-8
                     bh + np.array([0.0, 0.0, 3e-9]),
                     bh])
    ms = np.array([1.0, 2.5, 4.0, 5.0])
    t, err = bench.first_crossing(hist, ms, bh, 1e-8)
    assert t == 2.5
    assert math.isclose(err, 9e-9, rel_tol=1e-6)


def test_first_crossing_reports_the_last_error_when_never_reached():
    bh = np.array([3.0, 4.0])  # norm 5
    hist = np.stack([bh + 1.0, bh + np.array([0.5, 0.0])])
    t, err = bench.first_crossing(hist, np.array([1.0, 2.0]), bh, 1e-8)
    assert t is None
    assert math.isclose(err, 0.1)


def test_cost_model_fit_recovers_the_model_and_extrapolates():
    c, a, b = 0.7, 3e-7, 2e-6
    model = lambda n: c + a * n * math.log2(n) + b * n
    ns = [1 << k for k in (14, 15, 16, 17, 18)]
    fit = bench.cost_model_fit(ns, [model(n) for n in ns])
    for n in (1 << 19, 1 << 22):
        assert math.isclose(fit(n), model(n), rel_tol=1e-9)


def test_traffic_is_reported_only_for_the_profiled_source(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel A\n")
    import hashlib
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(
        json.dumps({"kern": {"source_sha256": sha, "dram_bytes_per_launch": 1234}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profile_traffic("kern", ["k.cu"]) == 1234
    assert bench.profile_traffic("other", ["k.cu"]) is None
    src.write_text("kernel B\n")  # the kernel changed since the counters were taken
    assert bench.profile_traffic("kern", ["k.cu"]) is None


def test_committed_traffic_entries_are_complete():
    # every entry of profiles/traffic.json names an existing source and a hash of it, and its
    # per-launch traffic is the captured read plus write bytes (a stale hash only makes the
    # bench report the traffic as null, which the lookup test above covers)
    import os
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        prof = json.load(f)
    assert prof
    for key, ent in prof.items():
        assert os.path.exists(os.path.join(bench.ROOT, ent["source"])), key
        assert len(ent["source_sha256"]) == 64, key
        assert ent["dram_bytes_per_launch"] == ent["captured_dram_read_bytes"] + ent["captured_dram_write_bytes"]
