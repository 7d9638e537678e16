"""Host logic of bench.py: the roofline entry picks the dominant single kernel, scales the
measured DRAM traffic to its launches only while the step kernel's sources still hash to the
capture's, and the argument parser offers every workload."""
import sys

import pytest

import bench


def _prof():
    return [
        {"name": "fd2_step[CGP|SMP]", "launches": 100, "cells": 100 * 3088656,
         "bytes_per_cell": 28.0, "ms": 1.5},
        {"name": "fd2_step[PT|AP]", "launches": 100, "cells": 100 * 3088656,
         "bytes_per_cell": 24.0, "ms": 1.4},
        {"name": "pc_net", "launches": 13, "cells": 10 ** 9, "bytes_per_cell": 1.5, "ms": 9.0},
    ]


def test_roofline_of_takes_the_dominant_single_kernel():
    r = bench.roofline_of(_prof(), {"hbm_gbs": 6000.0})
    assert r["kernel"] == "fd2_step[CGP|SMP]"            # pc_net groups 13 launches
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak_source"] == "measured"
    assert r["per_launch_us"] == pytest.approx(15.0)
    assert r["achieved"] == pytest.approx(28.0 * 3088656 / 15e-6 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6000.0)
    assert r["share"] == pytest.approx(1.5 / 11.9)
    assert bench.roofline_of(_prof(), {})["peak_source"] == "fallback"


def test_traffic_needs_the_capture_hash(monkeypatch):
    entry = _prof()[1]
    per_cell = bench.MEASURED_TRAFFIC["fd2_step[PT|AP]"][0]
    monkeypatch.setattr(bench, "_sources_sha", lambda: bench._SHA)
    assert bench.traffic_per_launch(entry) == pytest.approx(per_cell * 3088656)
    monkeypatch.setattr(bench, "_sources_sha", lambda: "another")
    assert bench.traffic_per_launch(entry) is None
    assert bench.traffic_per_launch({"name": "unknown", "cells": 1, "launches": 1}) is None


def test_parser_offers_every_workload(monkeypatch):
    for w in ("esi2d", "dft3d", "wri2d", "invert2d", "grad2d"):
        monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", w, "--no-compare"])
        a = bench.parse()
        assert a.workload == w and a.gpus == 1 and a.warmup >= 3


def test_roofline_of_concurrent_groups_and_the_whole_step():
    """With shot groups the per-launch rate is one group's (marked, no traffic scaling),
    and `step` divides the algorithmic bytes of every kernel by the step's device time."""
    prof = [{"name": "fd2_step[PT|AP]", "launches": 400, "cells": 4000, "bytes_per_cell": 28.0,
             "ms": 8.0},
            {"name": "cg_update", "launches": 4, "cells": 4000, "bytes_per_cell": 24.0, "ms": 3.0}]
    r1 = bench.roofline_of(prof, {"hbm_gbs": 1000.0}, 1, step_ms=5.0, steps=2)
    r4 = bench.roofline_of(prof, {"hbm_gbs": 1000.0}, 4, step_ms=5.0, steps=2)
    assert r1["achieved"] == r4["achieved"] == pytest.approx(4000 * 28 / 8e-3 / 1e9)
    assert "groups" not in r1 and r4["groups"] == 4 and r4["traffic"] is None
    step_bytes = (4000 * 28 + 4000 * 24) / 2
    assert r4["step"]["bytes_per_step"] == pytest.approx(step_bytes)
    assert r4["step"]["achieved"] == pytest.approx(step_bytes / 5e-3 / 1e9)
    assert r4["step"]["frac"] == pytest.approx(r4["step"]["achieved"] / 1000.0)
