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
