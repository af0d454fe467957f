"""Host-side logic of bench.py (no GPU): the roofline arithmetic, the traffic table's
gating on the device sources, and the profiles it cites."""
import importlib.util
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_host", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_fp64_peak_falls_back_to_the_derived_dfma_rate(bench):
    assert bench.FP64_PEAK_DERIVED == pytest.approx(152 * 2 * 2 * 2.07)
    run = {"kernel_ms": np.array([1.0, 2.0, 3.0]), "timed": 10, "wet_fraction": 0.25,
           "active_cells": 123.0}
    r = bench.kernel_roofline(run, "fp64", "ll", 1_000_000, 7000.0, "measured")
    assert r["peak"] == pytest.approx(bench.FP64_PEAK_DERIVED) and "derived" in r["peak_source"]
    m = bench.kernel_roofline(run, "fp64", "ll", 1_000_000, 7000.0, "measured",
                              fp64={"gflops": 1000.0, "how": "test"})
    assert m["peak"] == 1000.0 and m["frac"] == pytest.approx(r["achieved"] / 1000.0)
    assert m["peak_source"].startswith("measured")


def test_alu_roofline_counts_wet_cells(bench):
    # three kernels' summed milliseconds over 10 timed steps; stage 2 dominates
    run = {"kernel_ms": np.array([1.0, 2.0, 3.0]), "timed": 10, "wet_fraction": 0.25,
           "active_cells": 123.0}
    r = bench.kernel_roofline(run, "fp64", "ll", 1_000_000, 7000.0, "measured",
                              fp64={"gflops": 1200.0, "how": "test"})
    per = bench.FLOPS_PER_WET_CELL["stage2"]["ll"]
    expect = per * 250_000 / (0.3e-3) / 1e9
    assert r["bound"] == "alu" and r["unit"] == "GFLOP/s"
    assert r["achieved"] == pytest.approx(expect)
    assert r["frac"] == pytest.approx(expect / 1200.0)
    assert r["kernel_ms"]["stage2"] == pytest.approx(0.3)


def test_hbm_roofline_counts_computed_cells(bench):
    run = {"kernel_ms": np.array([0.5, 4.0, 1.0]), "timed": 4, "wet_fraction": 0.1,
           "active_cells": 200_000.0}
    r = bench.kernel_roofline(run, "fp32", "nl", 2_000_000, 6000.0, "measured")
    per = bench.BYTES_PER_CELL["fp32"]["stage1"]["nl"]
    expect = per * 200_000 / (1.0e-3) / 1e9
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6000.0
    assert r["achieved"] == pytest.approx(expect)
    assert r["frac"] == pytest.approx(expect / 6000.0)


def test_traffic_is_gated_on_the_device_sources(bench):
    h = bench.device_src_hash()
    for (key, kernel), (nbytes, src, prof) in bench.TRAFFIC.items():
        assert nbytes > 0
        got = bench.traffic_of(key, kernel)
        assert got == ((nbytes, prof) if src == h else (None, None))
        # the cited summary exists, names its ncu command and the kernel's DRAM bytes
        text = open(os.path.join(ROOT, prof)).read()
        assert "ncu " in text and "--clock-control none" in text
        assert "dram__bytes_read.sum" in text
    assert bench.traffic_of("no_such_variant", "stage2") == (None, None)
