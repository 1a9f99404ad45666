"""Host logic of the benchmark that needs no GPU: the DRAM traffic it
reports comes only from ncu captures taken on the current kernel sources;
the peak comes from the measured-peaks file; the CPU baseline times the
oracle on a sample of the step and scales it by the sampled fractions."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1206_6152_gb300 import inputs as I  # noqa: E402


def test_traffic_is_reported_only_for_the_sources_it_was_measured_on(monkeypatch):
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        t = json.load(fh)
    for kernel in ("kick6", "drift_yz", "drift_x"):
        ent = t[kernel]
        monkeypatch.setattr(bench, "kernel_source_hash", lambda h=ent["source_hash"]: h)
        assert bench.load_traffic(kernel) == pytest.approx(ent["dram_bytes_per_launch_full"])
        monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
        assert bench.load_traffic(kernel) is None
    assert bench.load_traffic("no_such_kernel") is None


def test_kernel_source_hash_is_stable():
    h = bench.kernel_source_hash()
    assert len(h) == 16 and h == bench.kernel_source_hash()
    int(h, 16)


def test_peak_is_the_measured_hbm_copy_rate():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if not os.path.exists(path):                # not measured yet: the fallback figure
        assert bench.load_peaks() == (6800.0, "fallback")
        return
    with open(path) as fh:
        hbm = float(json.load(fh)["hbm_gbs"])
    assert bench.load_peaks() == (hbm, "measured")


def test_oracle_step_rate_scales_its_samples():
    w = I.small_maxwell(n=(8, 4, 4), nv=(8, 8, 8), dtype="f64", amp=0.2)
    f0 = I.initial_condition(w)
    rate, full, desc = bench.oracle_step_rate(w, f0, 0.25)
    assert rate > 0 and full > 0
    assert rate == pytest.approx(w.cells / full)
    # 2 of 8 x planes of velocity cubes and 2 of 8 vx columns of velocity cells
    assert "(0.2500)" in desc and desc.count("(0.2500)") == 2


def test_aggregate_is_cells_over_the_slowest_rank():
    class One:
        world = 1

        def max(self, x):
            return x
    ms, value = bench.aggregate(8.0, 1.0e9, 10, One())
    assert ms == 8.0 and value == pytest.approx(1.0e9 * 10 / 8e-3)


def test_reference_steps_sample_the_density():
    w = I.small_maxwell(n=(8, 4, 4), nv=(8, 8, 8), dtype="f64", amp=0.2)
    f0 = I.initial_condition(w)
    rho = bench.oracle_density(w, f0)
    assert rho.shape == tuple(w.n)
    rate, full, desc = bench.oracle_step_rate(w, f0, 0.25, rho)
    assert rate > 0 and "density timed on 2 of 8 x planes" in desc


def test_cores_are_the_oracles_openmp_threads():
    from oracle import vp_oracle as O
    n = bench.oracle_threads()
    assert n == O.threads() and 1 <= n <= (os.cpu_count() or n)
