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
    assert t, "no traffic entries"
    for key, ent in t.items():
        monkeypatch.setattr(bench, "kernel_source_hash", lambda h=ent["source_hash"]: h)
        assert bench.load_traffic(key) == pytest.approx(ent["dram_bytes_per_launch_full"])
        monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
        assert bench.load_traffic(key) is None
    assert bench.load_traffic("no_such_kernel") is None


def test_traffic_is_recorded_from_an_ncu_launch_list(tmp_path, monkeypatch):
    """An ncu --csv launch list of one 48^6 step: each pass's DRAM bytes per
    launch, the two drift launches of one kernel told apart by their order."""
    rows = ['"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"']
    names = ["k_drift_fast<float, 48, 1, 0>(...)", "k_drift_fast<float, 48, 1, 0>(...)",
             "k_drift_fast<float, 48, 1, 1>(...)", "k_kick_pass_a<48>(...)",
             "k_kick_pass_b<48>(...)", "k_kick_pass_c<48>(...)"]
    for i, n in enumerate(names):
        rows.append(f'"{i}","{n}","dram__bytes_read.sum","Gbyte","{10 + i}"')
        rows.append(f'"{i}","{n}","dram__bytes_write.sum","Mbyte","{500 + i}"')
        rows.append(f'"{i}","{n}","gpu__time_duration.sum","msecond","{2 + i}"')
    csv_path = tmp_path / "l.csv"
    csv_path.write_text("\n".join(rows) + "\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "ab" * 8)
    out = bench.record_traffic(str(csv_path), "w48")
    want = {"drift_z": 0, "drift_y": 1, "drift_x": 2, "kick_a": 3, "kick_b": 4, "kick_c": 5}
    for slot, i in want.items():
        e = out[f"w48:{slot}"]
        assert e["dram_bytes_per_launch_full"] == pytest.approx((10 + i) * 1e9 + (500 + i) * 1e6)
        assert e["duration_us_under_ncu"] == pytest.approx((2 + i) * 1e3)
        assert e["source_hash"] == "ab" * 8


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
    rate, full, desc, measured = bench.oracle_step_rate(w, f0, 0.25)
    assert rate > 0 and full > 0 and measured > 0
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
    rate, full, desc, _ = bench.oracle_step_rate(w, f0, 0.25, rho)
    assert rate > 0 and "density timed on 2 of 8 x planes" in desc


def test_samples_from_the_factors_equal_the_initial_condition():
    """The oracle's samples of a separable initial condition are built from
    its two factors without a host copy of f: the same values."""
    import numpy as np
    w = I.small_maxwell(n=(8, 4, 4), nv=(8, 6, 4), dtype="f64", amp=0.2)
    f0 = I.initial_condition(w)
    src = bench.HostSource(w)
    assert np.array_equal(src.planes(2, 5), f0[2:5])
    assert np.array_equal(src.vcols(3), f0[:, :, :, :3])
    np.testing.assert_allclose(src.density(), bench.oracle_density(w, f0), rtol=1e-13)


def test_cores_are_the_oracles_openmp_threads():
    from oracle import vp_oracle as O
    n = bench.oracle_threads()
    assert n == O.threads() and 1 <= n <= (os.cpu_count() or n)


@pytest.mark.parametrize("big_kick,fused_yz", [(True, False), (True, True), (False, False),
                                               (False, True)])
def test_roofline_passes_follow_the_profiled_step(big_kick, fused_yz, monkeypatch):
    """The roofline's passes are the step's own: the three slab passes of
    the 48^3 kick or the one-pass kick, the fused z+y drift where the z slot
    holds both drifts (the y slot then empty) or the two separate drifts, and
    the x drift; the dominant kernel is the longest pass, the step fraction
    counts one read and one write of f per pass."""
    monkeypatch.setattr(bench, "load_peaks", lambda: (1000.0, "measured"))
    monkeypatch.setattr(bench, "load_traffic", lambda key: None)
    w = I.WORKLOADS["jeans48_modes8"]() if big_kick else I.WORKLOADS["jeans32_f32"]()
    avg = {"kick6": 30.0, "drift_z": 10.0, "drift_y": 0.001 if fused_yz else 9.0, "drift_x": 8.0,
           "density": 0.0, "field": 0.3, "tables": 0.2, "step": 0.0,
           "kick_a": 12.0 if big_kick else 0.0, "kick_b": 9.5 if big_kick else 0.0,
           "kick_c": 9.0 if big_kick else 0.0}
    if not big_kick:
        avg["kick6"] = 11.0
    kick = ["kick_a", "kick_b", "kick_c"] if big_kick else ["kick6"]
    drift = ["drift_yz", "drift_x"] if fused_yz else ["drift_z", "drift_y", "drift_x"]
    avg["step"] = sum(avg[k] for k in kick) + sum(avg.get(k, avg["drift_z"]) for k in drift) + 0.5
    r = bench.roofline_of(w, avg, 4)
    assert list(r["passes"]) == kick + drift
    longest = "kick_a" if big_kick else "kick6"
    assert r["pass"] == longest
    bytes_rw = 2 * w.cells * 4
    assert r["achieved"] == pytest.approx(bytes_rw / (avg[longest] / 1e3) / 1e9, rel=1e-3)
    assert r["step_bytes_algorithmic"] == len(kick + drift) * bytes_rw
    assert r["step_hbm_frac"] == pytest.approx(
        len(kick + drift) * bytes_rw / (avg["step"] / 1e3) / 1e9 / 1000.0, rel=1e-3)

