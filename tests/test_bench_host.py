"""Host logic of bench.py (no GPU): the workload sizes of the benchmark
configurations, the roofline's operation count, and the rule that a recorded
DRAM traffic figure stands only while its kernel's sources are unchanged."""
import json
import os

import pytest

import bench
from paper_2304_03311_gb300 import workloads as wl


@pytest.mark.parametrize("config,jobs,updates", [
    (1, 1, 1000 * 2 * 16 * 16 * (1000 + 200 * 1)),
    (2, 31, 31 * 16384 * 2 * 64 * 64 * (1000 + 1000 * 2)),
    (3, 8, 8 * 4096 * 2 * 16 * 16 * 16 * (1000 + 2000 * 1)),
])
def test_workload_sizes(config, jobs, updates):
    """Spin updates per launch: n_traj x V x (n_therm + N n_sweep) summed over
    the transformations (V counts both replicas)."""
    w = wl.CONFIGS[config]()
    assert len(w.jobs) == jobs
    assert w.updates == updates


def test_uneven_batch_is_charged_per_dimension():
    w = wl.CONFIGS[4]()
    total, per = bench.algorithmic_ops(w.jobs, sw=False)
    two = sum(j.updates for j in w.jobs if j.d == 2)
    three = sum(j.updates for j in w.jobs if j.d == 3)
    assert two > 0 and three > 0 and two + three == w.updates
    assert total == bench.N_ALG[2] * two + bench.N_ALG[3] * three
    assert per == {"2D": bench.N_ALG[2], "3D": bench.N_ALG[3]}


def test_single_dimension_reports_one_figure():
    w = wl.CONFIGS[3]()
    total, per = bench.algorithmic_ops(w.jobs, sw=False)
    assert per == bench.N_ALG[3] and total == bench.N_ALG[3] * w.updates
    total, per = bench.algorithmic_ops(w.jobs, sw=True)
    assert per == bench.N_ALG_SW[3] and total == bench.N_ALG_SW[3] * w.updates


def test_recorded_traffic_stands_only_for_unchanged_sources(tmp_path, monkeypatch):
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "dram_traffic.json")))
    for workload, r in rec["launches"].items():
        kernel = next(k for k, srcs in bench.KERNEL_SOURCES.items()
                      if list(srcs) == r["sources"] and r["kernel"].startswith(k))
        if r["source_sha256"] == bench.kernel_source_hash(kernel):
            assert bench.traffic_from_profile(kernel, workload) == r["dram_bytes_per_launch"]
    # a record whose hash does not match the sources is not reported
    fake_root = tmp_path
    (fake_root / "profiles").mkdir()
    bad = {"launches": {"w": {"kernel": "traj_kernel", "dram_bytes_per_launch": 1,
                              "sources": list(bench.KERNEL_SOURCES["traj_kernel"]),
                              "source_sha256": "0" * 64}}}
    (fake_root / "profiles" / "dram_traffic.json").write_text(json.dumps(bad))
    real_hash = bench.kernel_source_hash("traj_kernel")
    monkeypatch.setattr(bench, "ROOT", str(fake_root))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda k: real_hash)
    assert bench.traffic_from_profile("traj_kernel", "w") is None
    assert bench.traffic_from_profile("traj_kernel", "other") is None


def test_pulls_of_identical_and_shifted_scans():
    ref = [(0.1 * l, 0.01) for l in range(31)]
    same = bench.pulls(ref, ref)
    assert same["max_abs_pull"] == 0 and same["chi2_per_l"] == 0 and same["passes"]
    # every l high by 4 combined standard deviations: the check must fail
    shifted = [(v + 4 * 0.01 * 2 ** 0.5, e) for v, e in ref]
    bad = bench.pulls(shifted, ref)
    assert abs(bad["mean_pull"] - 4) < 1e-9 and not bad["passes"]


def test_fractions_against_the_three_ceilings():
    ceil = {"derived_int_ops_per_s": 40e12, "probe_mix_int_ops_per_s": 36e12,
            "philox_update_ceiling_per_s": 2e12}
    f = bench.fractions(20e12, 1e12, ceil)
    assert f == {"frac_derived": 0.5, "frac_probe": 20 / 36, "frac_philox_ceiling": 0.5}


def test_swendsen_wang_start_option_marks_every_job():
    """--therm-update 1 --n-therm 100: every job of the scan starts from
    Swendsen-Wang thermalisation, the workload's name says so, and a
    Swendsen-Wang scan ignores the option (its start is already one)."""
    w = bench.workload_for(2, 0, n_therm=100, therm_update=1)
    assert all(j.therm_update == 1 and j.n_therm == 100 and j.update == 0 for j in w.jobs)
    assert w.name.endswith("_therm100_swtherm")
    s = bench.workload_for(2, 0, update="sw", therm_update=1)
    assert all(j.therm_update == 0 and j.update == 1 for j in s.jobs)
    plain = bench.workload_for(2, 0)
    assert all(j.therm_update == 0 for j in plain.jobs)
    # rank 1 of a weak-scaling run owns the next trajectory range of every job
    r1 = bench.workload_for(2, 1, therm_update=1)
    assert all(a.traj0 == b.traj0 + b.n_traj for a, b in zip(r1.jobs, w.jobs))
