"""Host logic of bench.py, on CPU: the clock record taken from nvidia-smi's
CSV, the rank reduction at one rank, the serving HK-PR degree, and the
reference arm's JSON line (the oracle timed on a small R-MAT)."""
import argparse
import json
import math
import os
import time

import pytest

import bench


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.proc = _FakeProc()
    s.lines = list(lines)
    return s


def test_clock_record_median_max_and_reasons():
    na, act = "Not Active", "Active"
    lines = [
        f"0, 1965, 2070, 900.1, 0x0, {na}, {na}, {na}, {na}",
        f"0, 1980, 2070, 1100.4, 0x4, {na}, {na}, {na}, {act}",
        f"0, 1995, 2070, 1200.0, 0x4, {na}, {na}, {na}, {act}",
        "0, [N/A], 2070, 0, 0x0, N/A, N/A, N/A, N/A",      # unreadable sample: skipped
        "garbage",                                          # short line: skipped
    ]
    rec = _sampler(lines).stop()
    assert rec["sm_mhz"] == 1980 and rec["sm_max_mhz"] == 2070
    assert rec["reasons"] == ["sw_power_cap"] and rec["samples"] == 3


def test_clock_record_flags_slowdowns():
    act, na = "Active", "Not Active"
    rec = _sampler([f"0, 900, 2070, 1400, 0x8, {act}, {act}, {na}, {na}"]).stop()
    assert rec["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]


def test_clock_record_without_nvidia_smi():
    rec = bench.ClockSampler(0).stop()
    assert rec["sm_mhz"] is None and rec["reasons"] == ["nvidia-smi unavailable"]


def test_reduce_ranks_is_identity_on_one_rank():
    assert bench.reduce_ranks([1.5, 2.0], [3.0], 1, "cpu") == ([1.5, 2.0], [3.0])


def test_hk_terms_tail_bound():
    for t, eps in [(10.0, 1e-7), (5.0, 1e-4), (1.0, 1e-9)]:
        N = bench.hk_terms(t, eps)
        tail = 1.0 - sum(math.exp(-t) * t ** k / math.factorial(k) for k in range(N + 1))
        assert tail <= eps * 1.0001
        prev = 1.0 - sum(math.exp(-t) * t ** k / math.factorial(k) for k in range(N))
        assert N == 1 or prev > eps


def test_reference_arm_line(monkeypatch, capsys):
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.setattr(bench, "SCALE", 11)
    args = argparse.Namespace(gpus=1, steps=4, warmup=1)
    assert bench.run_reference(args) == 0
    out = capsys.readouterr().out.strip().splitlines()
    assert len(out) == 1
    line = json.loads(out[0])
    assert line["impl"] == "reference" and line["metric"] == "pushed_edges_per_s"
    assert line["value"] > 0 and line["unit"] == "edges/s"
    assert line["steps"] == 4 and line["warmup"] == 1 and line["n_gpus"] == 1
    assert line["higher_is_better"] is True and line["vs_baseline"] is None
    assert line["ms_per_step"] > 0 and line["data"] == "synthetic"
    assert "workload" in line["config"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_do_no_work(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    def boom(*a, **k):
        raise AssertionError("rank 1 must not run the oracle")

    monkeypatch.setattr(bench, "cpu_oracle_step", boom)
    assert bench.run_reference(argparse.Namespace(gpus=2, steps=1, warmup=0)) == 0
    assert capsys.readouterr().out == ""


def _fake_smi(tmp_path, body):
    d = tmp_path / "bin"
    d.mkdir()
    f = d / "nvidia-smi"
    f.write_text("#!/bin/sh\n" + body)
    f.chmod(0o755)
    return str(d)


def test_clock_sampler_counts_only_samples_inside_the_region(tmp_path, monkeypatch):
    line = "0, 2070, 2070, 500.0, 0x0, Not Active, Not Active, Not Active, Not Active"
    path = _fake_smi(tmp_path, f'while true; do echo "{line}"; sleep 0.05; done\n')
    monkeypatch.setenv("PATH", path + os.pathsep + os.environ["PATH"])
    s = bench.ClockSampler(0)
    s.start()
    assert s.mark >= 1                        # returned after the first sample
    time.sleep(0.4)
    rec = s.stop()
    assert rec["sm_mhz"] == 2070 and rec["reasons"] == []
    assert 2 <= rec["samples"] == len(s.lines) - s.mark


def test_clock_sampler_region_shorter_than_the_period(tmp_path, monkeypatch):
    line = "0, 1980, 2070, 500.0, 0x4, Not Active, Not Active, Not Active, Active"
    path = _fake_smi(tmp_path, f'echo "{line}"; exec sleep 30\n')
    monkeypatch.setenv("PATH", path + os.pathsep + os.environ["PATH"])
    s = bench.ClockSampler(0)
    s.start()
    rec = s.stop()                            # no sample inside: the one just before
    assert rec["samples"] == 0 and rec["sm_mhz"] == 1980 and rec["reasons"] == ["sw_power_cap"]


def test_clock_sampler_does_not_wait_for_a_dead_nvidia_smi(tmp_path, monkeypatch):
    path = _fake_smi(tmp_path, "exit 9\n")
    monkeypatch.setenv("PATH", path + os.pathsep + os.environ["PATH"])
    s = bench.ClockSampler(0)
    t0 = time.perf_counter()
    s.start(wait_s=20.0)
    assert time.perf_counter() - t0 < 5.0
    rec = s.stop()
    assert rec["sm_mhz"] is None and rec["samples"] == 0


def test_cpu_all_cores_counts_completed_clusters():
    """The all-cores oracle baseline: forked workers split the work list,
    the parent counts what completed within the budget."""
    from paper_1604_07515_gb300 import inputs
    off, col = inputs.rmat(10, seed=4)
    seeds, eps = bench.many_seed_list(inputs, off)
    items = [("pr", int(s), dict(alpha=0.01, eps=float(e))) for s, e in zip(seeds[:24], eps[:24])]
    bench._SHARED["t"] = (off, col, items)
    try:
        rec = bench.cpu_all_cores("t", 30.0)
    finally:
        bench._SHARED.clear()
    assert rec["clusters"] == 24 and rec["unfinished_workers"] >= 0
    assert rec["cores"] == (os.cpu_count() or 1) and rec["clusters_per_s"] > 0
    assert rec["edges_per_s"] > 0 and rec["per_cluster_s_mean"] > 0


def test_serving_mix_shape():
    from paper_1604_07515_gb300 import inputs
    off, col = inputs.rmat(10, seed=4)
    mix = bench.serving_mix(inputs, off, 500)
    kinds = [k for k, _, _ in mix]
    assert 0.7 < kinds.count("pr") / 500 < 0.9
    d = inputs.degrees(off)
    assert all(d[s] >= 2 for _, s, _ in mix)
    for k, _, prm in mix:
        if k == "hkpr":
            assert 3.0 <= prm["t"] <= 30.0 and prm["eps"] == 1e-7
            assert prm["N"] == bench.hk_terms(prm["t"], 1e-7)
        else:
            assert 1e-8 <= prm["eps"] <= 1e-5 and prm["alpha"] == 0.01


def test_occupancy_from_request_times():
    res = [dict(submit_s=0.0, start_s=0.0, end_s=2.0), dict(submit_s=1.0, start_s=2.0, end_s=3.0),
           dict(submit_s=1.5, start_s=2.5, end_s=4.0)]
    occ = bench.occupancy(res, None)
    # at t=0: 1 admitted, 0 queued; t=1: 1 admitted, 1 queued; t=1.5: 1 admitted, 2 queued
    assert occ["queued_max"] == 2 and occ["admitted_max"] == 1
    assert abs(occ["queued_mean"] - 1.0) < 1e-12


def test_pull_traffic_stretches_are_found_and_keys_well_formed():
    """The source stretches whose hash ties the recorded gather traffic to
    the kernels are all found (a moved marker would silently null the
    figure), and every configuration key is 'bin,batch,lanes,share'."""
    sha = bench.sources_sha(bench.PULL_TRAFFIC["sources"])
    assert sha is not None and len(sha) == 64
    for key, v in bench.PULL_TRAFFIC["per_round"].items():
        parts = [int(x) for x in key.split(",")]
        assert len(parts) == 4 and parts[3] in (8, 16) and v > 0
