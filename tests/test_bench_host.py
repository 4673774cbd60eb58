"""Host logic of bench.py, without a GPU: the work and byte counts behind
`value` and `roofline`, the roofline arithmetic, the rule that `traffic` is
reported only while the kernel sources match the ncu capture, and the parsing
of the nvidia-smi clock samples behind `clocks`."""
import json
import math
import os
import shutil

import bench


def test_pair_flops_closed_form():
    # 2.5 N log2 N per real transform, two per pair: 1024^3 -> 2 * 2.5 * 2^30 * 30
    assert bench.pair_flops(1024, 1024, 1024) == 2 * 2.5 * 2 ** 30 * 30
    assert math.isclose(bench.pair_flops(64, 48, 32), 5.0 * 98304 * math.log2(98304))


def test_pass_bytes_counts_three_read_write_passes():
    # one transform: the z-pass reads the real array and writes the spectrum,
    # the y- and x-passes read and write the spectrum
    n0 = n1 = n2 = 1024
    c = n0 * n1 * (n2 // 2 + 1) * 8
    r = n0 * n1 * n2 * 4
    assert bench.pass_bytes(n0, n1, n2, 4) == r + c + 2 * c + 2 * c
    assert round(2 * bench.pass_bytes(n0, n1, n2, 4) / 1e9, 1) == 51.6  # per pair


def test_roofline_takes_the_slowest_pass():
    stats = [
        {"name": "r2c.z", "total_ms": 12.0, "launches": 10, "bytes_per_launch": 8.6e9},
        {"name": "c2r.x", "total_ms": 16.0, "launches": 10, "bytes_per_launch": 8.6e9},
    ]
    r = bench.roofline_from(stats, 6773.2, {"c2r.x": 8.54e9})
    assert r["kernel"] == "c2r.x"
    assert r["avg_launch_ms"] == 1.6
    assert math.isclose(r["achieved"], 8.6e9 / 1.6e-3 / 1e9, rel_tol=1e-4)
    assert math.isclose(r["frac"], r["achieved"] / 6773.2, rel_tol=1e-3)
    assert r["traffic"] == 8.54e9
    assert bench.roofline_from(stats, 6773.2, None)["traffic"] is None
    assert bench.roofline_from([], 6773.2, None) is None


def test_traffic_only_while_sources_match(tmp_path, monkeypatch):
    root = tmp_path / "repo"
    csrc = root / "paper_2202_12756_gb300" / "csrc"
    shutil.copytree(os.path.join(bench.ROOT, "paper_2202_12756_gb300", "csrc"), csrc,
                    ignore=shutil.ignore_patterns("*.o", "*.so"))
    (root / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(root))
    h = bench.kernel_sources_hash()
    assert h == bench.kernel_sources_hash()  # deterministic
    per_pass = {"c2r.x": 8.54e9}
    (root / "profiles" / "ncu_traffic.json").write_text(
        json.dumps({"kernel_hash": h, "workloads": {"1024x1024x1024 f32": per_pass}}))
    assert bench.ncu_traffic("1024x1024x1024 f32") == per_pass
    assert bench.ncu_traffic("another workload") is None
    f = csrc / "pass_kernels.cuh"
    f.write_text(f.read_text() + "\n// edited\n")
    assert bench.kernel_sources_hash() != h
    assert bench.ncu_traffic("1024x1024x1024 f32") is None  # kernels changed since the capture


def test_clock_samples_median_and_reasons():
    class Proc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    class Thread:
        def join(self, timeout=None):
            pass

    s = bench.ClockSampler(0)
    s.proc, s.t = Proc(), Thread()
    # index, clocks.sm, clocks.max.sm, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    s.lines = [
        "0, 2070, 2070, 950.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2070, 2070, 990.4, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1980, 2070, 1001.0, 0x4, Not Active, Not Active, Not Active, Active",
        "garbage line",
    ]
    c = s.stop()
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    s2 = bench.ClockSampler(0)
    s2.proc, s2.t = Proc(), Thread()
    s2.lines = ["0, 1500, 2070, 500.0, 0x40, Active, Not Active, Not Active, Not Active"]
    assert s2.stop()["reasons"] == ["hw_slowdown"]


def test_reference_arm_labels_what_it_times():
    """The reference arm times the FP64 oracle on a small grid; its `config`
    must name that grid and dtype, matching its cpu_baseline sample."""
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
                        "--ref-n", "32", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, timeout=300, cwd=bench.ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    cfg = line["config"]
    assert cfg["grid"] == [32, 32, 32] and cfg["dtype"] == "f64" == line["dtype"]
    assert "32x32x32" in cfg["workload"] and "FP64" in cfg["workload"]
    assert "32^3" in line["cpu_baseline"]["sample"] and "FP64" in line["cpu_baseline"]["sample"]
    assert "1024" not in json.dumps(cfg)  # not the GPU arm's workload
    assert line["e2e"]["value"] == line["value"]


def test_fp64_roofline_arithmetic():
    stats = [{"name": "r2c.z", "total_ms": 80.0, "launches": 2, "bytes_per_launch": 1.0},
             {"name": "c2r.x", "total_ms": 62.0, "launches": 2, "bytes_per_launch": 1.0}]
    peak = {"fma_gflops": 1200.0, "add_gflops": 590.0, "mul_gflops": 600.0}
    ops = {"r2c.z": {"dadd": 30.0, "dmul": 6.0, "dfma": 4.0}}
    units = 1024 * 1024 * 513  # complex elements of one 1024^3 pass
    r = bench.fp64_roofline(stats, ops, peak, units)
    assert r["kernel"] == "r2c.z" and r["avg_launch_ms"] == 40.0
    assert r["peak"] == 600.0  # FP64 instructions/s: the best of FMA (1200 / 2), add and multiply
    assert math.isclose(r["achieved"], 40.0 * units / 40e-3 / 1e9, rel_tol=1e-3)
    assert math.isclose(r["frac"], r["achieved"] / 600.0, rel_tol=1e-3)
    assert math.isclose(r["achieved_gflops"], 44.0 * units / 40e-3 / 1e9, rel_tol=1e-3)
    # op counts unknown (kernels changed since they were counted): no fraction
    r2 = bench.fp64_roofline(stats, None, peak, units)
    assert r2["achieved"] is None and r2["frac"] is None and r2["peak"] == 600.0
    assert bench.fp64_roofline([], ops, peak, units) is None


def test_copy_streams_that_fit(tmp_path):
    """The copy-engine end-to-end runs lock (streams + 1) host fields per rank
    and stay within half of MemAvailable."""
    gib = 1024 ** 3
    info = tmp_path / "meminfo"
    info.write_text("MemTotal:       999999999 kB\nMemAvailable:   %d kB\n" % (200 * 1024 * 1024))
    field = 4 * gib  # one dense 1024^3 FP32 field
    assert bench.copy_streams_that_fit(field, 1, str(info)) == 3    # 16 GiB <= 100 GiB
    assert bench.copy_streams_that_fit(field, 8, str(info)) == 2    # 128 GiB > 100, 96 GiB fits
    assert bench.copy_streams_that_fit(field, 16, str(info)) == 0   # neither fits
    assert bench.copy_streams_that_fit(field, 1, str(tmp_path / "missing")) == 2
    assert bench.io_bytes_of((1024, 1024, 1024)) == field
