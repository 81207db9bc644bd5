"""The reference arm of bench.py runs on any host (it times the oracle) and prints one JSON line
with the contract's keys; its metric, unit and direction match the headline's."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["unit"] == "cell-updates/s" and d["dtype"] == "f64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    import bench
    assert d["config"] == bench.workload_config(1)      # the headline arm reports the same config


def test_reference_arm_under_torchrun_prints_once_from_rank_zero():
    """Launched as a two-rank job, rank 0 alone times the oracle and prints the line; the other
    rank exits 0 without work."""
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                          "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
                          "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0


def test_clock_samples_summary():
    """The timed region's clock record: median SM clock, the maximum, and every throttle reason
    seen Active in any sample (the reasons a run is rejected for, and sw_power_cap, which is kept
    and noted)."""
    import bench
    rows = ["0, 1965, 2070, 1010.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 1980, 2070, 1050.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, 2010, 2070, 990.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "garbage line"]
    d = bench.parse_clock_samples(rows)
    assert d == {"sm_mhz": 1980.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    hot = rows[:1] + ["0, 1200, 2070, 900.0, 0x0000000000000040, Not Active, Active, Not Active, Not Active"]
    assert bench.parse_clock_samples(hot)["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert bench.parse_clock_samples([])["samples"] == 0


def test_summary_carries_every_config_headline():
    """The line's last key condenses configs 1-4 (a truncated log keeps the end of the line)."""
    import bench
    line = {"value": 4.2e6, "roofline": {"frac": 0.37},
            "extras": {"ch4_les": {"cell_updates_per_s": 3.1e5, "fp64_frac_plain": 0.26, "fp64_frac_folded": 0.34},
                       "surrogate": {"surrogate_cell_updates_per_s": 2.6e8, "speedup_vs_fp64": 58.0,
                                     "hrr_l1_rel_error_vs_fp64": 0.0048, "tensor_frac_of_burst": 0.31},
                       "serving": {"p50_ms": 12.0, "p99_ms": 40.0, "cell_updates_per_s": 4e6}}}
    sm = bench.summary(line)
    assert sm["cfg2_fp64_frac_plain"] == 0.26 and sm["cfg2_fp64_frac_folded"] == 0.34
    assert sm["cfg3_speedup_vs_fp64"] == 58.0 and sm["cfg3_hrr_l1_rel_error"] == 0.0048
    assert sm["cfg4_p99_ms"] == 40.0 and sm["cfg1_h2_cells_per_s"] == 4.2e6
    assert len(json.dumps(sm)) < 700
    assert bench.summary({"value": 1.0, "roofline": {"frac": 0.1}})["cfg2_ch4_cells_per_s"] is None
