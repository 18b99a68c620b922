"""bench.py on the CPU: the reference arm's JSON line and the roofline arithmetic."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "4096",
                          "--steps", "1", "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_roofline_arithmetic():
    sys.path.insert(0, ROOT)
    import bench
    n = 1 << 20
    r = bench.roofline(1000.0, n, 152, {"sm_mhz": 1035.0}, {"sm_max_mhz": 2070.0})
    assert r["bound"] == "alu" and r["unit"] == "Gpair/s"
    assert abs(r["peak"] - 152 * 128 * 2.07e9 / 27 / 1e9) < 0.01
    assert abs(r["achieved"] - n * (n - 1) / 1e9) < 0.01
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-4
    assert abs(r["frac_at_sampled_clock"] - 2 * r["frac"]) < 1e-3


def test_traffic_record_matches_the_kernel_sources():
    """The committed ncu DRAM-traffic record of the benchmarked launch is keyed on the force kernel's code;
    it must match the sources as they stand, or the bench line reports no traffic."""
    sys.path.insert(0, ROOT)
    import bench
    for mode in ("plain", "comp"):
        t = bench.measured_traffic(mode, 1 << 20, [256, 1, 2])
        assert t is not None and t > 0, mode
