"""The benchmark's reference arm (the FP64 oracle on a bounded sample) runs on
CPU and prints one JSON line with the contract's keys."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ["metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "dtype", "config", "cpu_baseline", "e2e"]:
        assert key in line
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1


def test_relaxation_rooflines_arithmetic():
    """The HBM and issue-rate rooflines of the bench line: achieved over peak,
    the peak from the unit counts and the clock, and the HBM peak from the
    measured file when present."""
    sys.path.insert(0, ROOT)
    import bench
    peak, src = bench.measured_hbm_gbs()
    assert peak > 0 and src in ("of measured", "of fallback")
    h = bench.hbm_roofline(2.0e9, 4.0e9, 0.5)
    assert abs(h["achieved_gbs"] - 4.0) < 1e-12 and abs(h["dram_gbs"] - 8.0) < 1e-12
    assert abs(h["frac"] - 4.0 / peak) < 1e-15
    assert "dram_gbs" not in bench.hbm_roofline(2.0e9, None, 0.5)
    i = bench.issue_roofline(1.0e12, 1.0, 2000.0)
    want = 148 * 4 * 2000e6 * 32 / bench.INSTR_PER_PULL
    assert abs(i["peak_pulls_per_s"] - want) < 1e-3 * want
    assert abs(i["frac"] - 1.0e12 / want) < 1e-12
