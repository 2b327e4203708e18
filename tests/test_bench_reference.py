"""The reference arm of bench.py (`--impl reference`) times the oracle on the
host cores and prints one JSON line with the same metric, unit and workload as
the library's arm.  It needs no GPU, so its line is checked here on a small
workload: the keys the line must carry, an e2e object equal to the line's own
value with no host-device copies, and a cpu_baseline that says what it timed."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("warmup", [1, 0])
def test_reference_arm_prints_the_contract_line(orc, warmup):
    out = subprocess.run(
        [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "cube8_2lvl",
         "--steps", "2", "--warmup", str(warmup)],
        cwd=ROOT, capture_output=True, text=True, timeout=600, env=dict(os.environ, RANK="0"))
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    d = json.loads(lines[0])
    import bench
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["impl"] == "reference" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == warmup
    assert d["config"]["workload"] == "cube8_2lvl"
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    if warmup >= 1:  # the first warm-up step is one whole oracle solve, whose iterations the samples use
        assert d["full_solve"]["iterations"] == d["iterations_used"] >= 1
        assert d["full_solve"]["rel_residual"] <= 1e-8
    else:
        assert d["full_solve"] is None


def test_reference_arm_other_ranks_exit_quietly(orc):
    """Under torchrun only rank 0 runs the reference arm; the others exit 0
    without work and print nothing."""
    out = subprocess.run(
        [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "cube8_2lvl",
         "--steps", "1", "--warmup", "0"],
        cwd=ROOT, capture_output=True, text=True, timeout=600, env=dict(os.environ, RANK="1"))
    assert out.returncode == 0, out.stderr[-2000:]
    assert not [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
