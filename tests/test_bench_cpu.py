"""Host-side pieces of bench.py: the work counts behind the roofline, the
per-state-trial traffic figures, and the reference arm's JSON line (the
oracle on the host cores), none of which needs a GPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_work_counts_per_state():
    # one trial per state: 11 n^3 + 58 n^2 + 7 n FP64 flops (1,660 for n = 4);
    # one iteration per state outside the trials: 5 n^2 + 3 d_c^3 + 2 d_c^2 + 4 d_c
    assert bench.fp64_flops_per_trial_state(4) == 1660
    assert bench.fp64_flops_per_trial_state(14) == 11 * 14 ** 3 + 58 * 14 ** 2 + 7 * 14
    assert bench.fp64_flops_per_iter_state(4, 2) == 120


def test_traffic_per_state_trial_is_the_algorithmic_touch():
    """Both captured kernels move about one state's algorithmic touch per
    state-trial (both sweeps read five 4 x 4 blocks, the scratch is written and
    read back, the outputs are written: about 2.5 KB), i.e. no re-reads."""
    for b in (bench.LANE_DF_DRAM_BYTES_PER_STATE_TRIAL, bench.THREAD_F64_DRAM_BYTES_PER_STATE_TRIAL):
        assert 2000 < b < 2600
    assert bench.LANE_DF_MEASURED_EXPANSION > bench.DF_EXPANSION


def test_peaks_from_unit_counts():
    assert abs(bench.fp64_peak_tflops() - 1.202944) < 1e-9
    assert abs(bench.fp32_peak_tflops() - 76.988416) < 1e-9


@pytest.mark.timeout(600)
def test_reference_arm_prints_one_json_line():
    """`bench.py --impl reference` times the oracle on the host cores and prints
    the contract's line with impl = reference and no host-device traffic."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "plans/s" and d["value"] > 0
    assert d["metric"] == bench.METRIC and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
