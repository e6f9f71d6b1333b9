"""Host logic of bench.py (no GPU): the reference arm's JSON line carries
every key of the benchmark contract, and the clock sampler's parser finds
the median SM clock and the throttle reasons that reject a run."""
import json
import subprocess
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
sys.path.insert(0, str(ROOT))

import bench  # noqa: E402


def test_reference_arm_line_has_the_contract_keys():
    r = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.strip().splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["unit"] == "walks/s" and d["higher_is_better"] is True
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"],
                        "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


@pytest.mark.parametrize("rows, want", [
    ([("2070", "2070", "Not Active", "Not Active", "Not Active", "Not Active")] * 3,
     {"sm_mhz": 2070.0, "reasons": []}),
    ([("1980", "2070", "Not Active", "Not Active", "Not Active", "Active"),
      ("2010", "2070", "Not Active", "Not Active", "Not Active", "Not Active"),
      ("1995", "2070", "Not Active", "Not Active", "Not Active", "Active")],
     {"sm_mhz": 1995.0, "reasons": ["sw_power_cap"]}),
    ([("1500", "2070", "Active", "Not Active", "Active", "Not Active"),
      ("1600", "2070", "Not Active", "Not Active", "Not Active", "Not Active")],
     {"sm_mhz": 1550.0, "reasons": ["hw_slowdown", "sw_thermal_slowdown"]}),
])
def test_clock_samples_are_parsed(tmp_path, rows, want):
    csv = tmp_path / "clocks.csv"
    # nvidia-smi --format=csv,noheader,nounits: index, clocks.sm, clocks.max.sm,
    # power.draw, clocks_event_reasons.active, hw_slowdown, hw_thermal_slowdown,
    # sw_thermal_slowdown, sw_power_cap
    csv.write_text("".join(f"0, {sm}, {mx}, 812.40, 0x0000000000000000, {a}, {b}, {c}, {p}\n"
                           for sm, mx, a, b, c, p in rows) + "garbage line\n")
    s = bench.ClockSampler(0)
    s.path, s.proc = csv, _Done()
    got = s.stop()
    assert got["sm_mhz"] == want["sm_mhz"]
    assert got["sm_max_mhz"] == 2070.0
    assert got["reasons"] == want["reasons"]
    assert got["samples"] == len(rows)
    assert csv.exists()  # a caller's file is kept


def test_clock_sampler_without_nvidia_smi_reports_nothing():
    s = bench.ClockSampler(0)
    s.proc = None
    assert s.stop() is None


def test_svd_fp64_flop_accounts_for_the_preconditioned_path():
    """The SVD roofline's FP64 flop: QR 2mn^2 - 2n^3/3; above 256 and up to
    768 columns (FP32 sweeps first, unless FP64 sweeps alone are asked for)
    the Newton-Schulz and X Q products 4n^3; FP64 sweeps n(n-1)/2 pair
    visits of 6 flop a row of X (n rows)."""
    import bench
    m, n, sw = 1024, 768, 2
    qr = 2 * m * n * n - (2 * n ** 3) // 3
    sweeps = sw * (n * (n - 1) // 2) * 6 * n
    assert bench.fp32_preconditioned(n, "auto") and not bench.fp32_preconditioned(n, "fp64-sweeps")
    assert not bench.fp32_preconditioned(256, "auto") and not bench.fp32_preconditioned(769, "auto")
    assert bench.svd_fp64_flop(m, n, sw, "auto") == qr + 4 * n ** 3 + sweeps
    assert bench.svd_fp64_flop(m, n, sw, "fp64-sweeps") == qr + sweeps
    # small problems: V accumulated, no Newton-Schulz
    assert bench.svd_fp64_flop(256, 128, 9, "auto") == (
        2 * 256 * 128 ** 2 - (2 * 128 ** 3) // 3 + 9 * (128 * 127 // 2) * (12 * 128 + 6 * 128))
