"""Host-side parts of bench.py (no GPU): the committed DRAM-traffic profile
is read per stage and only for the sources it was taken from, the clock
sampler's summary, and the reference arm's JSON line."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _profile():
    path = os.path.join(ROOT, "profiles", "traffic_mid.txt")
    sha, rows = None, []
    for ln in open(path):
        p = ln.split()
        if not p or ln.startswith("#"):
            continue
        if p[0] == "csrc_sha256":
            sha = p[1]
        else:
            rows.append((p[0], int(p[2]) + int(p[3])))
    return sha, rows


def test_traffic_sums_each_stage_for_its_own_sources(monkeypatch):
    sha, rows = _profile()
    assert sha and rows
    monkeypatch.setattr(bench, "csrc_sha256", lambda: sha)
    for stage in ("support", "lists", "peel"):
        want = sum(b for s, b in rows if s == stage)
        assert want > 0 and bench.traffic_for(stage) == want
    assert sum(1 for s, _ in rows if s == "lists") == 2  # both list passes


def test_traffic_is_withheld_once_the_sources_change(monkeypatch):
    monkeypatch.setattr(bench, "csrc_sha256", lambda: "0" * 64)
    assert bench.traffic_for("peel") is None


def test_clock_summary_reports_median_max_and_active_reasons():
    cs = bench.ClockSampler(0)

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    cs.proc = Done()

    def row(mhz, power_cap):
        return ["0", str(mhz), "2070", "900.0", "0x0", "Not Active", "Not Active", "Not Active",
                power_cap]

    cs.rows = [row(2070, "Not Active"), row(1980, "Active"), row(2070, "Not Active"),
               ["garbled"]]
    out = cs.stop()
    assert out["sm_mhz"] == 2070 and out["sm_max_mhz"] == 2070
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3


@pytest.mark.timeout(600)
def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
