"""bench.py's host-side contract on CPU: the reference arm (the oracle timed on
the host cores) prints one JSON line with the keys the contract names, ranks
other than 0 print nothing, and the clock record summarises nvidia-smi's
samples (median SM clock, throttle reasons seen active)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

CMD = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
       "--workload", "sphere-2k", "--steps", "2", "--warmup", "1", "--cpu-seconds", "0.5"]


def _run(env_extra):
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    env.update(env_extra)
    return subprocess.run(CMD, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _run({})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert abs(d["value"] * d["ms_per_step"] * 1e-3 - d["config"]["queries"]) < 1e-6 * d["config"]["queries"]
    assert d["config"]["workload"] == "sphere-2k" and d["config"]["points"] == 2000
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert cb["unit"] == d["unit"] and "sample" in cb
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert d["vs_baseline"] is None


def test_reference_arm_other_ranks_do_no_work():
    r = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def _line(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return f"0, {sm}, {mx}, 900.5, 0x0000000000000000, {hw}, {hwt}, {swt}, {cap}"


def test_clock_summary_median_and_reasons():
    lines = [_line(2070, 2070), _line(1980, 2070, cap="Active"), _line(2070, 2070),
             "garbage", "", _line("[N/A]", 2070)]
    s = bench.ClockSampler.summarize(lines)
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "samples": 3,
                 "reasons": ["sw_power_cap"]}
    s = bench.ClockSampler.summarize([_line(1500, 2070, hw="Active", swt="Active")])
    assert s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.ClockSampler.summarize(["", "x"]) is None


def test_clock_sampler_stop_ends_its_process_and_summarises():
    cs = bench.ClockSampler.__new__(bench.ClockSampler)
    cs.proc = subprocess.Popen([sys.executable, "-c", "import time; time.sleep(60)"])
    cs.lines = [_line(2070, 2070), _line(2060, 2070, hwt="Active")]
    s = cs.stop()
    assert cs.proc.poll() is not None
    assert s["sm_mhz"] == 2065.0 and s["reasons"] == ["hw_thermal_slowdown"]


def test_clock_sampler_without_nvidia_smi_reports_nothing(monkeypatch):
    def refuse(*a, **k):
        raise FileNotFoundError("nvidia-smi")
    monkeypatch.setattr(bench.subprocess, "Popen", refuse)
    assert bench.ClockSampler("GPU-0").stop() is None


@pytest.mark.parametrize("world,per,steps,ms", [(1, 524288, 200, 500.0), (4, 1000, 3, 2.5)])
def test_job_throughput_is_all_units_over_slowest_span(world, per, steps, ms):
    assert bench.job_throughput(world, per, steps, ms) == pytest.approx(world * per * steps / (ms * 1e-3))
