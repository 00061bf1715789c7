"""bench.py's reference arm (the CPU FP64 oracle on the host cores) prints one JSON
line with the keys of the benchmark contract; under torchrun only rank 0 runs and
prints, the other ranks exit 0 without work.  The clock sampler behind the line's
`clocks` object summarises nvidia-smi's CSV (here from a stand-in script).  CPU only
(one oracle step of 16 intervals of the d = 729 chain, a few seconds)."""
import json
import os
import socket
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = ["impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"]


def _json_lines(text):
    return [json.loads(line) for line in text.splitlines() if line.startswith("{")]


def _check_line(out, n_gpus):
    for k in KEYS:
        assert k in out, k
    assert out["impl"] == "reference" and out["n_gpus"] == n_gpus and out["steps"] == 1
    assert out["value"] > 0 and out["higher_is_better"] is True and out["unit"] == "intervals/s"
    assert out["config"]["workload"].startswith("transmon_chain_d729")
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == out["value"] and cb["sample"]
    e2e = out["e2e"]
    assert e2e["value"] == out["value"] and e2e["unit"] == out["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1, r.stdout
    _check_line(lines[0], 1)


def test_reference_arm_under_torchrun_prints_from_rank_zero_only():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port),
           "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1, r.stdout
    _check_line(lines[0], 2)


def _fake_smi(tmp_path, rows):
    """An nvidia-smi stand-in that prints `rows` (CSV, no header, no units) until stopped."""
    script = tmp_path / "nvidia-smi"
    body = "\n".join(f"echo '{r}'" for r in rows)
    script.write_text(f"#!/bin/sh\n{body}\nwhile true; do sleep 0.05; done\n")
    script.chmod(0o755)
    return str(tmp_path)


def test_clock_sampler_reports_median_max_and_active_reasons(tmp_path, monkeypatch):
    """The clocks object of the JSON line: median SM clock under load, the maximum clock,
    and the throttle reasons seen active (power cap kept, the others absent here)."""
    rows = ["0, 1965, 2070, 850.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 900.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2070, 1010.2, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, [N/A], 2070, [N/A], 0x0, Not Active, Not Active, Not Active, Not Active"]
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, rows) + os.pathsep + os.environ["PATH"])
    sys.path.insert(0, ROOT)
    import bench
    s = bench.ClockSampler(0)
    s.start()
    time.sleep(1.0)
    clk = s.stop()
    assert clk["samples"] == 4 and clk["sm_mhz"] == 1980.0 and clk["sm_max_mhz"] == 2070.0
    assert clk["reasons"] == ["sw_power_cap"] and clk["power_w_max"] == 1010.2


def test_clock_sampler_flags_thermal_slowdown(tmp_path, monkeypatch):
    rows = ["0, 1500, 2070, 1300.0, 0x0000000000000048, Active, Active, Not Active, Not Active"]
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, rows) + os.pathsep + os.environ["PATH"])
    sys.path.insert(0, ROOT)
    import bench
    s = bench.ClockSampler(0)
    s.start()
    time.sleep(0.5)
    clk = s.stop()
    assert clk["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"] and clk["sm_mhz"] == 1500.0
