"""The benchmark's CPU-side contract.  CPU only: the reference arm times the CPU oracle,
and the traffic lookup is host logic."""
import importlib.util
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("_bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _run(env_extra, *args):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _run({}, "--impl", "reference", "--steps", "1", "--warmup", "0")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "k-th select Gelem/s (n=2^27 float32)" and d["unit"] == "Gelem/s"
    assert d["higher_is_better"] is True and d["value"] > 0
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "Gelem/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_reference_arm_other_ranks_exit_without_work():
    r = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, "--impl", "reference", "--steps", "1",
             "--warmup", "0")
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_traffic_is_reported_only_for_the_captured_sources(monkeypatch):
    b = _bench()
    with open(os.path.join(ROOT, "profiles", "select_kernel_f32_n2e27.md")) as f:
        text = f.read()
    recorded = [l.split(":")[1].strip() for l in text.splitlines() if l.startswith("kernel_sources_sha256:")]
    assert len(recorded) == 1 and len(recorded[0]) == 64
    monkeypatch.setattr(b, "select_sources_sha256", lambda: recorded[0])
    traffic, how = b.select_traffic()
    assert traffic is not None and traffic > 0 and "ncu" in how
    monkeypatch.setattr(b, "select_sources_sha256", lambda: "0" * 64)
    traffic, how = b.select_traffic()
    assert traffic is None and "changed" in how


def test_ranks_of_the_headline_workload():
    b = _bench()
    n = 1 << 27
    assert b.ranks_for(n) == [1, n // 100, (n + 1) // 2, 99 * n // 100, n]
    assert all(1 <= k <= n for k in b.ranks_for(n))
