"""Host logic of bench.py, on the CPU: the guard that reports the render
kernel's DRAM traffic only while its sources are the ones the counters were
taken on, the clock-sample summary that flags throttling, and the reference
arm (the FP64 oracle on the host's cores): its JSON line, and that under a
multi-rank launch only rank 0 runs and prints."""
import importlib.util
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_traffic_reported_only_for_the_profiled_sources(tmp_path, monkeypatch):
    b = load_bench()
    prof = tmp_path / "prof.md"
    monkeypatch.setattr(b, "TRAFFIC_PROFILE", str(prof))
    assert b.measured_traffic() is None  # no summary
    prof.write_text(f"notes\nsource_sha256: {b.render_source_digest()}\ndram_bytes_per_launch: 1234\n")
    assert b.measured_traffic() == 1234
    prof.write_text("source_sha256: " + "0" * 64 + "\ndram_bytes_per_launch: 1234\n")
    assert b.measured_traffic() is None  # the sources changed since the capture
    # a source edit changes the digest
    src = tmp_path / "k.cu"
    src.write_text("a")
    monkeypatch.setattr(b, "TRAFFIC_SOURCES", (str(src),))
    d0 = b.render_source_digest()
    src.write_text("b")
    assert b.render_source_digest() != d0


def test_clock_summary_flags_throttle_reasons():
    b = load_bench()
    s = b.ClockSampler(0)
    row = lambda mhz, hw="Not Active", cap="Not Active": ["0", str(mhz), "2070", "900", "0x0", hw, "Not Active",
                                                          "Not Active", cap]
    s.rows = [row(2070), row(2070), row(1950, cap="Active")]
    r = s.summary()
    assert r["sm_mhz"] == 2070 and r["sm_max_mhz"] == 2070 and r["samples"] == 3
    assert r["reasons"] == ["sw_power_cap"]
    s.rows = [row(1500, hw="Active"), ["garbage"]]
    r = s.summary()
    assert r["reasons"] == ["hw_slowdown"] and r["samples"] == 1
    assert b.ClockSampler(0).summary()["sm_mhz"] is None


def run_reference(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                           "small", "--steps", "1", "--warmup", "0"], capture_output=True, text=True, env=env,
                          timeout=600, cwd=ROOT)


def test_reference_arm_prints_one_line_with_the_contract_keys():
    r = run_reference({"RANK": "0", "WORLD_SIZE": "1", "LOCAL_RANK": "0"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "frames/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["cells"] == 400_000 and d["config"]["resolution"] == "1280x720"


def test_reference_arm_other_ranks_exit_without_work():
    r = run_reference({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [x for x in r.stdout.splitlines() if x.startswith("{")]
