"""bench.py's reference arm (the FP64 oracle on the host cores): one JSON
line with the contract's keys on rank 0, nothing on the other ranks, and a
run length bounded whatever the step count."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _run(args, env_extra=None, timeout=300):
    env = dict(os.environ)
    env.update(env_extra or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)
    assert r.returncode == 0, r.stderr[-2000:]
    return [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]


def test_reference_line_has_the_contract_keys(oracle_mod):
    lines = _run(["--workload", "uniform_box_256", "--steps", "3", "--warmup", "1"])
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference"
    # The same metric string and config object as the GPU arm's line.
    assert d["metric"] == bench.headline_metric("uniform_box_256")
    assert d["config"] == bench.headline_config("uniform_box_256")
    assert d["unit"] == "frames/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 3 and d["warmup"] == 1
    assert d["config"]["workload"] == "uniform_box_256"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert cb["sample"].startswith("3 whole frames")
    assert d["e2e"] == {"value": d["value"], "unit": "frames/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_sample_is_bounded(oracle_mod, monkeypatch):
    # A step count far beyond the time budget times only the frames that fit.
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(bench, "REFERENCE_BUDGET_S", 0.5)
    calls = []

    class FakeOracle:
        @staticmethod
        def build():
            pass

        @staticmethod
        def render(scene, cam):
            calls.append(1)
            import time
            time.sleep(0.1)

        @staticmethod
        def num_threads():
            return 1

    monkeypatch.setitem(sys.modules, "oracle", FakeOracle)

    class Args:
        workload, steps, warmup = "uniform_box_256", 100000, 20

    out = []
    monkeypatch.setattr("builtins.print", lambda s: out.append(s))
    bench.run_reference(Args)
    d = json.loads(out[0])
    # 3 warm-up frames, then 0.5 s / 0.1 s = 4 or 5 timed frames, not 100000.
    assert 3 + 1 <= len(calls) <= 3 + 6
    assert d["steps"] == 100000
    assert d["cpu_baseline"]["sample"].startswith(f"{len(calls) - 3} whole frames")


def test_reference_other_ranks_print_nothing():
    lines = _run(["--workload", "uniform_box_256", "--steps", "2", "--warmup", "1"],
                 {"WORLD_SIZE": "2", "RANK": "1", "LOCAL_RANK": "1"})
    assert lines == []
