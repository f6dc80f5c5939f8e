"""bench.py's reference arm: the FP64 oracle timed on the host cores (it
needs no GPU).  Its JSON line carries the metric, unit and config of the
GPU arm, impl "reference", a cpu_baseline describing the run and an e2e
entry with no host-device bytes; under several ranks only rank 0 works and
prints."""
import json
import os
import subprocess
import sys

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=REPO, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    sys.path.insert(0, REPO)
    import bench
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["higher_is_better"] is True and line["steps"] == 1
    assert line["config"]["workload"].startswith("large: 3200x2112")
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_nothing(monkeypatch, capsys):
    sys.path.insert(0, REPO)
    import bench
    monkeypatch.setattr(bench, "dist_setup", lambda want_cuda: (1, 2, 1, None))

    class Args:
        steps, warmup, gpus = 1, 0, 2
    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""
