"""bench.py's CPU baseline on a small budget: the all-core figure next to the single-thread one,
and the single-thread figure alone when the process pool cannot run.  CPU only."""
import numpy as np
import pytest


def test_all_cores_and_single_thread():
    import bench
    mlp, o, d = bench.workload()
    base = bench.cpu_baseline(mlp, o, d, budget_s=0.3)
    assert base["kind"] == "oracle" and base["unit"] == "faces/s" and base["value"] > 0
    assert "single_thread" in base and base["single_thread"]["cores"] == 1
    assert base["cores"] >= 1 and base["cpu"]


def test_pool_failure_keeps_the_single_thread_figure(monkeypatch):
    import bench
    from oracle import parallel

    class Broken:
        def __init__(self, *a, **k):
            raise RuntimeError("no workers")
    monkeypatch.setattr(parallel, "LevelMarcher", Broken)
    mlp, o, d = bench.workload()
    base = bench.cpu_baseline(mlp, o, d, budget_s=0.3)
    assert base["cores"] == 1 and "all_cores_unavailable" in base and base["value"] > 0


@pytest.mark.parametrize("broken", [False, True])
def test_reference_arm_line(monkeypatch, capsys, broken):
    import argparse
    import json

    import bench
    from oracle import parallel
    if broken:
        class Broken:
            def __init__(self, *a, **k):
                raise RuntimeError("no workers")
        monkeypatch.setattr(parallel, "LevelMarcher", Broken)
    args = argparse.Namespace(gpus=1, steps=1, warmup=0)
    dist = bench.Dist(1)
    assert bench.run_reference(args, dist) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "faces/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "faces/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert ("processes" in line["cpu_baseline"]["sample"]) != broken
