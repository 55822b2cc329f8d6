"""The oracle arm of bench.py (--impl reference) on the host: one JSON line on
rank 0 with the keys the measurement needs, nothing on the other ranks."""
import argparse
import importlib.util
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _args(**kw):
    d = dict(gpus=1, steps=1, warmup=0, workload="paper150")
    d.update(kw)
    return argparse.Namespace(**d)


def test_reference_arm_line(capsys, monkeypatch):
    monkeypatch.delenv("RANK", raising=False)
    b = _bench()
    b.run_reference(_args())
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == b.METRIC and d["unit"] == b.UNIT
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["value"] > 0
    assert d["config"]["workload"] == b.WORKLOADS["paper150"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": b.UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # one oracle step of one 150 x 150 run, N_s = 17
    assert abs(d["value"] * d["ms_per_step"] * 1e-3 - 150 * 150 * 17 * 4) < 1e-6 * 150 * 150 * 17 * 4


def test_reference_arm_other_ranks_are_silent(capsys, monkeypatch):
    monkeypatch.setenv("RANK", "1")
    _bench().run_reference(_args())
    assert capsys.readouterr().out == ""
