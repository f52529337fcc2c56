"""The benchmark's reference arm (the FP64 oracle on the host cores) on a tiny workload: one JSON
line with the keys the benchmark contract asks for, on rank 0 only."""
import io
import json
from contextlib import redirect_stdout

import bench


def _args(steps=2, warmup=1):
    return type("A", (), {"steps": steps, "warmup": warmup, "gpus": 1})()


def test_reference_line_keys(monkeypatch):
    monkeypatch.setitem(bench.WORKLOADS, "tiny_7pt", (0, "f64", 12, 10, 8, 4))
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(_args(), "tiny_7pt") == 0
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == "GLUP/s" and line["value"] > 0
    assert line["config"]["workload"] == "tiny_7pt" and line["higher_is_better"] is True
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "GLUP/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_other_ranks_do_nothing(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(_args(), "7pt_const_f64_512") == 0
    assert buf.getvalue() == ""
