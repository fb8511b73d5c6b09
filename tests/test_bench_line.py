"""The repo arm's final stdout line of bench.py: built from worst-case
figures (long floats, long sample text, all clock reasons), it parses, carries
the contract's keys and stays under 1 KB, so that a reader of only the last
kilobytes of the output sees all of it.  Side-leg selection is checked too."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _line():
    w = bench.WORKLOAD
    return bench.compact_line(
        metric=bench.METRIC, value=6.7412345678901234e11, unit=bench.UNIT, n_gpus=8, steps=20, warmup=5,
        ms_per_step=77.81234567890123, workload=w.name,
        config={"bins": w.bins, "parallelism": "replicas x8", "l2": "inputs>L2"},
        clocks={"sm_mhz": 2070.0, "sm_max_mhz": 2070.0,
                "reasons": ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"],
                "samples": 123},
        roofline={"bound": "alu", "achieved": 28.123456789, "peak": 40.27392, "unit": "Tinst/s",
                  "frac": 0.69912345678, "traffic": 705512345.678, "kernel": "fine_f32_d1_kernel"},
        cpu={"value": 336812345.6789, "unit": bench.UNIT, "cores": 144, "kind": "oracle",
             "sample": "1048576 particles x 1000 EM steps, 12.3 s",
             "single_core": {"value": 1.0}},
        e2e={"value": 6.581234567e11, "unit": bench.UNIT, "h2d_bytes_per_step": 8388608,
             "d2h_bytes_per_step": 209304},
        launches=1234567, fp32_over_fp64=101.23456, iters_to_w1=5, time_to_w1_ms=393.123456)


def test_final_line_is_compact_and_complete(capsys):
    s = bench.emit_line(_line())
    out = capsys.readouterr().out.strip().splitlines()
    assert out[-1] == s
    assert len(s.encode()) < 1024
    d = json.loads(s)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "gpu_launches", "clocks", "roofline",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["higher_is_better"] is True and d["config"]["workload"]
    assert set(d["roofline"]) >= {"bound", "achieved", "peak", "unit", "frac", "traffic"}
    assert abs(d["roofline"]["frac"] - d["roofline"]["achieved"] / d["roofline"]["peak"]) < 1e-3
    assert set(d["cpu_baseline"]) == {"value", "unit", "cores", "kind", "sample"}
    assert d["e2e"]["h2d_bytes_per_step"] > 0 and d["e2e"]["d2h_bytes_per_step"] > 0
    assert set(d["clocks"]) == {"sm_mhz", "sm_max_mhz", "reasons"}


def test_oversized_line_is_refused():
    line = _line()
    line["config"]["padding"] = "x" * 1024
    with pytest.raises(RuntimeError):
        bench.emit_line(line)


def test_leg_selection():
    assert bench.parse_legs("") == [] and bench.parse_legs(None) == []
    assert bench.parse_legs("all") == list(bench.LEGS)
    assert bench.parse_legs("adjoint, studies") == ["adjoint", "studies"]
    with pytest.raises(SystemExit):
        bench.parse_legs("nonsense")
