"""Host-side pieces of bench.py without a GPU: the algorithmic bytes of the
roofline, the peak lookup and the clock-sample summary."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
from paper_1601_07728_gb300 import synth as S  # noqa: E402


class _Shape:
    n_k, n_x, n_bands, n_alpha, n_proj = 512, 4096, 64, 6, 36


def test_algorithmic_bytes_of_the_l23_workload():
    b = bench.algorithmic_bytes(_Shape, "split_bf16")
    u = 512 * 4096 * 64 * 8                     # bf16 hi + lo of complex U: 8 bytes per element
    vec = 6 * 512 * 64 * 16
    phi = 512 * 4096 * 6 * 8
    assert b["band_to_grid"] == u + vec + phi
    assert b["grid_to_band"] == u + phi + 2 * vec + 36 * 512 * 64 * 16 + 512 * 64 * 8
    assert b["kconv"] == phi + phi + 512 * 4096 * 4
    assert bench.algorithmic_bytes(_Shape, "fp64")["band_to_grid"] == 2 * u + vec + 2 * phi


def test_peak_lookup_has_a_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6786.6}')
    assert bench.peaks() == (6786.6, "measured")


def test_clock_summary_keeps_this_gpu_and_reasons():
    c = bench.ClockSampler("00000009:01:00.0")
    c.proc = type("P", (), {"terminate": lambda self: None, "wait": lambda self, timeout=None: 0})()
    c.lines = [
        "00000009:01:00.0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "00000009:01:00.0, 1900, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "00000009:02:00.0, 1000, 2070, 100.0, 0x0, Active, Not Active, Not Active, Not Active",   # other GPU
        "garbage",
    ]
    s = c.stop()
    assert s["samples"] == 2
    assert s["sm_mhz"] == pytest.approx(1985.0)
    assert s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_workload_constants_match_the_generator():
    cfg = S.CONFIGS[bench.WORKLOAD]
    assert cfg["n_alpha"] == 6 and cfg["nk"] == (8, 8, 8) and cfg["n_bands"] == 64 and cfg["nx"] == (16, 16, 16)


def test_reference_arm_prints_one_contract_line(monkeypatch, capsys):
    """The reference arm (the FP64 oracle on the host cores) prints one JSON
    line with the contract's keys; the small 1s workload keeps it quick."""
    import json
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--workload", "k_edge_small",
                                      "--steps", "3", "--warmup", "3"])
    assert bench.main() == 0
    lines = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "k_edge_small" and d["config"]["desc"].startswith("k_edge_small")
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]


def test_step_bytes_and_flops_of_the_l23_workload():
    """Two streams of u_nk per step bound the HBM roofline; the FP64 form's
    flops are the two complex contractions (8 real flops per complex MAC)."""
    assert bench.u_bytes(_Shape) == 512 * 4096 * 64 * 8
    assert bench.u_bytes(_Shape, "fp64") == 512 * 4096 * 64 * 16
    assert bench.matvec_flops(_Shape) == 2 * 8 * 512 * 4096 * 64 * 6
