"""The flop convention of the throughput metric (Eq. nd) reproduces the
figures the paper prints (tests/golden/paper_figures.txt)."""
import os

import pytest

from paper_1708_01609_gb300 import metrics

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_figures.txt")


def golden():
    out = {}
    with open(GOLDEN) as fh:
        lines = fh.readlines()
    for line in lines:
        if line.startswith("#") or not line.strip():
            continue
        name, value, rel, _ = [f.strip() for f in line.split("|", 3)]
        out[name] = (float(value), float(rel))
    return out


def computed():
    n, m = 1 << 16, 2048
    per = metrics.nominal_flops_per_correlation(n)
    return {
        "realtime_tflops_N16_K1M_2e23_T16": metrics.realtime_flops(n, 1 << 23, 16.0),
        "block_M2_inverse_ffts_flops": per * m * m,
        "s6_total_correlations": (1 << 23) * 288 * m,
        "s6_total_flops": (1 << 23) * 288 * m * per,
        "block_bytes_complex_sp": n * m * 8,
        "segment_bytes_complex_sp": n * 8,
    }


@pytest.mark.parametrize("name", sorted(golden()))
def test_paper_figure(name):
    value, rel = golden()[name]
    got = computed()[name]
    assert abs(got / value - 1) <= rel, (name, got, value)


def test_fp32_peak_formula():
    # 152 SMs x 128 lanes x 2 flops x 2070 MHz
    assert abs(metrics.fp32_peak_flops(152, 2070.0) - 80.54e12) < 0.01e12
