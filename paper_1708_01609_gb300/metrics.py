"""Measurement conventions: the paper's FFT flop count and the FP32 ALU peak.

Eq. nd counts 5 N log2 N floating-point operations per length-N FFT
correlation (the clFFT GFLOP/s convention of Fig. 5); throughput in
correlations/s converts to FLOP/s with it.  The FP32 ALU peak of a GPU is
SMs x 128 FP32 lanes x 2 flops (one FMA) x SM clock.
"""
from __future__ import annotations

import math

FP32_LANES_PER_SM = 128


def nominal_flops_per_correlation(n: int) -> float:
    """5 N log2 N (Eq. nd)."""
    return 5.0 * n * math.log2(n)


def realtime_flops(n: int, bank: int, seconds: float) -> float:
    """Eq. nd: 5 N log2 N x (bank size) / T for one segment of duration T."""
    return nominal_flops_per_correlation(n) * bank / seconds


def fp32_peak_flops(sms: int, sm_mhz: float) -> float:
    return sms * FP32_LANES_PER_SM * 2.0 * sm_mhz * 1e6
