"""Filter output in the paper's block-file form (Sec. 4, Table 3).

A per-lag projection (bege_correlate_max / Context.bege_fetch_max) becomes one
row per sample offset with a hit: the 1-based sample offset, 1000 x rho/sigma
as a 4-byte integer (rounded toward zero) and the initial frequency f0 of the
hit's chirp template in whole Hz (rounded toward zero).
"""
from __future__ import annotations

import numpy as np

TABLE3_DTYPE = np.dtype([("offset", np.int64), ("rho1000", np.int32), ("f0", np.int32)])


def table3_rows(snr: np.ndarray, tmpl: np.ndarray, f0: np.ndarray) -> np.ndarray:
    """Rows of Table 3 for one channel: snr, tmpl as returned by
    bege_fetch_max (tmpl -1 = no hit); f0[k] the bank's initial frequencies."""
    tmpl = np.asarray(tmpl)
    hit = tmpl >= 0
    idx = np.flatnonzero(hit)
    rows = np.zeros(idx.size, dtype=TABLE3_DTYPE)
    rows["offset"] = idx.astype(np.int64) + 1
    rows["rho1000"] = np.trunc(np.asarray(snr, dtype=np.float64)[idx] * 1000.0).astype(np.int32)
    rows["f0"] = np.trunc(np.asarray(f0, dtype=np.float64)[tmpl[idx]]).astype(np.int32)
    return rows
