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


TABLE3_TWO_DTYPE = np.dtype([("offset", np.int64), ("rho1000_1", np.int32), ("rho1000_2", np.int32),
                             ("f0_1", np.int32), ("f0_2", np.int32)])


def table3_rows_two(snr1, tmpl1, snr2, tmpl2, f0) -> np.ndarray:
    """Table 3 for two channels (H1, L1): one row per sample offset where
    either channel has a hit, zeros for the channel without one."""
    tmpl1, tmpl2 = np.asarray(tmpl1), np.asarray(tmpl2)
    f0 = np.asarray(f0, dtype=np.float64)
    idx = np.flatnonzero((tmpl1 >= 0) | (tmpl2 >= 0))
    rows = np.zeros(idx.size, dtype=TABLE3_TWO_DTYPE)
    rows["offset"] = idx.astype(np.int64) + 1
    for col, snr, tm in (("1", snr1, tmpl1), ("2", snr2, tmpl2)):
        t = tm[idx]
        h = t >= 0
        r = np.zeros(idx.size, dtype=np.int32)
        f = np.zeros(idx.size, dtype=np.int32)
        r[h] = np.trunc(np.asarray(snr, dtype=np.float64)[idx][h] * 1000.0).astype(np.int32)
        f[h] = np.trunc(f0[t[h]]).astype(np.int32)
        rows["rho1000_" + col] = r
        rows["f0_" + col] = f
    return rows


def coincidences(tmpl1, tmpl2, f0, delta: float = 50.0) -> dict:
    """Simultaneous hits of two channels at the same sample offset (Sec. 5):
    hit counts per channel, lags where both hit, and those whose templates'
    initial frequencies differ by less than ``delta`` Hz."""
    tmpl1, tmpl2 = np.asarray(tmpl1), np.asarray(tmpl2)
    f0 = np.asarray(f0, dtype=np.float64)
    both = (tmpl1 >= 0) & (tmpl2 >= 0)
    lags = np.flatnonzero(both)
    close = np.abs(f0[tmpl1[lags]] - f0[tmpl2[lags]]) < delta
    return {"hits": (int((tmpl1 >= 0).sum()), int((tmpl2 >= 0).sum())),
            "simultaneous": int(both.sum()), "within_delta": int(close.sum()),
            "lags": lags[close].astype(np.int64)}
