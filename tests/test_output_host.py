"""Host logic of the paper's output form (Table 3, Sec. 5 coincidences) in
the product package, against the oracle's definitions on random per-lag
projections (no GPU): identical rows and counts."""
import numpy as np

import oracle as O
from paper_1708_01609_gb300 import output


def random_projection(rng, n, k, hit_rate):
    tmpl = np.where(rng.random(n) < hit_rate, rng.integers(0, k, n), -1).astype(np.int32)
    snr = np.where(tmpl >= 0, 5.5 + 3.0 * rng.random(n), 0.0).astype(np.float32)
    return snr, tmpl


def test_table3_rows_equal_the_oracle():
    rng = np.random.Generator(np.random.PCG64(11))
    f0 = 350.0 + 1650.0 * rng.random(4096)
    for rate in (0.0, 0.01, 0.3, 1.0):
        snr, tmpl = random_projection(rng, 20000, 4096, rate)
        got = output.table3_rows(snr, tmpl, f0)
        want = O.table3_rows(snr, tmpl, f0)
        assert len(got) == len(want) == int(np.sum(tmpl >= 0))
        for name in ("offset", "rho1000", "f0"):
            assert np.array_equal(got[name], want[name]), name


def test_two_channel_rows_and_coincidences_equal_the_oracle():
    rng = np.random.Generator(np.random.PCG64(12))
    f0 = 350.0 + 1650.0 * rng.random(1024)
    s1, t1 = random_projection(rng, 30000, 1024, 0.05)
    s2, t2 = random_projection(rng, 30000, 1024, 0.05)
    t2[:500] = t1[:500]  # some simultaneous hits with equal templates
    s2[:500] = np.where(t1[:500] >= 0, s2[:500], 0.0)
    got = output.table3_rows_two(s1, t1, s2, t2, f0)
    want = O.table3_rows_two(s1, t1, s2, t2, f0)
    assert len(got) == len(want)
    for name in want.dtype.names:
        assert np.array_equal(got[name], want[name]), name
    for delta in (50.0, 5.0):
        g = output.coincidences(t1, t2, f0, delta)
        w = O.coincidences(t1, t2, f0, delta)
        assert g["hits"] == w["hits"]
        assert g["simultaneous"] == w["simultaneous"] and g["within_delta"] == w["within_delta"]
        assert np.array_equal(np.asarray(g["lags"]), w["lags"])
        assert w["within_delta"] >= int(np.sum(t1[:500] >= 0))
