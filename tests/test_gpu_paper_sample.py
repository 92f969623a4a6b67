"""The paper-scale workload's error sample: every 256th chirp (k = 0 mod 256,
4096 templates) of the N = 2^16, 2^20-chirp bank against the paper-scale
segment, every lag of every template against the FP64 oracle, on the FP32
path and on both tensor-core forms; sigma and the kappa = 5.5 tail sets as
well.  The oracle runs in a spawn pool, one process per core.

Bars: FP32 within 1e-5 sigma, sigma within 1e-6 relative; BF16x3 / FP16x3
within 2e-3 sigma, sigma within 1e-5 relative; tail sets identical except entries
within max(1e-3, tolerance) sigma of the threshold.  The errors found are
printed (run with -s)."""
import multiprocessing as mp
import os

import numpy as np
import pytest

import synthetic as S
from gpu_helpers import compare_tails, make_ctx

pytestmark = pytest.mark.gpu

STRIDE = 256
CHUNK = 256
KAPPA = 5.5
FORMS = {0: ("FP32", 1e-5, 1e-6), 1: ("BF16x3", 2e-3, 1e-5), 2: ("FP16x3", 2e-3, 1e-5)}

_Y = None
_P = None


def _init():
    global _Y, _P
    seg, params = S.paper_case(seed=2017)
    _Y, _P = seg.y, params[::STRIDE]


def _oracle_rows(ks):
    import oracle as O
    bank = O.chirp_bank(_P[ks[0]:ks[-1] + 1], 4096.0, 4096, 0.05)
    res = O.search(_Y, bank, np.inf, batch=len(ks), return_rho=True)
    return res["rho"], res["sigma"]


@pytest.fixture(scope="module")
def pool():
    cores = max(1, min(16, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(cores, initializer=_init) as p:
        yield p


def test_paper_bank_sample_every_lag(pool):
    seg_data, params = S.paper_case(seed=2017)
    sub = params[::STRIDE]
    assert len(sub) == 4096
    ctxs, handles, recs, sigmas = {}, {}, {}, {}
    for prec in FORMS:
        c = make_ctx(tail_capacity=1 << 22, precision=prec)
        seg = c.bege_load_segment(seg_data.y)
        bid = c.bege_define_bank(sub, tau=1.0, taper_frac=0.05)
        job = c.bege_correlate(seg, bid, 0, len(sub), KAPPA)
        r, total = c.bege_fetch_tails(job)
        assert total == len(r)
        ctxs[prec], handles[prec] = c, (seg, bid)
        recs[prec], sigmas[prec] = r, c.bege_get_sigma(job, len(sub))
    err = {p: np.empty(len(sub)) for p in FORMS}
    sig_err = {p: 0.0 for p in FORMS}
    summary = {p: {"matched": 0, "near": 0, "worst": 0.0} for p in FORMS}
    for k0 in range(0, len(sub), CHUNK):
        ks = list(range(k0, k0 + CHUNK))
        parts = pool.map(_oracle_rows, [ks[i:i + 16] for i in range(0, CHUNK, 16)])
        rho = np.concatenate([p[0] for p in parts])
        sig = np.concatenate([p[1] for p in parts])
        ref = {k0 + i: (rho[i], sig[i]) for i in range(CHUNK)}
        for prec, (name, tol, stol) in FORMS.items():
            seg, bid = handles[prec]
            got = ctxs[prec].bege_dump_correlation(seg, bid, k0, k0 + CHUNK)
            err[prec][k0:k0 + CHUNK] = np.max(np.abs(got - rho), axis=1) / sig
            sig_err[prec] = max(sig_err[prec],
                                float(np.max(np.abs(sigmas[prec][k0:k0 + CHUNK] / sig - 1))))
            mine = recs[prec][(recs[prec]["tmpl"] >= k0) & (recs[prec]["tmpl"] < k0 + CHUNK)]
            for g0 in range(k0, k0 + CHUNK, 16):
                part = {k: ref[k] for k in range(g0, g0 + 16)}
                s = compare_tails(mine, part, KAPPA, tmpl_subset=set(part), tol=tol,
                                  near=max(1e-3, tol))
                summary[prec]["matched"] += s["matched"]
                summary[prec]["near"] += s["near"]
                summary[prec]["worst"] = max(summary[prec]["worst"], s["worst"])
    for c in ctxs.values():
        c.close()
    for prec, (name, tol, stol) in FORMS.items():
        print(f"{name}, 4096 chirps (k = 0 mod 256) of the N = 2^16 paper bank: max|err| "
              f"{err[prec].max():.2e} sigma (median {np.median(err[prec]):.2e}), sigma rel err "
              f"{sig_err[prec]:.1e}, {summary[prec]['matched']} oracle tails matched (worst "
              f"{summary[prec]['worst']:.1e} sigma), {summary[prec]['near']} near the threshold")
        assert np.all(err[prec] <= tol), (name, err[prec].max())
        assert sig_err[prec] <= stol, (name, sig_err[prec])
        assert summary[prec]["matched"] > 100
