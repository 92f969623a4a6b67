"""Shared helpers of the GPU parity tests: a context fixture factory and the
tail-set comparison rule (sets identical except entries within 1e-3 sigma of
the threshold; values within a tolerance times sigma)."""
import numpy as np

import oracle as O

NEAR = 1e-3       # sigma band around the threshold excluded from set parity
TOL_FP32 = 1e-5   # value tolerance, in units of the template's sigma


def make_ctx(**kw):
    from paper_1708_01609_gb300 import binding, build
    build()
    return binding.Context(0, **kw)


def compare_tails(gpu_recs, ref, kappa, tmpl_subset=None, tol=TOL_FP32, near=None):
    """gpu_recs: TAIL_DTYPE records; ref: dict template -> (rho FP64, sigma).

    Returns a summary dict; raises AssertionError on a parity violation.
    """
    if tmpl_subset is not None:
        gpu_recs = gpu_recs[np.isin(gpu_recs["tmpl"], np.array(sorted(tmpl_subset), np.uint32))]
    got = {(int(k), int(n)): float(v)
           for k, n, v in zip(gpu_recs["tmpl"], gpu_recs["lag"], gpu_recs["value"])}
    near_band = NEAR if near is None else near
    n_ref = n_near = 0
    worst = 0.0
    for k, (rho, sig) in ref.items():
        thr = kappa * sig
        lags = np.nonzero(np.abs(rho) > thr)[0]
        for n in lags:
            near = abs(abs(rho[n]) - thr) <= near_band * sig
            key = (k, int(n))
            if key not in got:
                assert near, f"missing tail {key}: rho={rho[n]} thr={thr}"
                n_near += 1
                continue
            n_ref += 1
            err = abs(got[key] - rho[n]) / sig
            worst = max(worst, err)
            assert err <= tol, f"tail {key}: gpu {got[key]} oracle {rho[n]} err {err} sigma"
        for (kk, n), v in got.items():
            if kk != k:
                continue
            if abs(rho[n]) > thr:
                continue
            assert abs(abs(rho[n]) - thr) <= near_band * sig, f"extra tail {(kk, n)}: rho={rho[n]} thr={thr}"
            n_near += 1
    return {"matched": n_ref, "near": n_near, "worst": worst}


def oracle_rho(y, templates, batch=16):
    res = O.search(y, templates, np.inf, batch=batch, return_rho=True)
    return res["rho"], res["sigma"]
