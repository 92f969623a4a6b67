"""Precision form: column FFTs on tcgen05 tensor cores with split 16-bit
operands (BF16x3, FP16x3) and FP32 accumulation, against the FP64 oracle.

Bar for the reduced-precision path: correlation values within 2e-3 sigma of
the oracle; sigma within 1e-5 relative (sigma is an FP32 sum over the
spectrum, whose split-precision error is near 1e-6 relative, so 1e-5 leaves
a margin of about five); tail sets identical except entries
within the value tolerance (2e-3 sigma) of the threshold.  The errors found
are printed (run with -s to see them).
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from gpu_helpers import compare_tails, make_ctx, oracle_rho

pytestmark = pytest.mark.gpu

TOL_TC = 2e-3
TOL_SIGMA_TC = 1e-5
PRECISIONS = {1: "BF16x3", 2: "FP16x3"}


@pytest.fixture(scope="module", params=[1, 2], ids=["bf16x3", "fp16x3"])
def tctx(request):
    c = make_ctx(tail_capacity=1 << 24, precision=request.param)
    yield request.param, c
    c.close()


@pytest.mark.parametrize("n,length", [(1 << 14, 4096), (1 << 15, 2048), (1 << 16, 4096),
                                      (1 << 16, 4000), (1 << 17, 4096)])
def test_tc_dump_matches_oracle(tctx, n, length):
    prec, ctx = tctx
    y = S.band_limited_noise(n, n + 5).astype(np.float64)
    y += 0.05 * np.random.Generator(np.random.PCG64(n)).standard_normal(n)
    y = y.astype(np.float32)
    bank = S.random_samples_bank(6, length, length + 9)
    seg = ctx.bege_load_segment(y)
    bid = ctx.bege_define_bank_samples(bank)
    got = ctx.bege_dump_correlation(seg, bid, 0, 6)
    rho, sig = oracle_rho(y, bank.astype(np.float64))
    err = np.max(np.abs(got - rho), axis=1) / sig
    rms = np.sqrt(np.mean((got - rho) ** 2, axis=1)) / sig
    job = ctx.bege_correlate(seg, bid, 0, 6, 5.0)
    sg = ctx.bege_get_sigma(job, 6)
    serr = np.max(np.abs(sg / sig - 1))
    print(f"{PRECISIONS[prec]} N={n} L={length}: max|err| {err.max():.2e} sigma, "
          f"rms {rms.max():.2e} sigma, sigma rel err {serr:.2e}")
    assert np.all(err <= TOL_TC), err
    assert serr <= TOL_SIGMA_TC
    for h in (job, bid, seg):
        ctx.bege_release(h)


def test_tc_small_case_tails(tctx):
    prec, ctx = tctx
    seg_data, params = S.small_case()
    kappa = 5.0
    seg = ctx.bege_load_segment(seg_data.y)
    bid = ctx.bege_define_bank(params)
    job = ctx.bege_correlate(seg, bid, 0, len(params), kappa)
    recs, total = ctx.bege_fetch_tails(job)
    assert total == len(recs)
    bank = O.chirp_bank(params, 4096.0, 4096, 0.05)
    rho, sig = oracle_rho(seg_data.y, bank)
    s = compare_tails(recs, {k: (rho[k], sig[k]) for k in range(len(params))}, kappa,
                      tol=TOL_TC, near=TOL_TC)
    print(f"{PRECISIONS[prec]} small case: {s}")
    k_inj, lag, _ = seg_data.injections[0]
    assert any((int(r["tmpl"]), int(r["lag"])) == (k_inj, lag) for r in recs)
    for h in (job, bid, seg):
        ctx.bege_release(h)


def test_tc_rejects_short_segments_and_long_templates(tctx):
    from paper_1708_01609_gb300.binding import BegeError
    prec, ctx = tctx
    seg = ctx.bege_load_segment(S.band_limited_noise(1 << 13, 1))
    bid = ctx.bege_define_bank_samples(np.ones((2, 1024), np.float32))
    with pytest.raises(BegeError):
        ctx.bege_correlate(seg, bid, 0, 2, 5.0)          # N = 2^13
    seg2 = ctx.bege_load_segment(S.band_limited_noise(1 << 15, 1))
    bid2 = ctx.bege_define_bank_samples(np.ones((2, 8192), np.float32))
    with pytest.raises(BegeError):
        ctx.bege_correlate(seg2, bid2, 0, 2, 5.0)        # L > 4096
    for h in (bid, seg, bid2, seg2):
        ctx.bege_release(h)


@pytest.fixture(scope="module")
def paper_subset():
    """Every 4096th chirp of the N = 2^16, 2^20-chirp paper-scale bank (256
    templates) with the oracle's correlations of the paper-scale segment."""
    seg_data, params = S.paper_case(seed=2017)
    sub = params[::4096]
    bank = O.chirp_bank(sub, 4096.0, 4096, 0.05)
    rho, sig = oracle_rho(seg_data.y, bank)
    return seg_data.y, sub, rho, sig


def test_tc_paper_bank_subset_error(tctx, paper_subset):
    prec, ctx = tctx
    y, sub, rho, sig = paper_subset
    seg = ctx.bege_load_segment(y)
    bid = ctx.bege_define_bank(sub)
    got = np.concatenate([ctx.bege_dump_correlation(seg, bid, k0, min(k0 + 64, len(sub)))
                          for k0 in range(0, len(sub), 64)])
    err = np.max(np.abs(got - rho), axis=1) / sig
    rms = np.sqrt(np.mean((got - rho) ** 2, axis=1)) / sig
    print(f"{PRECISIONS[prec]} N=2^16 paper bank, {len(sub)} templates: max|err| {err.max():.2e} "
          f"sigma (median {np.median(err):.2e}), rms {rms.max():.2e} sigma")
    assert np.all(err <= TOL_TC), err.max()
    for h in (bid, seg):
        ctx.bege_release(h)


def _tail_map(recs):
    key = recs["tmpl"].astype(np.int64) << 32 | recs["lag"].astype(np.int64)
    order = np.argsort(key)
    return key[order], recs["value"][order]


@pytest.mark.parametrize("prec", [1, 2], ids=["bf16x3", "fp16x3"])
def test_tc_paper_scale_tails_match_fp32_path(prec):
    """The N = 2^16 x 2^20-chirp workload: the precision form's tail set is
    the FP32 path's except entries within 2e-3 sigma of the threshold, and
    the common entries agree within 2e-3 sigma."""
    kappa = 5.5
    seg_data, params = S.paper_case(seed=2017)
    out = {}
    for p in (0, prec):
        ctx = make_ctx(tail_capacity=1 << 25, precision=p)
        seg = ctx.bege_load_segment(seg_data.y)
        bid = ctx.bege_define_bank(params, tau=1.0, taper_frac=0.05)
        job = ctx.bege_correlate(seg, bid, 0, len(params), kappa)
        recs, total = ctx.bege_fetch_tails(job)
        assert total == len(recs)
        out[p] = (_tail_map(recs), ctx.bege_get_sigma(job, len(params)))
        ctx.close()
    (k32, v32), sig32 = out[0]
    (ktc, vtc), sigtc = out[prec]
    assert np.max(np.abs(sigtc / sig32 - 1)) <= TOL_SIGMA_TC
    both, i32, itc = np.intersect1d(k32, ktc, assume_unique=True, return_indices=True)
    tmpl = (both >> 32).astype(np.int64)
    err = np.abs(v32[i32] - vtc[itc]) / sig32[tmpl]
    only = np.concatenate([np.setdiff1d(k32, ktc, assume_unique=True),
                           np.setdiff1d(ktc, k32, assume_unique=True)])
    vals = np.concatenate([v32[np.isin(k32, only)], vtc[np.isin(ktc, only)]])
    t_only = np.concatenate([k32[np.isin(k32, only)], ktc[np.isin(ktc, only)]]) >> 32
    dist = np.abs(np.abs(vals) - kappa * sig32[t_only]) / sig32[t_only]
    print(f"{PRECISIONS[prec]} vs FP32 over 2^20 chirps: {len(both)} common tails, "
          f"{len(only)} only in one set (all within {dist.max() if len(dist) else 0:.1e} sigma "
          f"of the threshold), max value difference {err.max():.2e} sigma")
    assert len(both) > 1e6
    assert np.all(err <= TOL_TC)
    assert np.all(dist <= TOL_TC)


def _sorted(recs):
    key = recs["tmpl"].astype(np.int64) << 32 | recs["lag"].astype(np.int64)
    return recs[np.argsort(key)]


def test_tc_subrange_equals_full_run(tctx):
    """Each template is computed on its own: a range [k0, k1) of the bank
    gives bitwise the records and sigma of those rows in a full run, and a
    repeated run is bitwise the same."""
    prec, ctx = tctx
    seg_data, params = S.small_case()
    seg = ctx.bege_load_segment(seg_data.y)
    bid = ctx.bege_define_bank(params)
    full = ctx.bege_correlate(seg, bid, 0, len(params), 4.0)
    r_full, _ = ctx.bege_fetch_tails(full)
    s_full = ctx.bege_get_sigma(full, len(params))
    again = ctx.bege_correlate(seg, bid, 0, len(params), 4.0)
    r_again, _ = ctx.bege_fetch_tails(again)
    assert np.array_equal(_sorted(r_full), _sorted(r_again))
    k0, k1 = 5, 37
    part = ctx.bege_correlate(seg, bid, k0, k1, 4.0)
    r_part, _ = ctx.bege_fetch_tails(part)
    s_part = ctx.bege_get_sigma(part, k1 - k0)
    sel = r_full[(r_full["tmpl"] >= k0) & (r_full["tmpl"] < k1)]
    assert len(sel) > 0
    assert np.array_equal(_sorted(sel), _sorted(r_part))
    assert np.array_equal(s_full[k0:k1], s_part)
    from paper_1708_01609_gb300.binding import BegeError
    with pytest.raises(BegeError):
        ctx.bege_correlate(seg, bid, 7, 7, 4.0)  # an empty range is an argument error
    for h in (full, again, part, bid, seg):
        ctx.bege_release(h)


def test_tc_tail_overflow_keeps_count():
    """A device tail buffer smaller than the tails: the true count is
    returned and the records kept are real tails of the full set."""
    seg_data, params = S.small_case()
    c = make_ctx(tail_capacity=64, precision=1)
    seg = c.bege_load_segment(seg_data.y)
    bid = c.bege_define_bank(params)
    job = c.bege_correlate(seg, bid, 0, len(params), 4.0)
    recs, total = c.bege_fetch_tails(job, capacity=64)
    c.close()
    big = make_ctx(tail_capacity=1 << 20, precision=1)
    seg = big.bege_load_segment(seg_data.y)
    bid = big.bege_define_bank(params)
    job = big.bege_correlate(seg, bid, 0, len(params), 4.0)
    allrecs, total_all = big.bege_fetch_tails(job)
    big.close()
    assert total == total_all > 64
    assert len(recs) == 64
    keys = set(zip(allrecs["tmpl"].tolist(), allrecs["lag"].tolist()))
    assert all((int(t), int(l)) in keys for t, l in zip(recs["tmpl"], recs["lag"]))
