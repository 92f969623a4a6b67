"""Precision form: column FFTs on tcgen05 tensor cores with split 16-bit
operands (BF16x3, FP16x2) and FP32 accumulation, against the FP64 oracle.

Bar for the reduced-precision path: correlation values within 2e-3 sigma of
the oracle; sigma within 1e-3 relative; tail sets identical except entries
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
PRECISIONS = {1: "BF16x3", 2: "FP16x2"}


@pytest.fixture(scope="module", params=[1, 2], ids=["bf16x3", "fp16x2"])
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
    assert serr <= 1e-3
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
