"""Per-lag maximum over the bank (Eq. Ak, Aa, BA) on the GPU: against the
oracle's projection, against the per-lag maximum of the job's own all-hit
records (bitwise: same FP32 values), and in Table 3's encoding."""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from gpu_helpers import make_ctx, oracle_rho

pytestmark = pytest.mark.gpu


def band_case(n):
    """The 64-chirp parity bank against a segment of n samples with one
    20-sigma injection of template 27: the N = 2^14 parity case itself, or
    N = 2^16 (the clustered, interleaved-column kernel)."""
    if n == 1 << 14:
        return S.small_case()
    params = S.grid_small()
    return S.make_segment(n, params, 1, 1234, fixed=[(27, 20000, 20.0)]), params


def projection_of_records(recs, sigma, kappa, n, k0=0):
    """The kernel's rule on its own records: v > fl(kappa sigma), key
    fl(v (1 / sigma)), ties to the smaller template; in FP32."""
    sig = sigma.astype(np.float32)
    k = recs["tmpl"].astype(np.int64) - k0
    v = recs["value"].astype(np.float32)
    thr = np.float32(kappa) * sig[k]
    sel = v > thr
    v, k, lag = v[sel], k[sel], recs["lag"][sel].astype(np.int64)
    snr = v * (np.float32(1.0) / sig[k])
    order = np.lexsort((k, -snr.astype(np.float64), lag))   # per lag: largest snr, then smallest k
    lag, snr, k = lag[order], snr[order], k[order]
    first = np.ones(len(lag), bool)
    first[1:] = lag[1:] != lag[:-1]
    out_snr = np.zeros(n, np.float32)
    out_k = np.full(n, -1, np.int32)
    out_snr[lag[first]] = snr[first]
    out_k[lag[first]] = (k[first] + k0).astype(np.int32)
    return out_snr, out_k


@pytest.mark.parametrize("n_seg", [1 << 14, 1 << 16], ids=["N16384", "N65536"])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16x3"])
def test_projection_matches_oracle(prec, n_seg):
    seg_data, params = band_case(n_seg)
    kappa = 4.0
    ctx = make_ctx(tail_capacity=1 << 20, precision=prec)
    seg = ctx.bege_load_segment(seg_data.y)
    bid = ctx.bege_define_bank(params)
    job = ctx.bege_correlate_max(seg, bid, 0, len(params), kappa)
    snr, tmpl = ctx.bege_fetch_max(job, len(seg_data.y))
    ctx.close()
    bank = O.chirp_bank(params, 4096.0, 4096, 0.05)
    rho, sig = oracle_rho(seg_data.y, bank)
    o_snr, o_tmpl = O.max_projection(rho, sig, kappa)
    tol = 1e-5 if prec == 0 else 2e-3
    both = (tmpl >= 0) & (o_tmpl >= 0)
    assert both.sum() > 100
    at_gpu_pick = rho[tmpl[both], np.flatnonzero(both)] / sig[tmpl[both]]
    assert np.all(np.abs(snr[both] - at_gpu_pick) <= tol)          # value of the kept hit
    assert np.all(at_gpu_pick >= o_snr[both] - 2 * tol)            # it is a maximum
    only = (tmpl >= 0) != (o_tmpl >= 0)
    # a lag with a hit on one side only has its best value at the threshold
    best = np.where(o_tmpl >= 0, o_snr, (rho / sig[:, None]).max(axis=0))
    assert np.all(np.abs(best[only] - kappa) <= max(1e-3, 2 * tol))
    k_inj, lag, _ = seg_data.injections[0]
    assert tmpl[lag] >= 0 and snr[lag] >= rho[k_inj, lag] / sig[k_inj] - tol


@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16x3"])
def test_projection_is_the_maximum_of_the_records(prec):
    """65536 chirps of the paper bank at N = 2^16 with its injections (many
    templates hit the same lags): the projection equals, bitwise, the per-lag
    maximum recomputed from the job's own records and sigma."""
    seg_data, params = S.paper_case(seed=2017)
    kappa, nt, n = 5.5, 65536, len(seg_data.y)
    ctx = make_ctx(tail_capacity=1 << 24, precision=prec)
    seg = ctx.bege_load_segment(seg_data.y)
    bid = ctx.bege_define_bank(params[:nt], tau=1.0, taper_frac=0.05)
    job = ctx.bege_correlate_max(seg, bid, 0, nt, kappa)
    snr, tmpl = ctx.bege_fetch_max(job, n)
    recs, total = ctx.bege_fetch_tails(job)
    sigma = ctx.bege_get_sigma(job, nt)
    ctx.close()
    assert total == len(recs) > 1000
    r_snr, r_tmpl = projection_of_records(recs, sigma, kappa, n)
    assert np.array_equal(tmpl, r_tmpl)
    assert np.array_equal(snr.view(np.uint32), r_snr.view(np.uint32))
    assert (tmpl >= 0).sum() > 100


def test_table3_encoding_of_a_gpu_projection():
    from paper_1708_01609_gb300.output import table3_rows
    seg_data, params = S.small_case()
    ctx = make_ctx(tail_capacity=1 << 20)
    seg = ctx.bege_load_segment(seg_data.y)
    bid = ctx.bege_define_bank(params)
    job = ctx.bege_correlate_max(seg, bid, 0, len(params), 4.0)
    snr, tmpl = ctx.bege_fetch_max(job, len(seg_data.y))
    ctx.close()
    rows = table3_rows(snr, tmpl, params[:, 0])
    ref = O.table3_rows(snr.astype(np.float64), tmpl.astype(np.int64), params[:, 0])
    assert len(rows) == len(ref) > 0
    assert np.array_equal(rows["offset"], ref["offset"])
    assert np.array_equal(rows["rho1000"], ref["rho1000"])
    assert np.array_equal(rows["f0"], ref["f0"])
    assert rows["rho1000"].min() >= 4000


def test_fetch_max_rejects_plain_jobs_and_wrong_length():
    from paper_1708_01609_gb300.binding import BegeError
    seg_data, params = S.small_case()
    ctx = make_ctx(tail_capacity=1 << 20)
    seg = ctx.bege_load_segment(seg_data.y)
    bid = ctx.bege_define_bank(params)
    plain = ctx.bege_correlate(seg, bid, 0, len(params), 4.0)
    with pytest.raises(BegeError):
        ctx.bege_fetch_max(plain, len(seg_data.y))
    job = ctx.bege_correlate_max(seg, bid, 0, len(params), 4.0)
    with pytest.raises(BegeError):
        ctx.bege_fetch_max(job, len(seg_data.y) // 2)
    ctx.close()



@pytest.mark.parametrize("n_seg", [1 << 14, 1 << 16], ids=["N16384", "N65536"])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16x3"])
def test_band_tails_match_oracle(prec, n_seg):
    """Tails over a finite band (Sec. 5): kappa_lo sigma < |rho| < kappa_hi
    sigma on the parity bank (N = 2^14 and 2^16), against the oracle; entries within the
    tolerance band of either end are excluded from set parity."""
    seg_data, params = band_case(n_seg)
    lo, hi = 3.5, 4.25
    ctx = make_ctx(tail_capacity=1 << 20, precision=prec)
    seg = ctx.bege_load_segment(seg_data.y)
    bid = ctx.bege_define_bank(params)
    job = ctx.bege_correlate_band(seg, bid, 0, len(params), lo, hi)
    recs, total = ctx.bege_fetch_tails(job)
    ctx.close()
    assert total == len(recs)
    bank = O.chirp_bank(params, 4096.0, 4096, 0.05)
    rho, sig = oracle_rho(seg_data.y, bank)
    tol = 1e-5 if prec == 0 else 2e-3
    near = max(1e-3, tol)
    got = {(int(t), int(l)): float(v) for t, l, v in zip(recs["tmpl"], recs["lag"], recs["value"])}
    n_ref = 0
    for k in range(len(params)):
        ref = O.tails_band(rho[k], sig[k], lo, hi, k)
        for n, v in zip(ref["lag"], ref["value"]):
            a = abs(v) / sig[k]
            if (k, int(n)) not in got:
                assert min(abs(a - lo), abs(a - hi)) <= near, (k, n, a)
                continue
            n_ref += 1
            assert abs(got[(k, int(n))] - v) <= tol * sig[k]
    for (k, n), v in got.items():
        a = abs(rho[k][n]) / sig[k]
        assert lo - near <= a <= hi + near, (k, n, a)
    assert n_ref > 300  # from noise alone ~470 at N = 2^14 (four times that at 2^16), plus the injection


@pytest.mark.parametrize("n_seg", [1 << 14, 1 << 16], ids=["N16384", "N65536"])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16x3"])
def test_linear_tails_match_oracle(prec, n_seg):
    """Overlap-save mask: tails only at lags n <= N - L (the windows that do
    not wrap), on the parity bank (N = 2^14 and 2^16) against the oracle's tails_linear; sigma
    is the full Parseval value."""
    seg_data, params = band_case(n_seg)
    kappa, length, n = 4.0, 4096, len(seg_data.y)
    ctx = make_ctx(tail_capacity=1 << 20, precision=prec)
    seg = ctx.bege_load_segment(seg_data.y)
    bid = ctx.bege_define_bank(params)
    job = ctx.bege_correlate_ex(seg, bid, 0, len(params), kappa, linear=True)
    recs, total = ctx.bege_fetch_tails(job)
    sg = ctx.bege_get_sigma(job, len(params))
    full = ctx.bege_correlate(seg, bid, 0, len(params), kappa)
    r_full, _ = ctx.bege_fetch_tails(full)
    ctx.close()
    assert total == len(recs)
    assert np.all(recs["lag"] <= n - length)
    assert np.sum(r_full["lag"] > n - length) > 0  # the mask removes something here
    bank = O.chirp_bank(params, 4096.0, 4096, 0.05)
    rho, sig = oracle_rho(seg_data.y, bank)
    tol = 1e-5 if prec == 0 else 2e-3
    assert np.max(np.abs(sg / sig - 1)) <= (1e-6 if prec == 0 else 1e-5)
    near = max(1e-3, tol)
    got = {(int(t), int(l)): float(v) for t, l, v in zip(recs["tmpl"], recs["lag"], recs["value"])}
    n_ref = 0
    for k in range(len(params)):
        ref = O.tails_linear(rho[k], sig[k], kappa, length, k)
        lin = O.correlate_linear(bank[k], seg_data.y)
        assert np.allclose(rho[k][:n - length + 1], lin, atol=1e-9)
        for lag, v in zip(ref["lag"], ref["value"]):
            if (k, int(lag)) not in got:
                assert abs(abs(v) / sig[k] - kappa) <= near, (k, lag)
                continue
            n_ref += 1
            assert abs(got[(k, int(lag))] - v) <= tol * sig[k]
    for (k, lag), v in got.items():
        assert abs(rho[k][lag]) / sig[k] >= kappa - near
    assert n_ref > 100


@pytest.mark.parametrize("n_seg", [1 << 14, 1 << 16], ids=["N16384", "N65536"])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16x3"])
def test_ex_options_compose(prec, n_seg):
    """bege_correlate_ex with band, mask and projection together: the
    records are the plain search's records filtered by both rules, and the
    projection is the per-lag maximum of those records."""
    seg_data, params = band_case(n_seg)
    lo, hi, length, n = 3.5, 6.0, 4096, len(seg_data.y)
    ctx = make_ctx(tail_capacity=1 << 20, precision=prec)
    seg = ctx.bege_load_segment(seg_data.y)
    bid = ctx.bege_define_bank(params)
    plain = ctx.bege_correlate(seg, bid, 0, len(params), lo)
    r_plain, _ = ctx.bege_fetch_tails(plain, sort=True)
    sig = ctx.bege_get_sigma(plain, len(params))
    job = ctx.bege_correlate_ex(seg, bid, 0, len(params), lo, kappa_hi=hi, linear=True,
                                project=True)
    recs, total = ctx.bege_fetch_tails(job, sort=True)
    snr, tmpl = ctx.bege_fetch_max(job, n)
    assert np.array_equal(ctx.bege_get_sigma(job, len(params)), sig)
    ctx.close()
    assert total == len(recs)
    s32 = sig.astype(np.float32)[r_plain["tmpl"]]
    keep = (np.abs(r_plain["value"]) < np.float32(hi) * s32) & (r_plain["lag"] <= n - length)
    want = r_plain[keep]
    # the same FP32 values: bitwise equal except where |rho| meets hi sigma in the last bit
    edge = np.abs(np.abs(want["value"]) / s32[keep] - hi) <= 1e-6
    key = lambda r: set(zip(r["tmpl"].tolist(), r["lag"].tolist()))
    assert key(want[~edge]) <= key(recs) <= key(want)
    common = np.isin(want["tmpl"].astype(np.int64) << 32 | want["lag"],
                     recs["tmpl"].astype(np.int64) << 32 | recs["lag"])
    assert np.array_equal(want[common], recs)
    ps, pk = projection_of_records(recs, sig, lo, n)
    assert np.array_equal(ps, snr) and np.array_equal(pk, tmpl)
    assert np.all(tmpl[n - length + 1:] == -1) and np.any(tmpl >= 0)


def test_ex_rejects_bad_options():
    from paper_1708_01609_gb300.binding import BegeError
    seg_data, params = S.small_case()
    ctx = make_ctx(tail_capacity=1 << 16)
    seg = ctx.bege_load_segment(seg_data.y)
    bid = ctx.bege_define_bank(params)
    for kw in ({"kappa": 5.0, "kappa_hi": 4.0}, {"kappa": 5.0, "kappa_hi": 5.0},
               {"kappa": float("nan")}, {"kappa": -1.0}, {"kappa": 5.0, "kappa_hi": float("inf")}):
        with pytest.raises(BegeError):
            ctx.bege_correlate_ex(seg, bid, 0, len(params), **kw)
    import ctypes
    from paper_1708_01609_gb300.binding import bege_search_opts
    o = bege_search_opts(5.0, 0.0, 2, 0)
    jid = ctypes.c_int32()
    assert ctx.lib.bege_correlate_ex(ctx.h, seg, bid, 0, len(params), ctypes.byref(o), None,
                                     ctypes.byref(jid)) != 0
    ctx.close()


def test_two_channel_coincidences():
    """Two detector channels (independent band-limited noise) with the same
    chirp injected at the same offset, each projected on the GPU: the
    simultaneous hits within 50 Hz include the injection, and the counts and
    Table 3 rows equal the oracle's encoding of the same projections."""
    from paper_1708_01609_gb300.output import coincidences, table3_rows_two
    params = S.grid_paper(32, 32)
    n, lag, k = 1 << 16, 20000, 517
    f0, fd = params[k]
    sig_e = S.expected_filter_rms(n)
    ys = [S.inject(S.band_limited_noise(n, 900 + c).astype(np.float64),
                   S.chirp_signal(f0, fd, 4096), lag, 25.0 * sig_e) for c in (0, 1)]
    ctx = make_ctx(tail_capacity=1 << 22)
    bid = ctx.bege_define_bank(params)
    proj = []
    for y in ys:
        seg = ctx.bege_load_segment(y)
        job = ctx.bege_correlate_max(seg, bid, 0, len(params), 5.5)
        proj.append(ctx.bege_fetch_max(job, n))
    ctx.close()
    (s1, t1), (s2, t2) = proj
    c = coincidences(t1, t2, params[:, 0])
    ref = O.coincidences(t1, t2, params[:, 0])
    assert c["hits"] == ref["hits"] and c["simultaneous"] == ref["simultaneous"]
    assert c["within_delta"] == ref["within_delta"] and np.array_equal(c["lags"], ref["lags"])
    assert lag in c["lags"].tolist()
    assert abs(params[t1[lag], 0] - f0) < 50 and abs(params[t2[lag], 0] - f0) < 50
    rows = table3_rows_two(s1, t1, s2, t2, params[:, 0])
    ref_rows = O.table3_rows_two(s1.astype(np.float64), t1, s2.astype(np.float64), t2, params[:, 0])
    assert len(rows) == len(ref_rows) > 0
    for name in ref_rows.dtype.names:
        assert np.array_equal(rows[name], ref_rows[name])


def test_two_channel_search_matches_oracle():
    """Sec. 5 end to end: two channels (independent band-limited noise, the
    same chirp injected at the same offset in both, a second chirp in one
    channel only), each searched on the GPU with the per-lag maximum, against
    the oracle's own per-lag maxima of both channels (from FP64 rho and
    sigma) and the oracle's simultaneous-hit analysis of those.  At every
    lag the two sides keep the same template, except where the choice is not
    fixed by the arithmetic: the lag's best value lies within the tolerance
    of the threshold (a hit on one side only) or two templates' values lie
    within twice the tolerance of each other (a near tie).  Kept values agree
    within 1e-5; the coincidence lag sets differ only at such lags."""
    params = S.grid_paper(16, 32)                    # 512 in-band chirps
    n, kappa, tol = 1 << 16, 4.0, 1e-5
    lag, k, k_one = 20000, 277, 90                 # k_one: injected in channel 0 only
    sig_e = S.expected_filter_rms(n)
    ys = []
    for c in (0, 1):
        y = S.inject(S.band_limited_noise(n, 950 + c).astype(np.float64),
                     S.chirp_signal(*params[k], 4096), lag, 25.0 * sig_e)
        if c == 0:
            y = S.inject(y.astype(np.float64), S.chirp_signal(*params[k_one], 4096), 41000,
                         20.0 * sig_e)
        ys.append(y)
    ctx = make_ctx(tail_capacity=1 << 22)
    bid = ctx.bege_define_bank(params)
    gpu = []
    for y in ys:
        seg = ctx.bege_load_segment(y)
        job = ctx.bege_correlate_max(seg, bid, 0, len(params), kappa)
        gpu.append(ctx.bege_fetch_max(job, n))
    ctx.close()
    bank = O.chirp_bank(params, 4096.0, 4096, 0.05)
    undecided = np.zeros(n, bool)       # lags where the kept template is not fixed
    orc = []
    for (snr, tmpl), y in zip(gpu, ys):
        rho, sig = oracle_rho(y, bank, batch=32)
        val = rho / sig[:, None]
        o_snr, o_tmpl = O.max_projection(rho, sig, kappa)
        orc.append((o_snr, o_tmpl))
        best = val.max(axis=0)
        near_thr = np.abs(best - kappa) <= max(1e-3, 2 * tol)
        second = np.partition(val, -2, axis=0)[-2]
        tie = (best - second) <= 2 * tol
        undecided |= near_thr | tie
        same = (tmpl == o_tmpl)
        assert np.all(same | near_thr | tie)
        both = same & (tmpl >= 0)
        assert both.sum() > 1000
        assert np.all(np.abs(snr[both] - o_snr[both]) <= tol)
        assert tmpl[lag] == o_tmpl[lag] >= 0
    f0 = params[:, 0]
    g = coincidences_of(gpu, f0)
    o = O.coincidences(orc[0][1], orc[1][1], f0)
    assert o["simultaneous"] > 10 and lag in o["lags"].tolist()
    diff = np.setxor1d(g["lags"], o["lags"])
    assert np.all(undecided[diff]), diff[~undecided[diff]]
    assert abs(g["within_delta"] - o["within_delta"]) <= int(undecided.sum())
    for c in (0, 1):
        assert abs(g["hits"][c] - o["hits"][c]) <= int(undecided.sum())


def coincidences_of(proj, f0):
    from paper_1708_01609_gb300.output import coincidences
    (_, t1), (_, t2) = proj
    return coincidences(t1, t2, f0)
