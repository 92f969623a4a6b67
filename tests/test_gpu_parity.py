"""GPU parity: libbege (through its C ABI) against the FP64 oracle.

Tolerances (from the required bar for the FP32 path): correlation values
within 1e-5 sigma_k of the oracle, sigma_k within 1e-6 relative, tail sets
identical except entries within 1e-3 sigma_k of the threshold.
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from gpu_helpers import TOL_FP32, compare_tails, make_ctx, oracle_rho

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = make_ctx(tail_capacity=1 << 25)
    yield c
    c.close()


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


# ---------------------------------------------------------------------------
# S1: segment spectrum
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1 << 10, 1 << 11, 1 << 12, 1 << 13, 1 << 14, 1 << 15, 1 << 16,
                               1 << 17])
def test_segment_spectrum(ctx, n):
    """D_j = sum_n y[n] e^{-2 pi i j n/N}, j = 0..N/2 (Eq. 3S first step),
    against the oracle's FP64 FFT; includes DC and Nyquist content."""
    y = rng(n).standard_normal(n).astype(np.float32) + np.float32(0.25)
    seg = ctx.bege_load_segment(y)
    d = ctx.bege_get_segment_spectrum(seg)
    ref = O.fft(y.astype(np.float64))[: n // 2 + 1]
    rms = np.sqrt(np.mean(np.abs(ref) ** 2))
    assert np.max(np.abs(d - ref)) <= 2e-6 * rms * np.log2(n)
    ctx.bege_release(seg)


# ---------------------------------------------------------------------------
# S2-S5: full correlation (debug dump), identical FP32 inputs on both sides
# ---------------------------------------------------------------------------
DUMP_CASES = [
    (1 << 10, 1024), (1 << 10, 301), (1 << 11, 1000), (1 << 12, 4096), (1 << 13, 4096),
    (1 << 14, 4096), (1 << 14, 16384), (1 << 14, 7), (1 << 15, 4096), (1 << 15, 9999),
    (1 << 16, 4096), (1 << 16, 65536), (1 << 17, 4096), (1 << 17, 8191),
    # degenerate and maximum lengths: a one-sample template (rho = w0 y), and
    # the longest template in the longest segment (the folded first pass)
    (1 << 12, 1), (1 << 16, 1), (1 << 17, 65536),
]


@pytest.mark.parametrize("n,length", DUMP_CASES)
def test_correlation_dump_matches_oracle(ctx, n, length):
    """Every lag of rho_k (Eq. A1 via Eq. 3S) within 1e-5 sigma_k, and the
    Parseval sigma_k (Eq. PT) within 1e-6 relative; 6 templates (a ragged
    count against the cluster grid), random FP32 samples."""
    r = rng(n + length)
    y = S.band_limited_noise(n, n + 3)
    y = (y + 0.1 * r.standard_normal(n)).astype(np.float32)   # some out-of-band power too
    bank = S.random_samples_bank(6, length, n * 7 + length)
    seg = ctx.bege_load_segment(y)
    bid = ctx.bege_define_bank_samples(bank)
    got = ctx.bege_dump_correlation(seg, bid, 0, 6)
    rho, sig = oracle_rho(y, bank.astype(np.float64))
    err = np.max(np.abs(got - rho), axis=1) / sig
    assert np.all(err <= TOL_FP32), err
    job = ctx.bege_correlate(seg, bid, 0, 6, 5.0)
    sg = ctx.bege_get_sigma(job, 6)
    assert np.all(np.abs(sg / sig - 1) <= 1e-6), sg / sig - 1
    for h in (job, bid, seg):
        ctx.bege_release(h)


def test_injection_recovered_noise_free(ctx):
    """A unit-norm template injected at lag l with amplitude A into an
    otherwise empty segment reads rho[l] = A (to FP32 rounding) and is the
    only lag above 0.5 A once the template's sidelobes are below it."""
    n, length, lag, a = 1 << 16, 4096, 40000, 9.0
    w = S.chirp_signal(1100.0, 60.0, length)
    y = np.zeros(n)
    y[(lag + np.arange(length)) % n] = a * w
    seg = ctx.bege_load_segment(y.astype(np.float32))
    bid = ctx.bege_define_bank_samples(w[None, :].astype(np.float32))
    rho = ctx.bege_dump_correlation(seg, bid, 0, 1)[0]
    assert abs(rho[lag] - a) < 1e-5 * a
    assert int(np.argmax(np.abs(rho))) == lag


# ---------------------------------------------------------------------------
# Bank synthesis (chirps of Sec. 3)
# ---------------------------------------------------------------------------
def test_chirp_bank_matches_oracle(ctx):
    """Device chirps (fixed-point phase, FP64 sin/taper/norm, stored FP32)
    equal the oracle's FP64 chirps to FP32 rounding."""
    params = np.concatenate([S.grid_small(), S.grid_paper(4, 4), [[2047.9, 0.0], [350.0, 200.0]]])
    bid = ctx.bege_define_bank(params, tau=1.0, taper_frac=0.05)
    got = ctx.bege_get_bank_samples(bid, 0, len(params)).astype(np.float64)
    ref = O.chirp_bank(params, 4096.0, 4096, 0.05)
    scale = np.max(np.abs(ref), axis=1, keepdims=True)
    assert np.max(np.abs(got - ref) / scale) < 1e-6
    ctx.bege_release(bid)
    # tau = 0.5 s (L = 2048), no taper
    bid = ctx.bege_define_bank(params[:8], tau=0.5, taper_frac=0.0)
    got = ctx.bege_get_bank_samples(bid, 0, 8).astype(np.float64)
    ref = O.chirp_bank(params[:8], 4096.0, 2048, 0.0)
    assert np.max(np.abs(got - ref)) < 1e-6 * np.max(np.abs(ref))
    ctx.bege_release(bid)


def test_symmetric_chirp_bank_matches_oracle(ctx):
    """Time-symmetric chirps (Fig. 2 caption) synthesised on the device equal
    the oracle's FP64 ones to FP32 rounding (tau 1 s with taper, 0.5 s without)."""
    params = np.concatenate([S.grid_small(), S.grid_paper(4, 4), [[2047.9, 0.0], [350.0, 200.0]]])
    for tau, frac, length in ((1.0, 0.05, 4096), (0.5, 0.0, 2048)):
        bid = ctx.bege_define_bank(params, tau=tau, taper_frac=frac, symmetric=True)
        got = ctx.bege_get_bank_samples(bid, 0, len(params)).astype(np.float64)
        ref = O.chirp_bank(params, 4096.0, length, frac, symmetric=True)
        scale = np.max(np.abs(ref), axis=1, keepdims=True)
        assert np.max(np.abs(got - ref) / scale) < 1e-6
        assert np.allclose(got, got[:, ::-1], rtol=0, atol=2e-7 * scale.max())
        ctx.bege_release(bid)


@pytest.mark.parametrize("n", [1 << 14, 1 << 17])
def test_symmetric_bank_finds_a_descending_chirp(ctx, n):
    """Noise (N = 2^14, and 2^17 for the interleaved-column kernel with 16
    columns) with a time-reversed (descending) chirp injected at lag 5000:
    the symmetric bank's tails match the oracle's and contain the injection
    at its template, which the plain bank misses."""
    params = S.grid_small()
    lag, k = 5000, 27
    f0, fd = params[k]
    y = S.band_limited_noise(n, 77).astype(np.float64)
    down = S.chirp_signal(f0, fd, 4096)[::-1]
    y = S.inject(y, down, lag, 20.0 * S.expected_filter_rms(n))
    kappa = 5.0
    seg = ctx.bege_load_segment(y)
    bid = ctx.bege_define_bank(params, symmetric=True)
    job = ctx.bege_correlate(seg, bid, 0, len(params), kappa)
    recs, total = ctx.bege_fetch_tails(job)
    bank = O.chirp_bank(params, 4096.0, 4096, 0.05, symmetric=True)
    rho, sig = oracle_rho(y, bank)
    compare_tails(recs, {kk: (rho[kk], sig[kk]) for kk in range(len(params))}, kappa)
    assert any((int(r["tmpl"]), int(r["lag"])) == (k, lag) for r in recs)
    plain = ctx.bege_define_bank(params)
    job2 = ctx.bege_correlate(seg, plain, 0, len(params), kappa)
    recs2, _ = ctx.bege_fetch_tails(job2)
    assert not any((int(r["tmpl"]), int(r["lag"])) == (k, lag) for r in recs2)
    for h in (job, job2, bid, plain, seg):
        ctx.bege_release(h)


# ---------------------------------------------------------------------------
# S6/S7: tails of the N = 2^14 parity case
# ---------------------------------------------------------------------------
def test_small_case_tails(ctx):
    """N = 2^14, 64 chirps (8 f0 x 8 fdot), one 20-sigma injection at lag
    5000, kappa = 5: tail sets and values against the oracle."""
    seg_data, params = S.small_case()
    kappa = 5.0
    seg = ctx.bege_load_segment(seg_data.y)
    bid = ctx.bege_define_bank(params, tau=1.0, taper_frac=0.05)
    job = ctx.bege_correlate(seg, bid, 0, len(params), kappa)
    recs, total = ctx.bege_fetch_tails(job)
    assert total == len(recs)
    sg = ctx.bege_get_sigma(job, len(params))
    bank = O.chirp_bank(params, 4096.0, 4096, 0.05)
    rho, sig = oracle_rho(seg_data.y, bank)
    assert np.all(np.abs(sg / sig - 1) <= 1e-6)
    summary = compare_tails(recs, {k: (rho[k], sig[k]) for k in range(len(params))}, kappa)
    k_inj, lag, _ = seg_data.injections[0]
    assert any((int(r["tmpl"]), int(r["lag"])) == (k_inj, lag) for r in recs)
    assert summary["matched"] > 0
    for h in (job, bid, seg):
        ctx.bege_release(h)


# ---------------------------------------------------------------------------
# Paper-scale workload: N = 2^16, 2^20 chirps, 32 injections, kappa = 5.5
# ---------------------------------------------------------------------------
def test_paper_scale_sampled(ctx):
    """The benchmarked configuration in the benchmarked launch: all 2^20
    templates in one correlate call; the oracle checks sigma and tails of a
    sample of templates (every injected template, its grid neighbours, the
    first and last rows, and 24 random rows), and every injection must be a
    tail at its template and lag."""
    seg_data, params = S.paper_case()
    kappa = 5.5
    seg = ctx.bege_load_segment(seg_data.y)
    bid = ctx.bege_define_bank(params, tau=1.0, taper_frac=0.05)
    job = ctx.bege_correlate(seg, bid, 0, len(params), kappa)
    recs, total = ctx.bege_fetch_tails(job)
    assert total == len(recs) and total > 0
    sg = ctx.bege_get_sigma(job, len(params))
    assert np.all(np.isfinite(sg)) and np.all(sg > 0)
    keys = recs["tmpl"].astype(np.uint64) << np.uint64(32) | recs["lag"].astype(np.uint64)
    inj = np.array([(k << 32) | lag for k, lag, _ in seg_data.injections], np.uint64)
    assert np.all(np.isin(inj, keys)), "an injection is not a tail at its template and lag"
    sample = {0, len(params) - 1}
    for k, _, _ in seg_data.injections:
        sample.update({k, max(0, k - 1), min(len(params) - 1, k + 1)})
    sample.update(rng(99).integers(0, len(params), 24).tolist())
    sample = sorted(sample)
    bank = O.chirp_bank(params[sample], 4096.0, 4096, 0.05)
    rho, sig = oracle_rho(seg_data.y, bank)
    assert np.all(np.abs(sg[sample] / sig - 1) <= 1e-6)
    ref = {k: (rho[i], sig[i]) for i, k in enumerate(sample)}
    compare_tails(recs, ref, kappa, tmpl_subset=set(sample))
    for h in (job, bid, seg):
        ctx.bege_release(h)


@pytest.mark.parametrize("lg", [14, 15, 17])
def test_full_bank_sampled_other_lengths(ctx, lg):
    """All 2^20 chirps in one correlate call against noise segments of the
    other supported lengths (4 s, 8 s and the longest, 32 s); the oracle
    checks sigma and tails of a sample of templates."""
    _, params = S.paper_case()
    n = 1 << lg
    y = S.band_limited_noise(n, 700 + lg)
    kappa = 5.0
    seg = ctx.bege_load_segment(y)
    bid = ctx.bege_define_bank(params, tau=1.0, taper_frac=0.05)
    job = ctx.bege_correlate(seg, bid, 0, len(params), kappa)
    recs, total = ctx.bege_fetch_tails(job)
    assert total == len(recs) and total > 0
    sg = ctx.bege_get_sigma(job, len(params))
    sample = sorted({0, len(params) - 1} | set(rng(lg).integers(0, len(params), 14).tolist()))
    bank = O.chirp_bank(params[sample], 4096.0, 4096, 0.05)
    rho, sig = oracle_rho(y, bank)
    assert np.all(np.abs(sg[sample] / sig - 1) <= 1e-6)
    ref = {k: (rho[i], sig[i]) for i, k in enumerate(sample)}
    compare_tails(recs, ref, kappa, tmpl_subset=set(sample))
    for h in (job, bid, seg):
        ctx.bege_release(h)


# ---------------------------------------------------------------------------
# Edge cases and errors
# ---------------------------------------------------------------------------
def test_template_subrange_and_single(ctx):
    """k_begin > 0 and a single template give the same rows as the full call."""
    n = 1 << 16
    y = S.band_limited_noise(n, 5)
    bank = S.random_samples_bank(9, 4096, 6)
    seg = ctx.bege_load_segment(y)
    bid = ctx.bege_define_bank_samples(bank)
    full = ctx.bege_dump_correlation(seg, bid, 0, 9)
    part = ctx.bege_dump_correlation(seg, bid, 4, 9)
    one = ctx.bege_dump_correlation(seg, bid, 7, 8)
    assert np.array_equal(full[4:], part)
    assert np.array_equal(full[7], one[0])
    for h in (bid, seg):
        ctx.bege_release(h)


def test_overflow_reports_true_count(ctx):
    """kappa = 0 makes every non-zero lag a tail; a small host buffer gets the
    first records and BEGE_EOVERFLOW semantics (true total returned)."""
    n = 1 << 12
    y = S.band_limited_noise(n, 8)
    bank = S.random_samples_bank(3, 1000, 9)
    seg = ctx.bege_load_segment(y)
    bid = ctx.bege_define_bank_samples(bank)
    job = ctx.bege_correlate(seg, bid, 0, 3, 0.0)
    recs, total = ctx.bege_fetch_tails(job, capacity=100)
    assert len(recs) == 100
    assert 3 * n - 10 <= total <= 3 * n
    recs_all, total2 = ctx.bege_fetch_tails(job, capacity=4 * n)
    assert total2 == total == len(recs_all)
    keys = set(zip(recs_all["tmpl"].tolist(), recs_all["lag"].tolist()))
    assert len(keys) == total
    for h in (job, bid, seg):
        ctx.bege_release(h)


def test_device_capacity_overflow():
    """A context whose device tail buffer is smaller than the tail count keeps
    the first records and still counts every tail."""
    from paper_1708_01609_gb300 import binding
    c = make_ctx(tail_capacity=64)
    n = 1 << 12
    seg = c.bege_load_segment(S.band_limited_noise(n, 8))
    bid = c.bege_define_bank_samples(S.random_samples_bank(2, 500, 1))
    job = c.bege_correlate(seg, bid, 0, 2, 0.0)
    recs, total = c.bege_fetch_tails(job, capacity=1 << 16)
    assert len(recs) == 64 and total > 64
    c.close()
    assert binding.BEGE_EOVERFLOW == -4


def test_repeatable(ctx):
    """Two runs give bit-identical sigma and the same tail set (record order
    across CTAs may differ)."""
    seg_data, params = S.small_case(77)
    seg = ctx.bege_load_segment(seg_data.y)
    bid = ctx.bege_define_bank(params)
    out = []
    for _ in range(2):
        job = ctx.bege_correlate(seg, bid, 0, len(params), 4.0)
        recs, _ = ctx.bege_fetch_tails(job)
        out.append((ctx.bege_get_sigma(job, len(params)), np.sort(recs, order=["tmpl", "lag"])))
        ctx.bege_release(job)
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    for h in (bid, seg):
        ctx.bege_release(h)


def test_device_segment_equals_host_segment(ctx):
    import torch
    n = 1 << 15
    y = S.band_limited_noise(n, 12)
    t = torch.from_numpy(y).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    s1 = ctx.bege_load_segment(y)
    s2 = ctx.bege_load_segment_device(t.data_ptr(), n, 0, stream)
    torch.cuda.synchronize()
    assert np.array_equal(ctx.bege_get_segment_spectrum(s1), ctx.bege_get_segment_spectrum(s2))
    ctx.bege_release(s1)
    ctx.bege_release(s2)


def test_invalid_arguments(ctx):
    from paper_1708_01609_gb300.binding import BegeError
    with pytest.raises(BegeError) as e:
        ctx.bege_load_segment(np.zeros(1000, np.float32))      # not a power of two
    assert e.value.code == -1
    with pytest.raises(BegeError):
        ctx.bege_load_segment(np.zeros(1 << 18, np.float32))   # too long
    seg = ctx.bege_load_segment(np.zeros(1 << 10, np.float32))
    bid = ctx.bege_define_bank_samples(np.ones((2, 2048), np.float32))
    with pytest.raises(BegeError):
        ctx.bege_correlate(seg, bid, 0, 2, 5.0)                  # L > N
    bid2 = ctx.bege_define_bank_samples(np.ones((2, 16), np.float32))
    with pytest.raises(BegeError):
        ctx.bege_correlate(seg, bid2, 0, 3, 5.0)                 # range outside bank
    with pytest.raises(BegeError) as e:
        ctx.bege_correlate(seg, bid2, 1, 1, 5.0)                 # empty range
    assert e.value.code == -1
    with pytest.raises(BegeError):
        ctx.bege_correlate(seg, bid2, 0, 2, float("nan"))
    with pytest.raises(BegeError):
        ctx.bege_correlate(seg, bid2, 0, 2, float("inf"))
    with pytest.raises(BegeError):
        ctx.bege_correlate(seg, 999999, 0, 1, 5.0)               # unknown handle
    with pytest.raises(BegeError):
        ctx.bege_release(999999)
    for h in (bid, bid2, seg):
        ctx.bege_release(h)


def test_zero_segment_gives_no_tails(ctx):
    """All-zero data: sigma = 0 and no lag exceeds kappa * 0 (strict >)."""
    seg = ctx.bege_load_segment(np.zeros(1 << 14, np.float32))
    bid = ctx.bege_define_bank(S.grid_small()[:4])
    job = ctx.bege_correlate(seg, bid, 0, 4, 5.0)
    recs, total = ctx.bege_fetch_tails(job)
    assert total == 0
    assert np.all(ctx.bege_get_sigma(job, 4) == 0)
    for h in (job, bid, seg):
        ctx.bege_release(h)


def test_budget_refusal():
    from paper_1708_01609_gb300.binding import BegeError
    c = make_ctx(hbm_budget_bytes=1 << 20)
    with pytest.raises(BegeError) as e:
        c.bege_define_bank_samples(np.ones((1000, 4096), np.float32))
    assert e.value.code == -3
    c.close()


@pytest.mark.parametrize("n", [1 << 14, 1 << 15, 1 << 16, 1 << 17])
def test_every_launch_shape_matches_oracle(ctx, n):
    """Every compiled launch shape (columns per CTA, threads per CTA) gives
    the same correlation (bitwise: each column FFT does identical arithmetic)
    and sigma within 1e-6 of the oracle; the autotuner picks one of them."""
    y = S.band_limited_noise(n, 21)
    bank = S.random_samples_bank(5, 4096, 22)
    seg = ctx.bege_load_segment(y)
    bid = ctx.bege_define_bank_samples(bank)
    rho, sig = oracle_rho(y, bank.astype(np.float64))
    shapes = ctx.bege_list_configs(n)
    assert len(shapes) >= 1
    dumps = []
    for nc, threads in shapes:
        ctx.bege_set_config(n, nc, threads)
        assert ctx.bege_get_config(n) == (nc, threads)
        d = ctx.bege_dump_correlation(seg, bid, 0, 5)
        assert np.all(np.max(np.abs(d - rho), axis=1) / sig <= TOL_FP32)
        job = ctx.bege_correlate(seg, bid, 0, 5, 4.0)
        assert np.all(np.abs(ctx.bege_get_sigma(job, 5) / sig - 1) <= 1e-6)
        ctx.bege_release(job)
        dumps.append(d)
    for d in dumps[1:]:
        assert np.array_equal(d, dumps[0])
    best = ctx.bege_autotune(seg, bid, 0, 5, reps=1)
    assert best > 0 and ctx.bege_get_config(n) in shapes
    for h in (bid, seg):
        ctx.bege_release(h)
