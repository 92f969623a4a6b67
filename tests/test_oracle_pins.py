"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names the passage it checks.  Chosen so that a plausible slip in the
oracle (a sign, a dropped term, a conjugate, an off-by-one in lags, a wrong
Parseval weight, >= for >) fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle as O
import synthetic as S


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------
# FFT (Eq. 3S, sign of Eq. A2)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 4, 8, 64, 1024, 4096])
def test_fft_matches_library(n):
    """Library special case: numpy.fft uses the same e^{-i...} forward kernel."""
    r = rng(n)
    x = r.standard_normal((3, n)) + 1j * r.standard_normal((3, n))
    got = O.fft(x)
    ref = np.fft.fft(x, axis=-1)
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
    inv = O.fft(x, inverse=True)
    ref_inv = np.fft.ifft(x, axis=-1) * n
    assert np.max(np.abs(inv - ref_inv)) <= 1e-12 * max(1.0, np.max(np.abs(ref_inv)))


def test_fft_closed_forms():
    """Closed forms: a delta transforms to ones; exp(+2 pi i q n/N) transforms
    to N at bin q under the forward kernel exp(-2 pi i j n / N) (Eq. A2)."""
    n = 256
    d = np.zeros(n)
    d[0] = 1.0
    assert np.allclose(O.fft(d), np.ones(n), atol=1e-14)
    q = 37
    x = np.exp(2j * np.pi * q * np.arange(n) / n)
    X = O.fft(x)
    expect = np.zeros(n, complex)
    expect[q] = n
    assert np.max(np.abs(X - expect)) < 1e-10
    # round trip with the 1/N of the inverse
    r = rng(5).standard_normal(n)
    assert np.max(np.abs(O.fft(O.fft(r), inverse=True) / n - r)) < 1e-13


def test_fft_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        O.fft(np.zeros(12))


# --------------------------------------------------------------------------
# Correlation (Eq. A1, Eq. 3S)
# --------------------------------------------------------------------------
def test_cosine_closed_form():
    """Eq. A1 against a closed form: y[n] = cos(th n), w[m] = cos(th m), m < L
    gives rho[n] = (L/2) cos(th n) + (1/2) Re[e^{i th n} (1 - e^{2 i th L}) /
    (1 - e^{2 i th})] (sum of a geometric series)."""
    n, length, q = 128, 21, 5
    th = 2 * np.pi * q / n
    y = np.cos(th * np.arange(n))
    w = np.cos(th * np.arange(length))
    nn = np.arange(n)
    geo = (1 - np.exp(2j * th * length)) / (1 - np.exp(2j * th))
    expect = 0.5 * length * np.cos(th * nn) + 0.5 * (np.exp(1j * th * nn) * geo).real
    assert np.max(np.abs(O.correlate_direct(w, y) - expect)) < 1e-12
    assert np.max(np.abs(O.correlate_fft(w, y) - expect)) < 1e-11


@pytest.mark.parametrize("n,length", [(16, 5), (256, 100), (1024, 1024), (1024, 7)])
def test_fft_correlation_equals_direct(n, length):
    """Eq. 3S reproduces Eq. A1 (brute force on small inputs)."""
    r = rng(n + length)
    y = r.standard_normal(n)
    w = r.standard_normal(length)
    a = O.correlate_direct(w, y)
    b = O.correlate_fft(w, y)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a)) * math.log2(n)


@pytest.mark.parametrize("lag", [0, 1, 300, 1023])
@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_injection_recovered_at_lag_and_amplitude(lag, sign):
    """Lag convention y(t+s): a unit-norm template placed at y[l + m] gives
    rho[l] = A exactly, and |rho| peaks there (Cauchy-Schwarz).  Also covers a
    wrap past the end of the segment (circular correlation)."""
    n, length = 1024, 200
    w = rng(3).standard_normal(length)
    w /= np.linalg.norm(w)
    y = np.zeros(n)
    a = 7.25 * sign
    y[(lag + np.arange(length)) % n] += a * w
    rho = O.correlate_fft(w, y)
    assert abs(rho[lag] - a) < 1e-12
    assert int(np.argmax(np.abs(rho))) == lag


def test_self_correlation_is_one():
    """A unit-norm chirp template against itself (zero-padded) gives rho[0] = 1."""
    w = O.chirp_template(1000.0, 50.0, 4096.0, 4096, 0.05)
    y = O.zero_pad(w, 1 << 14)
    rho = O.correlate_fft(w, y)
    assert abs(rho[0] - 1.0) < 1e-12


# --------------------------------------------------------------------------
# sigma (definition below Eq. 3S; Eq. PT)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [16, 1024, 4096])
def test_parseval_identity(n):
    """Parseval: the spectral sigma equals the RMS of rho, including data with
    non-zero DC and Nyquist (all Parseval weights matter)."""
    r = rng(n)
    y = r.standard_normal(n) + 0.3          # non-zero mean -> DC bin
    y[::2] += 0.2                            # Nyquist content
    w = r.standard_normal(min(n, 300))
    p = O.correlation_spectrum(w, y)
    rho = (O.fft(p, inverse=True) / n).real
    assert abs(O.sigma_parseval(p) / O.sigma_rms(rho) - 1.0) < 1e-12


def test_paper_form_needs_vanishing_dc_and_nyquist():
    """Eq. PT as printed equals the full form when DC and Nyquist vanish
    (band-limited data), and differs when they do not."""
    n = 4096
    y = S.band_limited_noise(n, 11).astype(np.float64)
    y -= 0.0
    w = O.chirp_template(900.0, -30.0, 4096.0, 2048, 0.05)
    p = O.correlation_spectrum(w, y)
    p[0] = 0.0
    p[n // 2] = 0.0
    assert abs(O.sigma_parseval(p) / O.sigma_parseval_paper_form(p) - 1) < 1e-13
    p2 = p.copy()
    p2[0] = 50.0 * np.abs(p).max()
    assert O.sigma_parseval(p2) > 1.01 * O.sigma_parseval_paper_form(p2)


@pytest.mark.slow
def test_sigma_matches_ensemble_prediction():
    """On band-limited Gaussian noise the Parseval sigma matches the ensemble
    prediction sigma_E^2 = (s^2/N^2) sum_{in band} 2|W_j|^2 within sampling
    error (200 seeds, 4 standard errors)."""
    n = 4096
    w = O.chirp_template(800.0, 40.0, 4096.0, 2048, 0.05)
    big_w = np.fft.rfft(O.zero_pad(w, n))
    jb = S.band_bins(n)
    s = S.noise_scale(n)
    sig_e2 = (s * s / n / n) * 2.0 * np.sum(np.abs(big_w[jb]) ** 2)
    ratios = []
    for seed in range(200):
        y = S.band_limited_noise(n, 1000 + seed)
        ratios.append(O.sigma_parseval(O.correlation_spectrum(w, y)) ** 2 / sig_e2)
    ratios = np.array(ratios)
    se = ratios.std(ddof=1) / math.sqrt(len(ratios))
    assert abs(ratios.mean() - 1.0) < 4 * se


# --------------------------------------------------------------------------
# Tails (Eq. tail)
# --------------------------------------------------------------------------
def test_tails_strict_and_absolute():
    """|rho| > kappa sigma, strict, on the absolute value (text under Eq. tail)."""
    rho = np.array([0.0, 5.0, -5.0, 5.0000001, -6.0, 4.9])
    t = O.tails(rho, 1.0, 5.0, 9)
    assert t["lag"].tolist() == [3, 4]
    assert t["tmpl"].tolist() == [9, 9]
    assert t["value"].tolist() == [5.0000001, -6.0]


@pytest.mark.slow
def test_noise_tail_rate_is_gaussian():
    """For Gaussian noise the rate of |rho| > kappa sigma is 2 Q(kappa).

    Broadband templates keep the filter output's degrees of freedom high
    (~2 x 1650 Hz x 1 s); a narrowband chirp on a 1 s segment has so few that
    the realised sigma tracks its own peaks and the rate falls below 2 Q."""
    n, kappa = 4096, 3.0
    bank = rng(8).standard_normal((8, 1024))
    counts = []
    for seed in range(40):
        y = S.band_limited_noise(n, 500 + seed)
        counts.append(len(O.search(y, bank, kappa)["tails"]))
    counts = np.array(counts, float)
    expect = math.erfc(kappa / math.sqrt(2)) * n * len(bank)
    se = counts.std(ddof=1) / math.sqrt(len(counts))
    assert abs(counts.mean() - expect) < 4 * se + 0.02 * expect


def test_search_matches_per_template_definition():
    """search() batches, offsets template indices and sorts; compare it with
    the direct definition applied template by template (batch 3 over 7)."""
    n = 256
    r = rng(77)
    y = r.standard_normal(n)
    bank = r.standard_normal((7, 40))
    kappa = 2.0
    got = O.search(y, bank, kappa, k0=100, batch=3, return_rho=True)
    recs = []
    for i, w in enumerate(bank):
        rho = O.correlate_direct(w, y)
        sg = O.sigma_rms(rho)
        assert abs(got["sigma"][i] / sg - 1) < 1e-12
        assert np.max(np.abs(got["rho"][i] - rho)) < 1e-11
        recs.append(O.tails(rho, sg, kappa, 100 + i))
    ref = np.concatenate(recs)
    assert got["tails"]["tmpl"].tolist() == ref["tmpl"].tolist()
    assert got["tails"]["lag"].tolist() == ref["lag"].tolist()
    assert np.allclose(got["tails"]["value"], ref["value"], rtol=0, atol=1e-11)


# --------------------------------------------------------------------------
# Templates (Sec. 3 chirps)
# --------------------------------------------------------------------------
def test_taper_matches_library():
    """Library special case: scipy's Tukey window with the same fraction."""
    sw = pytest.importorskip("scipy.signal.windows")
    for length, frac in [(4096, 0.05), (2048, 0.05), (101, 0.3), (11, 0.5)]:
        assert np.max(np.abs(O.taper(length, frac) - sw.tukey(length, frac))) < 1e-14


def test_chirp_template_closed_form():
    """Scalar evaluation of T(m) sin(2 pi (f0 t + fdot t^2/2)) with math.sin at
    a few samples of the untapered middle; the template is that times 1/norm."""
    f0, fd, fs, length = 1234.5, -87.25, 4096.0, 4096
    w = O.chirp_template(f0, fd, fs, length, 0.05)
    raw = [math.sin(2 * math.pi * (f0 * (m / fs) + 0.5 * fd * (m / fs) ** 2))
           for m in range(length)]
    tap = O.taper(length, 0.05)
    norm = math.sqrt(sum((tap[m] * raw[m]) ** 2 for m in range(length)))
    for m in [0, 1, 57, 102, 103, 2000, 3333, 4095]:
        assert abs(w[m] - tap[m] * raw[m] / norm) < 1e-15
    assert abs(np.dot(w, w) - 1.0) < 1e-13


def test_injected_signal_matches_template():
    """The generator's injected chirp (independent code) equals the oracle's
    template: a noise-free injection of amplitude A reads rho = A at its lag."""
    params = S.grid_small()
    k = 27
    f0, fd = params[k]
    n = 1 << 14
    sig = S.chirp_signal(f0, fd, 4096)
    y = np.zeros(n)
    y[(5000 + np.arange(4096)) % n] = 3.5 * sig
    w = O.chirp_template(f0, fd, 4096.0, 4096, 0.05)
    rho = O.correlate_fft(w, y)
    assert abs(rho[5000] - 3.5) < 1e-12


def test_chirp_spectrum_inside_band():
    """Every chirp of the paper-scale grid sweeps inside 350-2000 Hz: its
    spectral energy more than 50 Hz outside the band (taper and 1 s
    time-limiting leakage only) is tiny."""
    params = S.grid_paper(8, 8)
    n = 1 << 16
    f = np.arange(n // 2 + 1) * 4096.0 / n
    out_band = (f < 300) | (f > 2050)
    for f0, fd in params:
        w = O.chirp_template(f0, fd, 4096.0, 4096, 0.05)
        p = np.abs(np.fft.rfft(O.zero_pad(w, n))) ** 2
        assert p[out_band].sum() / p.sum() < 1e-4


# --------------------------------------------------------------------------
# Recovery and the time-randomisation null (Sec. 5)
# --------------------------------------------------------------------------
def test_small_case_recovers_injection():
    """The N=2^14 parity case: the 20-sigma injection of template 27 at lag
    5000 is a tail of template 27 at lag 5000 with |rho - A| <= 4 sigma."""
    seg, params = S.small_case()
    bank = O.chirp_bank(params, 4096.0, 4096, 0.05)
    res = O.search(seg.y, bank, 5.0)
    k, lag, a = seg.injections[0]
    t = res["tails"]
    hit = t[(t["tmpl"] == k) & (t["lag"] == lag)]
    assert len(hit) == 1
    assert abs(hit["value"][0] - a) <= 4 * res["sigma"][k]


def test_time_randomised_null():
    """Time-randomising the injected segment (Sec. 5) removes the injection's
    coherent peak: before, |rho|/sigma > 8 at the injection (the injection's
    own power raises the Parseval sigma above the noise-only value); after,
    the largest |rho|/sigma over the bank is Gaussian-like (< 6.5)."""
    seg, params = S.small_case()
    bank = O.chirp_bank(params, 4096.0, 4096, 0.05)
    k, lag, a = seg.injections[0]
    before = O.search(seg.y, bank[k:k + 1], 5.0, return_rho=True)
    assert abs(before["rho"][0][lag]) / before["sigma"][0] > 8
    y2 = rng(4).permutation(seg.y)
    after = O.search(y2, bank, 5.0, return_rho=True)
    z = np.max(np.abs(after["rho"]), axis=1) / after["sigma"]
    assert z.max() < 6.5


# --------------------------------------------------------------------------
# The synthetic noise recipe
# --------------------------------------------------------------------------
def test_noise_recipe():
    """Unit variance in expectation and no power outside the band."""
    n = 1 << 14
    ys = np.stack([S.band_limited_noise(n, s) for s in range(20)]).astype(np.float64)
    assert abs(np.mean(ys * ys) - 1.0) < 0.02
    spec = np.abs(np.fft.rfft(ys[0])) ** 2
    f = np.arange(n // 2 + 1) * 4096.0 / n
    outside = (f < 350) | (f > 2000)
    assert spec[outside].sum() < 1e-9 * spec.sum()


# ----------------------------------------------------------------------------
# Per-lag maximum over the bank (Eq. Ak, Eq. Aa, Eq. BA) and Table 3
# ----------------------------------------------------------------------------
def test_max_projection_matches_brute_force():
    """Scalar loops over lags and templates, written from the definition:
    keep the largest rho/sigma among templates with rho > kappa sigma, the
    smaller template on equal values."""
    g = np.random.default_rng(41)
    k, n = 7, 40
    rho = g.standard_normal((k, n)) * 2.0
    rho[3, 5] = rho[1, 5] = 9.0                     # an exact tie: template 1 wins
    sigma = np.ones(k)
    sigma[4] = 0.5                                  # normalisation matters
    kappa = 1.5
    snr, tmpl = O.max_projection(rho, sigma, kappa, k0=100)
    for j in range(n):
        best, arg = 0.0, -1
        for r in range(k):
            if rho[r, j] > kappa * sigma[r]:
                v = rho[r, j] / sigma[r]
                if arg < 0 or v > best:
                    best, arg = v, 100 + r
        assert tmpl[j] == arg and snr[j] == best
    assert tmpl[5] == 101
    # negative correlations are not hits of the projection (signed, Eq. C)
    neg = -np.abs(rho)
    assert np.all(O.max_projection(neg, sigma, kappa)[1] == -1)


def test_max_projection_is_the_per_lag_maximum_of_the_tails():
    """The projection keeps, per lag, the largest positive tail of the
    all-hits search, normalised by its template's sigma."""
    y = S.band_limited_noise(1024, 12)
    bank = S.random_samples_bank(9, 200, 13).astype(np.float64)
    kappa = 2.0
    res = O.search(y, bank, kappa, return_rho=True)
    snr, tmpl = O.max_projection(res["rho"], res["sigma"], kappa)
    t = res["tails"]
    t = t[t["value"] > 0]
    for j in range(1024):
        at = t[t["lag"] == j]
        if len(at) == 0:
            assert tmpl[j] == -1 and snr[j] == 0.0
            continue
        norm = at["value"] / res["sigma"][at["tmpl"]]
        i = int(np.argmax(norm))
        assert tmpl[j] == at["tmpl"][i] and snr[j] == norm[i]


def test_table3_rows_encoding():
    """Table 3: 1-based sample offset, 1000 rho as a 4-byte integer, the
    template's initial frequency in whole Hz; lags without a hit are left out."""
    snr = np.array([0.0, 5.5227, 0.0, 6.0])
    tmpl = np.array([-1, 2, -1, 0])
    f0 = np.array([486.7, 500.0, 623.2])
    rows = O.table3_rows(snr, tmpl, f0)
    assert rows["offset"].tolist() == [2, 4]
    assert rows["rho1000"].tolist() == [5522, 6000]
    assert rows["f0"].tolist() == [623, 486]
    assert rows["rho1000"].dtype == np.int32


# ----------------------------------------------------------------------------
# Time-symmetric chirps (Fig. 2 caption)
# ----------------------------------------------------------------------------
def test_symmetric_chirp_closed_form():
    """Scalar math.sin of the forward chirp at m and at L - 1 - m, summed,
    tapered and normalised; the template reads the same backwards."""
    f0, fd, fs, length = 812.25, 143.5, 4096.0, 4096
    w = O.chirp_template(f0, fd, fs, length, 0.05, symmetric=True)

    def ph(m):
        t = m / fs
        return math.sin(2 * math.pi * (f0 * t + 0.5 * fd * t * t))
    tap = O.taper(length, 0.05)
    raw = [tap[m] * (ph(m) + ph(length - 1 - m)) for m in range(length)]
    norm = math.sqrt(sum(v * v for v in raw))
    for m in [0, 3, 99, 102, 1500, 2047, 2048, 4000, 4095]:
        assert abs(w[m] - raw[m] / norm) < 1e-15
    assert np.allclose(w, w[::-1], rtol=0, atol=1e-15)
    assert abs(np.dot(w, w) - 1.0) < 1e-13


def test_symmetric_chirp_responds_to_both_directions():
    """Against an ascending chirp and its time reversal (a descending chirp)
    the symmetric template gives the same peak correlation at the start of
    the chirp; the plain template sees only the ascending one strongly."""
    fs, length, n = 4096.0, 4096, 16384
    f0, fd = 600.0, 150.0
    up = O.chirp_template(f0, fd, fs, length, 0.05)
    down = up[::-1].copy()
    sym = O.chirp_template(f0, fd, fs, length, 0.05, symmetric=True)
    y_up = np.zeros(n)
    y_up[3000:3000 + length] = up
    y_down = np.zeros(n)
    y_down[3000:3000 + length] = down
    r_up = O.correlate_fft(sym, y_up)[3000]
    r_down = O.correlate_fft(sym, y_down)[3000]
    assert abs(r_up - r_down) < 1e-9 and r_up > 0.6
    plain_down = O.correlate_fft(up, y_down)[3000]
    assert O.correlate_fft(up, y_up)[3000] > 0.999 and abs(plain_down) < 0.1


# ----------------------------------------------------------------------------
# Band threshold (Sec. 5: Eq. tail over a finite band)
# ----------------------------------------------------------------------------
def test_tails_band_definition():
    """Scalar check of kappa_lo sigma < |rho| < kappa_hi sigma, and the band
    as the lower tails minus those at or above the upper bound; both ends
    are excluded."""
    g = np.random.default_rng(5)
    rho = g.standard_normal(500) * 2.0
    sigma = 1.25
    rho[10], rho[11], rho[12] = 4.0 * sigma, -5.0 * sigma, 4.5 * sigma  # on the bounds, inside
    band = O.tails_band(rho, sigma, 4.0, 5.0, 9)
    want = [n for n in range(500) if 4.0 * sigma < abs(rho[n]) < 5.0 * sigma]
    assert band["lag"].tolist() == want
    assert np.all(band["tmpl"] == 9) and np.array_equal(band["value"], rho[want])
    assert 10 not in want and 11 not in want and 12 in want
    lo = O.tails(rho, sigma, 4.0, 9)
    hi = set(np.nonzero(np.abs(rho) >= 5.0 * sigma)[0].tolist())
    assert band["lag"].tolist() == [n for n in lo["lag"].tolist() if n not in hi]


# ----------------------------------------------------------------------------
# Overlap-save lag mask (the circular correlation restricted to unwrapped lags)
# ----------------------------------------------------------------------------
def test_correlate_linear_is_numpy_valid_correlation():
    """Eq. A1 without wrap is numpy's 'valid' cross-correlation, sum_m
    y[n+m] w[m] for n = 0..N-L (a library special case)."""
    g = rng(41)
    y, w = g.standard_normal(300), g.standard_normal(37)
    got = O.correlate_linear(w, y)
    assert len(got) == 300 - 37 + 1
    assert np.allclose(got, np.correlate(y, w, mode="valid"), rtol=0, atol=1e-12)


def test_circular_equals_linear_on_unwrapped_lags_only():
    """The FFT path's circular rho equals the linear correlation at the
    lags n <= N - L, and differs at lags whose window wraps (there the sum
    takes samples from the start of the segment)."""
    g = rng(42)
    n, length = 1024, 100
    y, w = g.standard_normal(n), g.standard_normal(length)
    circ = O.correlate_fft(w, y)
    lin = O.correlate_linear(w, y)
    assert np.allclose(circ[:n - length + 1], lin, rtol=0, atol=1e-10)
    wrapped = circ[n - length + 1:]
    direct = [sum(w[m] * y[(k + m) % n] for m in range(length)) for k in range(n - length + 1, n)]
    assert np.allclose(wrapped, direct, atol=1e-10)
    no_wrap = [sum(w[m] * y[k + m] for m in range(length) if k + m < n)
               for k in range(n - length + 1, n)]
    assert np.max(np.abs(np.asarray(no_wrap) - wrapped)) > 1e-3


def test_tails_linear_is_the_unwrapped_part_of_the_tails():
    """tails_linear keeps exactly the tails at lags n <= N - L, with the
    same sigma; a tail at the last unwrapped lag N - L is kept and one at
    N - L + 1 dropped."""
    g = rng(43)
    n, length = 512, 64
    rho = g.standard_normal(n)
    sigma = 0.5
    rho[n - length] = 3.0
    rho[n - length + 1] = -3.0
    full = O.tails(rho, sigma, 4.0, 3)
    lin = O.tails_linear(rho, sigma, 4.0, length, 3)
    assert lin["lag"].tolist() == [int(x) for x in full["lag"] if x <= n - length]
    assert n - length in lin["lag"].tolist() and n - length + 1 not in lin["lag"].tolist()
    assert n - length + 1 in full["lag"].tolist()


# ----------------------------------------------------------------------------
# Two channels: simultaneous hits and Table 3 (Sec. 5)
# ----------------------------------------------------------------------------
def test_coincidences_worked_example():
    f0 = np.array([400.0, 440.0, 460.0, 1000.0])
    t1 = np.array([-1, 0, 1, 3, -1, 2])
    t2 = np.array([1, 1, -1, 2, -1, 2])
    c = O.coincidences(t1, t2, f0, delta=50.0)
    assert c["hits"] == (4, 4)
    assert c["simultaneous"] == 3              # lags 1, 3, 5
    assert c["within_delta"] == 2              # lag 1 (40 Hz) and lag 5 (0 Hz); lag 3 is 540 Hz
    assert c["lags"].tolist() == [1, 5]
    assert O.coincidences(t1, t2, f0, delta=40.0)["within_delta"] == 1   # strict


def test_table3_two_channel_rows():
    """The three rows Table 3 prints (1000 rho and f0 per channel, zeros for
    no hit: 0/5522/0/1988, 5747/0/486/0, 5516/0/623/0), rebuilt from
    projections with those values at offsets renumbered 1..3."""
    f0 = np.array([486.4, 623.9, 1988.2])
    s1 = np.array([0.0, 5.7471, 5.5169, 0.0])
    t1 = np.array([-1, 0, 1, -1])
    s2 = np.array([5.5229, 0.0, 0.0, 0.0])
    t2 = np.array([2, -1, -1, -1])
    rows = O.table3_rows_two(s1, t1, s2, t2, f0)
    assert rows.tolist() == [(1, 0, 5522, 0, 1988), (2, 5747, 0, 486, 0), (3, 5516, 0, 623, 0)]
