"""Plain FP64 CPU oracle of the matched-filter search (van Putten, arXiv:1708.01609).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product library.

What it computes, in the paper's order (Sec. 3 and Sec. 3.2):

1. Templates (Sec. 3, Eq. s; chirp form of the synthetic bank):
   w[m] = T(m) sin(2 pi (f0 t_m + fdot t_m^2 / 2)), t_m = m / fs, m < L, with
   T a cosine (Tukey) taper, scaled to unit L2 norm, zero-padded to N.
2. Correlation (Eq. A1 discretised, circular):
   rho[n] = sum_m w[m] y[(n + m) mod N], n = 0..N-1.
   ``correlate_direct`` writes this sum out; ``correlate_fft`` evaluates it by
   the three steps of Eq. 3S with this module's own radix-2 FFT:
   {W, D} = FFT{w, y}; P = conj(W) D; rho = FFT^-1{P}.
3. sigma (the definition below Eq. 3S, and Eq. PT): RMS of rho about zero,
   predicted from the spectrum by Parseval's theorem.
4. Tails (Eq. tail, applied to |rho| as the paper states): every
   (k, n, rho_k[n]) with |rho_k[n]| > kappa sigma_k ("all hits", Sec. 3.3).

Readings of the paper taken here (the paper is garbled or silent):

* Eq. A1 integrates over "dt"; it must be ds.  The lag convention y(t+s)
  places a template injected at y[l + m] at lag n = l.
* Eq. A3 normalises c_k with 1/N, which contradicts the sqrt(2)/N prefactor
  of Eq. PT.  Eq. PT holds for UNnormalised coefficients P_j = sum_n rho_n
  e^{-2 pi i j n / N}; then sigma^2 = (1/N^2) sum_{j<N} |P_j|^2
  = (1/N^2)(|P_0|^2 + |P_{N/2}|^2 + 2 sum_{j=1}^{N/2-1} |P_j|^2).  The printed
  form drops DC and Nyquist; ``sigma_parseval_paper_form`` keeps that form and
  equals ``sigma_parseval`` when those two bins vanish.
* The forward transform uses e^{-i k t} (Eq. A2), the inverse e^{+...}/N.
* The threshold is strict: |rho| > kappa sigma (Eq. tail writes ">").
* The correlation is circular over all N lags (the template is zero-padded to
  N, Sec. 3.2 step ii, and transformed with an N-point FFT).  The optional
  overlap-save form keeps the tails at the lags n <= N - L only, where the
  circular sum equals the linear one (``correlate_linear``, ``tails_linear``);
  sigma is unchanged.
"""
from __future__ import annotations

import math

import numpy as np

TAIL_DTYPE = np.dtype([("tmpl", np.uint32), ("lag", np.uint32), ("value", np.float64)])


# ----------------------------------------------------------------------------
# FFT (Eq. 3S, with the sign convention of Eq. A2)
# ----------------------------------------------------------------------------
def _bit_reverse(n: int) -> np.ndarray:
    bits = n.bit_length() - 1
    idx = np.arange(n)
    rev = np.zeros(n, dtype=np.int64)
    for b in range(bits):
        rev |= ((idx >> b) & 1) << (bits - 1 - b)
    return rev


def fft(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    """Unnormalised radix-2 Cooley-Tukey FFT over the last axis, FP64.

    Forward: X_j = sum_n x_n exp(-2 pi i j n / N)   (sign of Eq. A2)
    Inverse: x_n = sum_j X_j exp(+2 pi i j n / N)   (no 1/N here)

    Textbook decimation in time: bit-reversal permutation, then log2(N)
    stages of size-2 butterflies, each stage vectorised over the batch.
    """
    a = np.asarray(x, dtype=np.complex128)
    n = a.shape[-1]
    if n & (n - 1) or n == 0:
        raise ValueError("FFT length must be a power of two")
    lead = a.shape[:-1]
    a = a[..., _bit_reverse(n)].copy()
    sign = 1.0 if inverse else -1.0
    size = 2
    while size <= n:
        half = size // 2
        tw = np.exp(sign * 2j * np.pi * np.arange(half) / size)
        blocks = a.reshape(*lead, n // size, size)
        even = blocks[..., :half]
        odd = blocks[..., half:] * tw
        a = np.concatenate([even + odd, even - odd], axis=-1).reshape(*lead, n)
        size *= 2
    return a


# ----------------------------------------------------------------------------
# Templates (Sec. 3, Eq. s: chirps over a range of f and fdot)
# ----------------------------------------------------------------------------
def taper(length: int, frac: float) -> np.ndarray:
    """Cosine taper: 0.5(1 - cos(2 pi m / (frac (L-1)))) on the first
    floor(frac (L-1) / 2) + 1 samples, mirrored at the end, 1 in between."""
    t = np.ones(length, dtype=np.float64)
    if frac <= 0.0 or length < 2:
        return t
    width = int(math.floor(frac * (length - 1) / 2.0))
    for m in range(width + 1):
        v = 0.5 * (1.0 - math.cos(2.0 * math.pi * m / (frac * (length - 1))))
        t[m] = v
        t[length - 1 - m] = v
    return t


def chirp_template(f0: float, fdot: float, fs: float, length: int,
                   taper_frac: float, symmetric: bool = False) -> np.ndarray:
    """Unit-norm tapered linear chirp, FP64, length ``length``.

    symmetric: the time-symmetric chirp of the paper's banks (Fig. 2
    caption: the superposition of the chirp forward and backward in time),
    read on the sample grid as sin(phi(m)) + sin(phi(L - 1 - m)) under the
    (symmetric) taper.  A template whose two halves cancel is all zeros."""
    t = np.arange(length, dtype=np.float64) / fs
    core = np.sin(2.0 * np.pi * (f0 * t + 0.5 * fdot * t * t))
    if symmetric:
        core = core + core[::-1]
    w = taper(length, taper_frac) * core
    norm = math.sqrt(float(np.dot(w, w)))
    return w / norm if norm > 0.0 else w


def chirp_bank(params: np.ndarray, fs: float, length: int, taper_frac: float,
               symmetric: bool = False) -> np.ndarray:
    """Templates for rows (f0, fdot) of ``params``; shape (K, length), FP64."""
    return np.stack([chirp_template(f0, fd, fs, length, taper_frac, symmetric)
                     for f0, fd in params])


# ----------------------------------------------------------------------------
# Correlation (Eq. A1, Eq. 3S)
# ----------------------------------------------------------------------------
def correlate_direct(w: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Eq. A1 as a finite circular sum: rho[n] = sum_m w[m] y[(n+m) mod N]."""
    w = np.asarray(w, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = len(y)
    rho = np.zeros(n)
    for m in range(len(w)):
        rho += w[m] * np.roll(y, -m)   # np.roll(y, -m)[n] = y[(n+m) mod N]
    return rho


def zero_pad(w: np.ndarray, n: int) -> np.ndarray:
    w = np.asarray(w, dtype=np.float64)
    if w.shape[-1] > n:
        raise ValueError("template longer than segment")
    out = np.zeros(w.shape[:-1] + (n,))
    out[..., : w.shape[-1]] = w
    return out


def correlation_spectrum(w: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Eq. 3S steps 1-2: P = conj(FFT w) * FFT y (w zero-padded to N)."""
    n = len(y)
    big_w = fft(zero_pad(w, n))
    big_d = fft(np.asarray(y, dtype=np.float64))
    return np.conj(big_w) * big_d


def correlate_fft(w: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Eq. 3S: rho = FFT^-1{conj(W) D}; returns the real part (the imaginary
    part is rounding noise because rho is real)."""
    p = correlation_spectrum(w, y)
    n = p.shape[-1]
    return (fft(p, inverse=True) / n).real


# ----------------------------------------------------------------------------
# sigma (definition below Eq. 3S; Eq. PT)
# ----------------------------------------------------------------------------
def sigma_rms(rho: np.ndarray) -> np.ndarray:
    """sigma = (1/sqrt N) sqrt(sum_n rho_n^2): the RMS of rho about zero."""
    rho = np.asarray(rho, dtype=np.float64)
    return np.sqrt(np.sum(rho * rho, axis=-1) / rho.shape[-1])


def sigma_parseval(p: np.ndarray) -> np.ndarray:
    """Eq. PT with unnormalised coefficients of rho (reading in module doc):
    sigma = (1/N) sqrt(sum_{j=0}^{N/2} c_j |P_j|^2), c_0 = c_{N/2} = 1, else 2."""
    p = np.asarray(p)
    n = p.shape[-1]
    h = n // 2
    mag2 = (p[..., : h + 1] * np.conj(p[..., : h + 1])).real
    c = np.full(h + 1, 2.0)
    c[0] = 1.0
    c[h] = 1.0
    return np.sqrt(np.sum(c * mag2, axis=-1)) / n


def sigma_parseval_paper_form(p: np.ndarray) -> np.ndarray:
    """Eq. PT as printed: (sqrt 2 / N) sqrt(sum_{j=1}^{N/2-1} |P_j|^2)."""
    p = np.asarray(p)
    n = p.shape[-1]
    h = n // 2
    mag2 = (p[..., 1:h] * np.conj(p[..., 1:h])).real
    return math.sqrt(2.0) * np.sqrt(np.sum(mag2, axis=-1)) / n


# ----------------------------------------------------------------------------
# Tails (Eq. tail, all hits)
# ----------------------------------------------------------------------------
def tails(rho: np.ndarray, sigma: float, kappa: float, k: int) -> np.ndarray:
    """All (k, n, rho[n]) with |rho[n]| > kappa * sigma, ordered by n."""
    rho = np.asarray(rho, dtype=np.float64)
    lags = np.nonzero(np.abs(rho) > kappa * sigma)[0]
    out = np.empty(len(lags), dtype=TAIL_DTYPE)
    out["tmpl"] = k
    out["lag"] = lags
    out["value"] = rho[lags]
    return out


def tails_band(rho: np.ndarray, sigma: float, kappa_lo: float, kappa_hi: float,
               k: int) -> np.ndarray:
    """Eq. tail generalised to a finite band (Sec. 5, deep searches): every
    (k, n, rho[n]) with kappa_lo sigma < |rho[n]| < kappa_hi sigma, by n."""
    rho = np.asarray(rho, dtype=np.float64)
    a = np.abs(rho)
    lags = np.nonzero((a > kappa_lo * sigma) & (a < kappa_hi * sigma))[0]
    out = np.empty(len(lags), dtype=TAIL_DTYPE)
    out["tmpl"] = k
    out["lag"] = lags
    out["value"] = rho[lags]
    return out


def correlate_linear(w: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Eq. A1 over the segment alone, without wrapping: rho[n] = sum_m w[m]
    y[n + m] for the lags n = 0..N-L whose window y[n .. n+L-1] lies inside
    the segment (the lags an overlap-save search keeps)."""
    w = np.asarray(w, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n_valid = len(y) - len(w) + 1
    out = np.zeros(max(n_valid, 0))
    for m in range(len(w)):
        out += w[m] * y[m:m + n_valid]
    return out


def tails_linear(rho: np.ndarray, sigma: float, kappa: float, length: int,
                 k: int) -> np.ndarray:
    """Eq. tail restricted to the lags n <= N - L of a length-L template
    (overlap-save: only lags whose window does not wrap); sigma stays the
    Parseval value over all N lags."""
    rho = np.asarray(rho, dtype=np.float64)
    keep = tails(rho, sigma, kappa, k)
    return keep[keep["lag"] <= len(rho) - length]


def search(y: np.ndarray, templates: np.ndarray, kappa: float, k0: int = 0,
           batch: int = 32, return_rho: bool = False) -> dict:
    """Correlate segment ``y`` with every template row and keep the tails.

    Returns {"tails": TAIL_DTYPE array sorted by (tmpl, lag), "sigma": (K,),
    "rho": (K, N) if requested}.  Template index = k0 + row.
    """
    y = np.asarray(y, dtype=np.float64)
    n = len(y)
    templates = np.atleast_2d(np.asarray(templates, dtype=np.float64))
    big_d = fft(y)
    sig = np.empty(len(templates))
    recs = []
    rhos = np.empty((len(templates), n)) if return_rho else None
    for s in range(0, len(templates), batch):
        w = templates[s:s + batch]
        p = np.conj(fft(zero_pad(w, n))) * big_d
        rho = (fft(p, inverse=True) / n).real
        sg = sigma_parseval(p)
        sig[s:s + len(w)] = sg
        for r in range(len(w)):
            recs.append(tails(rho[r], sg[r], kappa, k0 + s + r))
        if return_rho:
            rhos[s:s + len(w)] = rho
    t = np.concatenate(recs) if recs else np.empty(0, dtype=TAIL_DTYPE)
    t = np.sort(t, order=["tmpl", "lag"])
    out = {"tails": t, "sigma": sig}
    if return_rho:
        out["rho"] = rhos
    return out


# ----------------------------------------------------------------------------
# Per-lag maximum over the bank (Eq. Ak, Eq. Aa, Eq. BA; Table 3)
# ----------------------------------------------------------------------------
def max_projection(rho: np.ndarray, sigma: np.ndarray, kappa: float, k0: int = 0):
    """The per-lag projection of a bank's correlations onto one array of size
    N (Eq. Ak over the templates of a bank, gathered as in Eq. Aa and Eq. BA
    with the maximal value kept per sample): for every lag n, among the
    templates k whose rho_k[n] > kappa sigma_k, the largest normalised value
    rho_k[n] / sigma_k and its template (reading: the signed value, as in
    Eq. C; the strict threshold of Eq. tail; equal values go to the smaller
    template index).  Returns (snr, tmpl): snr 0 and tmpl -1 where no
    template passes.  rho: (K, N); sigma: (K,); template index = k0 + row.
    """
    rho = np.asarray(rho, dtype=np.float64)
    sigma = np.asarray(sigma, dtype=np.float64)
    n = rho.shape[1]
    snr = np.zeros(n)
    tmpl = np.full(n, -1, dtype=np.int64)
    for r in range(rho.shape[0]):
        hit = rho[r] > kappa * sigma[r]
        val = rho[r] / sigma[r]
        better = hit & (val > snr)
        better |= hit & (tmpl < 0)
        snr[better] = val[better]
        tmpl[better] = k0 + r
    return snr, tmpl


def table3_rows(snr: np.ndarray, tmpl: np.ndarray, f0: np.ndarray) -> np.ndarray:
    """Table 3's encoding of a projection: one row per lag with a hit, the
    sample offset (1-based, as the table counts), 1000 x snr as an integer
    and the hit template's initial frequency f0 [Hz] as an integer.  Both
    integers round the exact value toward zero: the product is taken in
    FP64, which is exact for FP32 inputs."""
    lags = np.nonzero(tmpl >= 0)[0]
    rows = np.empty(len(lags), dtype=[("offset", np.int64), ("rho1000", np.int32),
                                       ("f0", np.int32)])
    rows["offset"] = lags + 1
    rows["rho1000"] = np.floor(1000.0 * np.asarray(snr, dtype=np.float64)[lags]).astype(np.int32)
    rows["f0"] = np.floor(np.asarray(f0)[tmpl[lags]]).astype(np.int32)
    return rows


def coincidences(tmpl1: np.ndarray, tmpl2: np.ndarray, f0: np.ndarray,
                 delta: float = 50.0) -> dict:
    """Simultaneous hits of two channels (Sec. 5: H1 and L1 at the same
    sample offset), from their per-lag projections (tmpl -1 = no hit): the
    counts of each channel, of lags where both hit, and of those whose
    templates' initial frequencies differ by less than delta [Hz]."""
    n1 = n2 = both = near = 0
    lags = []
    for n in range(len(tmpl1)):
        a, b = int(tmpl1[n]), int(tmpl2[n])
        n1 += a >= 0
        n2 += b >= 0
        if a >= 0 and b >= 0:
            both += 1
            if abs(float(f0[a]) - float(f0[b])) < delta:
                near += 1
                lags.append(n)
    return {"hits": (n1, n2), "simultaneous": both, "within_delta": near,
            "lags": np.array(lags, dtype=np.int64)}


def table3_rows_two(snr1, tmpl1, snr2, tmpl2, f0) -> np.ndarray:
    """Table 3 with both channels: one row per lag where either hits, with
    1000 rho and f0 of each channel and zeros for a channel without a hit."""
    rows = []
    for n in range(len(tmpl1)):
        a, b = int(tmpl1[n]), int(tmpl2[n])
        if a < 0 and b < 0:
            continue
        rows.append((n + 1,
                     math.floor(1000.0 * float(snr1[n])) if a >= 0 else 0,
                     math.floor(1000.0 * float(snr2[n])) if b >= 0 else 0,
                     math.floor(float(f0[a])) if a >= 0 else 0,
                     math.floor(float(f0[b])) if b >= 0 else 0))
    return np.array(rows, dtype=[("offset", np.int64), ("rho1000_1", np.int32),
                                 ("rho1000_2", np.int32), ("f0_1", np.int32),
                                 ("f0_2", np.int32)])
