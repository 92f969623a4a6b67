"""Seeded synthetic strain segments, injections and chirp grids.

The paper searches LIGO S6 strain band-passed to 350-2000 Hz at 4096 Hz
(Sec. 2, Sec. 3), where the noise is close to Gaussian.  These generators make
stand-ins with that shape:

* ``band_limited_noise``: complex-Gaussian Fourier bins inside the band, zero
  outside, scaled so that E[y_n^2] = 1, transformed to the time domain in FP64
  and rounded to FP32.  Both the oracle and the CUDA path consume the same
  FP32 array.
* ``chirp_signal``: the injected signal model, a tapered linear chirp
  sin(2 pi (f0 t + fdot t^2 / 2)) of unit L2 norm.  It is written here on its
  own (FP64, scalar-free numpy) and is deliberately not shared with either
  side's template synthesis: recovering an injection therefore checks the
  template code of each side against an independent waveform.
* ``grid_small`` / ``grid_paper``: the (f0, fdot) grids of the 64-template
  parity bank and of the 2^20-template paper-scale bank.

Everything is drawn from numpy's PCG64 with an explicit seed.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

FS = 4096.0          # Hz, the paper's down-sampled rate (Sec. 3)
BAND = (350.0, 2000.0)  # Hz, the analysis band (Sec. 2)


def band_bins(n: int, fs: float = FS, band=BAND) -> np.ndarray:
    """Indices j of the rfft bins with band[0] <= j*fs/n <= band[1]."""
    j = np.arange(n // 2 + 1)
    f = j * fs / n
    return j[(f >= band[0]) & (f <= band[1])]


def noise_scale(n: int, fs: float = FS, band=BAND) -> float:
    """Per-bin amplitude s with E|Y_j|^2 = s^2 that makes E[y_n^2] = 1."""
    k_band = len(band_bins(n, fs, band))
    return n / math.sqrt(2.0 * k_band)


def expected_filter_rms(n: int, fs: float = FS, band=BAND) -> float:
    """Expected RMS of the filter output for a unit-norm template whose energy
    lies inside the band, under the noise model of ``band_limited_noise``.

    This is a property of the noise recipe (s / sqrt(n)); it sets injection
    amplitudes ("20 sigma", "SNR 8-30") without using either side's
    Parseval prediction.
    """
    return noise_scale(n, fs, band) / math.sqrt(n)


def band_limited_noise(n: int, seed: int, fs: float = FS, band=BAND) -> np.ndarray:
    """Unit-variance Gaussian noise limited to ``band``; FP32, length n."""
    rng = np.random.Generator(np.random.PCG64(seed))
    spec = np.zeros(n // 2 + 1, dtype=np.complex128)
    jb = band_bins(n, fs, band)
    s = noise_scale(n, fs, band)
    a = rng.normal(0.0, math.sqrt(0.5), size=len(jb))
    b = rng.normal(0.0, math.sqrt(0.5), size=len(jb))
    spec[jb] = s * (a + 1j * b)
    y = np.fft.irfft(spec, n=n)
    return y.astype(np.float32)


def tukey_taper(length: int, frac: float) -> np.ndarray:
    """Cosine taper with total tapered fraction ``frac`` (half at each end)."""
    m = np.arange(length, dtype=np.float64)
    t = np.ones(length)
    if frac <= 0.0 or length < 2:
        return t
    width = int(math.floor(frac * (length - 1) / 2.0))
    ramp = 0.5 * (1.0 - np.cos(2.0 * np.pi * m[: width + 1] / (frac * (length - 1))))
    t[: width + 1] = ramp
    t[length - width - 1:] = ramp[::-1]
    return t


def chirp_signal(f0: float, fdot: float, length: int, fs: float = FS,
                 taper_frac: float = 0.05) -> np.ndarray:
    """Injected signal: tapered linear chirp of unit L2 norm, FP64."""
    t = np.arange(length, dtype=np.float64) / fs
    phase_cycles = f0 * t + 0.5 * fdot * t * t
    s = tukey_taper(length, taper_frac) * np.sin(2.0 * np.pi * phase_cycles)
    return s / np.sqrt(np.dot(s, s))


def inject(y: np.ndarray, signal: np.ndarray, lag: int, amplitude: float) -> np.ndarray:
    """Return y with amplitude*signal added circularly starting at ``lag``."""
    out = y.astype(np.float64)
    n = len(out)
    idx = (lag + np.arange(len(signal))) % n
    np.add.at(out, idx, amplitude * signal)
    return out.astype(np.float32)


def grid_small():
    """64 chirps: f0 in linspace(400,1800,8) x fdot in linspace(-100,100,8).

    Template index k = i_fdot * 8 + i_f0.
    """
    f0 = np.linspace(400.0, 1800.0, 8)
    fd = np.linspace(-100.0, 100.0, 8)
    F0, FD = np.meshgrid(f0, fd)  # rows: fdot, cols: f0
    return np.stack([F0.ravel(), FD.ravel()], axis=1)


def grid_paper(n_fdot: int = 1024, n_f0: int = 1024, tau: float = 1.0,
               band=BAND, fdot_max: float = 200.0):
    """n_fdot x n_f0 chirps whose frequency stays inside ``band`` over tau.

    fdot_i = linspace(-fdot_max, fdot_max, n_fdot); for each fdot the f0 grid
    is linspace(band0 + max(0, -fdot tau), band1 - max(0, fdot tau), n_f0).
    Template index k = i_fdot * n_f0 + i_f0.
    """
    fd = np.linspace(-fdot_max, fdot_max, n_fdot)
    out = np.empty((n_fdot * n_f0, 2))
    for i, d in enumerate(fd):
        lo = band[0] + max(0.0, -d * tau)
        hi = band[1] - max(0.0, d * tau)
        out[i * n_f0:(i + 1) * n_f0, 0] = np.linspace(lo, hi, n_f0)
        out[i * n_f0:(i + 1) * n_f0, 1] = d
    return out


@dataclasses.dataclass
class Segment:
    y: np.ndarray            # FP32 strain, length n
    n: int
    injections: list         # [(k, lag, amplitude)]
    sigma_expected: float    # expected filter RMS for unit-norm in-band templates


def make_segment(n: int, params: np.ndarray, n_inject: int, seed: int,
                 tau: float = 1.0, taper_frac: float = 0.05, fs: float = FS,
                 snr_range=(8.0, 30.0), fixed=None) -> Segment:
    """Band-limited noise plus chirp injections drawn from ``params``.

    ``fixed`` = [(k, lag, snr)] places injections explicitly; otherwise
    ``n_inject`` injections take k uniform over the bank, lag uniform in
    [0, n - L] and SNR uniform in ``snr_range``.  Amplitude = SNR times the
    expected filter RMS of the noise recipe.
    """
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    y = band_limited_noise(n, seed, fs)
    length = int(round(tau * fs))
    sig_e = expected_filter_rms(n, fs)
    if fixed is None:
        ks = rng.integers(0, len(params), size=n_inject)
        lags = rng.integers(0, max(1, n - length + 1), size=n_inject)
        snrs = rng.uniform(snr_range[0], snr_range[1], size=n_inject)
        fixed = list(zip(ks.tolist(), lags.tolist(), snrs.tolist()))
    inj = []
    for k, lag, snr in fixed:
        f0, fd = params[int(k)]
        a = float(snr) * sig_e
        y = inject(y, chirp_signal(f0, fd, length, fs, taper_frac), int(lag), a)
        inj.append((int(k), int(lag), a))
    return Segment(y=y, n=n, injections=inj, sigma_expected=sig_e)


def small_case(seed: int = 1234) -> tuple[Segment, np.ndarray]:
    """N = 2^14 parity case: 64-chirp grid, one injection at lag 5000, 20 sigma."""
    params = grid_small()
    seg = make_segment(1 << 14, params, 1, seed, fixed=[(27, 5000, 20.0)])
    return seg, params


def paper_case(seed: int = 2017, n_fdot: int = 1024, n_f0: int = 1024,
               n_inject: int = 32) -> tuple[Segment, np.ndarray]:
    """N = 2^16 paper-scale case: 2^20 in-band chirps, 32 injections SNR 8-30."""
    params = grid_paper(n_fdot, n_f0)
    seg = make_segment(1 << 16, params, n_inject, seed)
    return seg, params


def random_samples_bank(count: int, length: int, seed: int) -> np.ndarray:
    """Arbitrary FP32 templates (unit-variance Gaussian samples) for tests that
    feed identical template samples to both sides."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((count, length)).astype(np.float32)


@dataclasses.dataclass
class BatchEntry:
    seg: Segment
    tau: float
    k0: int          # sub-bank: rows [k0, k1) of the bank for this tau
    k1: int


def batch_case(seed: int = 4242, n_segments: int = 64, n_inject: int = 8,
               sizes=(1 << 14, 1 << 15, 1 << 16, 1 << 17),
               sub_bank=(1 << 12, 1 << 16), taus=(0.5, 1.0), n_fdot: int = 1024,
               n_f0: int = 1024):
    """Batching-form workload: segments of lengths drawn uniformly from
    ``sizes``, each with its own sub-bank (a contiguous row range of the
    in-band grid for its tau, size log-uniform in ``sub_bank``) and
    ``n_inject`` injections drawn from that sub-bank.

    Returns (entries, {tau: params}).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    grids = {tau: grid_paper(n_fdot, n_f0, tau=tau) for tau in taus}
    entries = []
    for s in range(n_segments):
        n = int(rng.choice(sizes))
        tau = float(rng.choice(taus))
        size = int(round(2.0 ** rng.uniform(math.log2(sub_bank[0]), math.log2(sub_bank[1]))))
        total = len(grids[tau])
        size = min(size, total)
        k0 = int(rng.integers(0, total - size + 1))
        sub = grids[tau][k0:k0 + size]
        seg = make_segment(n, sub, n_inject, seed * 1000 + s, tau=tau)
        seg.injections = [(k + k0, lag, a) for k, lag, a in seg.injections]
        entries.append(BatchEntry(seg=seg, tau=tau, k0=k0, k1=k0 + size))
    return entries, grids


@dataclasses.dataclass
class Arrival:
    t: float          # arrival time, seconds from the start of the stream
    channel: int
    n: int            # samples
    y: np.ndarray     # FP32 strain


def serving_stream(n_requests: int, seed: int = 99, channels: int = 2,
                   durations=(8.0, 16.0, 32.0), speed: float = 2.0, fs: float = FS,
                   n_inject: int = 0, params=None):
    """Requests of the serving form: each channel emits band-limited noise
    segments of durations drawn uniformly from ``durations`` with Poisson
    arrivals whose mean rate carries ``speed`` data-seconds per wall-second
    per channel (speed = 2: twice real time).  Returns the first
    ``n_requests`` arrivals over all channels in time order.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    rate = speed / float(np.mean(durations))  # requests per second per channel
    per = []
    for c in range(channels):
        t = 0.0
        for i in range(n_requests):
            t += float(rng.exponential(1.0 / rate))
            dur = float(rng.choice(durations))
            per.append((t, c, int(round(dur * fs)), seed * 100000 + c * 10000 + i))
    per.sort()
    out = []
    for t, c, n, s in per[:n_requests]:
        if n_inject and params is not None:
            y = make_segment(n, params, n_inject, s).y
        else:
            y = band_limited_noise(n, s, fs)
        out.append(Arrival(t=t, channel=c, n=n, y=y))
    return out
