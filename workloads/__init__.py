"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds input synthesis only (initial fields, signal construction,
ensemble sizes).  It contains none of the solver's or of sp-DBA's arithmetic,
and it imports neither the oracle nor the CUDA path, so both sides can start
from bit-identical data.

Random numbers come from numpy's PCG64 generator; uniforms are drawn with
Generator.random(), which maps the top 53 bits of each 64-bit output to
[0, 1).  Run r of a workload uses seed 1234 + r.
"""
import math

import numpy as np

BASE_SEED = 1234


def _rng(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


def ch_initial_condition(dims, mean=0.0, amplitude=0.05, seed=BASE_SEED):
    """c0 = mean + U[-amplitude, amplitude] on the given grid (FP64, row-major)."""
    u = _rng(seed).random(tuple(int(d) for d in dims))
    return float(mean) + float(amplitude) * (2.0 * u - 1.0)


def ensemble_members(nruns=64, sides=(128, 192, 256, 384, 512), mean_range=0.2, seed=BASE_SEED):
    """Uneven 2-D ensemble: per run a side drawn uniformly from `sides` and a mean
    uniform in [-mean_range, mean_range]; returns a list of (side, mean, run_seed)."""
    rng = _rng(seed)
    side_idx = rng.integers(0, len(sides), size=nruns)
    means = mean_range * (2.0 * rng.random(nruns) - 1.0)
    return [(int(sides[i]), float(m), seed + 1 + r) for r, (i, m) in enumerate(zip(side_idx, means))]


def nls_lengths(count=512, emin=12, emax=18, seed=BASE_SEED):
    """Signal lengths 2^e with e uniform on the integers emin..emax."""
    e = _rng(seed).integers(emin, emax + 1, size=count)
    return [1 << int(x) for x in e]


def nls_signal(n, seed=BASE_SEED, channels=8, slots=32, peak_power_w=0.01):
    """One transmitted field of n complex samples: the sum of `channels` random-QPSK
    channels, each confined to one of `slots` equal frequency slots (distinct,
    seeded), with a Gaussian spectral shape, scaled so that each channel's peak
    power max|E_c(t)|^2 equals peak_power_w.  Bins outside the occupied slots are
    exactly zero.  Returns complex128.
    """
    if n % slots != 0:
        raise ValueError("n must be a multiple of the slot count")
    rng = _rng(seed)
    W = n // slots
    chosen = rng.choice(slots, size=channels, replace=False)
    E = np.zeros(n, dtype=np.complex128)
    f = np.arange(W) - (W - 1) / 2.0
    shape = np.exp(-(f * f) / (2.0 * (W / 6.0) ** 2))
    for slot in chosen:
        bits = rng.integers(0, 2, size=(W, 2))
        sym = ((2 * bits[:, 0] - 1) + 1j * (2 * bits[:, 1] - 1)) / math.sqrt(2.0)
        spec_local = np.fft.fftshift(np.fft.fft(sym)) * shape
        spec = np.zeros(n, dtype=np.complex128)
        spec[slot * W:(slot + 1) * W] = spec_local
        e_c = np.fft.ifft(spec)
        peak = np.max(np.abs(e_c) ** 2)
        E += e_c * math.sqrt(peak_power_w / peak)
    return E


def nls_cw(n, bin_index, amplitude):
    """Continuous wave A exp(+i w0 t) sitting exactly on FFT bin `bin_index`."""
    t = np.arange(n)
    return amplitude * np.exp(2j * math.pi * bin_index * t / n)


def gaussian_pulse(n, width, amplitude=1.0, center=None):
    """A exp(-(t - t0)^2 / (2 width^2)) sampled at t = 0..n-1 (unit sample spacing)."""
    t = np.arange(n, dtype=np.float64)
    t0 = n / 2.0 if center is None else center
    return amplitude * np.exp(-((t - t0) ** 2) / (2.0 * width * width)).astype(np.complex128)


def rcd_initial_condition(dims, M, base, rel_amplitude=0.1, seed=BASE_SEED):
    """M component fields near a homogeneous state: base * (1 + rel_amplitude *
    U[-1, 1]) independently per component and grid point (FP64, (M, *dims))."""
    u = _rng(seed).random((int(M),) + tuple(int(d) for d in dims))
    return float(base) * (1.0 + float(rel_amplitude) * (2.0 * u - 1.0))


def rcd_lv_homogeneous(M, r=1.0, a=1.0, alpha=1.0, beta=0.3):
    """Equal-concentration fixed point of the Lotka-Volterra reaction with
    interactions beta + alpha to the two neighbouring components (one for M = 2)
    and beta to the others: u* = r / (a + sum_{j != i} alpha_ij).  The base of the
    RCD initial condition."""
    if M <= 1:
        off = 0.0
    elif M == 2:
        off = beta + alpha
    else:
        off = 2.0 * (beta + alpha) + (M - 3) * beta
    return float(r) / (float(a) + off)
