"""Oracle runs for the scale-parity tests, executed in spawned worker processes.

Each job takes the seeded input (rebuilt from its seed in the worker), the
block states the GPU had in force (checked in lock-step by the test before
submission) and the GPU's final field, re-runs the steps in the FP64 oracle
with those states and returns the rel-L2 error.  No value here comes from the
CUDA path except the states (already checked against the oracle's own
classifier) and the field under test.
"""
import os

import numpy as np


def init_worker(threads):
    """Process-pool initializer: the oracle's OpenMP thread count for this worker."""
    os.environ["OMP_NUM_THREADS"] = str(int(threads))


def fp32_floor(E0, steps, beta2=-21.7, gamma=1.3, h=0.1):
    """rel-L2 after `steps` dense split steps in numpy single precision (an
    independent FP32 FFT) against the same in double precision: the error FP32
    arithmetic itself leaves on this signal."""
    import oracle as O
    n = E0.size
    H = O.nls_half_factor(O.nls_omega(n, 1.0), beta2, h)

    def run(E, cdt):
        E = E.astype(cdt)
        hh = H.astype(cdt)
        for _ in range(steps):
            E = np.fft.ifft(np.fft.fft(E) * hh).astype(cdt)
            p = E.real ** 2 + E.imag ** 2
            E = (E * np.exp(1j * gamma * p * h)).astype(cdt)
            E = np.fft.ifft(np.fft.fft(E) * hh).astype(cdt)
        return E
    E0 = E0.astype(np.complex64)
    return O.rel_l2(run(E0, np.complex64), run(E0, np.complex128))


def nls_job(n, seed, steps, reassess, masks, gpu_fields, with_floor):
    """One NLS signal, started from its complex64-rounded samples: the oracle
    with the GPU's states; returns ({name: rel-L2 of gpu_fields[name]}, FP32
    floor or None)."""
    import oracle as O
    import workloads as W
    E0 = W.nls_signal(n, seed=seed).astype(np.complex64).astype(np.complex128)
    cfg = O.NLSConfig(n, n // 64, threshold=1e-6, reassess=reassess)
    ref, _ = O.run_nls(E0, cfg, steps, on_assess=lambda s, E, st, tau: masks.get(s))
    errs = {k: O.rel_l2(f, ref) for k, f in gpu_fields.items()}
    floor = fp32_floor(W.nls_signal(n, seed=seed), steps) if with_floor else None
    return errs, floor


def ch_job(dims, block, mean, seed, steps, reassess, masks, gpu_field, threshold=1e-6):
    """One CH run (complex64 input rounding) with the GPU's states; returns rel-L2."""
    import oracle as O
    import workloads as W
    c0 = W.ch_initial_condition(dims, mean=mean, seed=seed).astype(np.float32).astype(np.float64)
    cfg = O.CHConfig(dims, block, threshold=threshold, reassess=reassess)
    ref_hat, _ = O.run_ch(c0, cfg, steps, on_assess=lambda s, ch, st, tau: masks.get(s))
    return O.rel_l2(gpu_field, O.ch_real_field(ref_hat))


def ch_fp32_floor(dims, mean, seed, steps, dt=0.01, kappa=1.0, workers=4):
    """rel-L2 after `steps` dense CH steps computed in single precision (scipy's
    FFT keeps complex64 inputs in single precision) against the same steps in
    double precision, from the same complex64-rounded start: the error FP32
    arithmetic itself leaves on this run (coarsening amplifies rounding)."""
    import scipy.fft as sf
    import workloads as W
    c0 = W.ch_initial_condition(dims, mean=mean, seed=seed).astype(np.float32)
    k2 = 0.0
    for a, n in enumerate(dims):
        j = np.arange(n)
        j = np.where(j <= n // 2, j, j - n)
        shape = [1] * len(dims)
        shape[a] = n
        k2 = k2 + ((2.0 * np.pi * j / n) ** 2).reshape(shape)

    def run(cdt, rdt):
        kk = np.asarray(k2, dtype=rdt)
        den = np.asarray(1.0 + dt * kappa * k2 * k2, dtype=rdt)
        ch = sf.fftn(c0.astype(rdt), workers=workers).astype(cdt)
        for _ in range(steps):
            c = sf.ifftn(ch, workers=workers).real.astype(rdt)
            g = c * c * c - c
            ch = ((ch - rdt(dt) * kk * sf.fftn(g, workers=workers)) / den).astype(cdt)
        return sf.ifftn(ch.astype(np.complex128)).real

    a = run(np.complex64, np.float32)
    b = run(np.complex128, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
