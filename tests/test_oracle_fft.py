"""Pins for the oracle's own FFT: brute-force DFT, a library FFT, Parseval, round trip."""
import math

import numpy as np
import pytest

import oracle as O


def brute_dft_1d(x, sign):
    n = x.shape[-1]
    j = np.arange(n)
    M = np.exp(sign * 2j * math.pi * np.outer(j, j) / n)
    return x @ M.T


def brute_dftn(x, sign=-1):
    y = np.asarray(x, dtype=np.complex128)
    for axis in range(y.ndim):
        y = np.moveaxis(brute_dft_1d(np.moveaxis(y, axis, -1), sign), -1, axis)
    return y


def rand_c(shape, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal(shape) + 1j * r.standard_normal(shape)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 8, 9, 10, 12, 16, 18, 24, 27, 32, 48, 64, 96, 192])
def test_fft_1d_vs_brute(n):
    x = rand_c((n,), n)
    ref = brute_dftn(x)
    got = O.fftn(x)
    assert np.max(np.abs(got - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("shape", [(6, 8), (12, 9), (4, 6, 8), (3, 4, 5), (16, 16), (8, 24, 2)])
def test_fft_nd_vs_brute(shape):
    x = rand_c(shape, sum(shape))
    ref = brute_dftn(x)
    assert np.max(np.abs(O.fftn(x) - ref)) <= 1e-12 * np.max(np.abs(ref))
    refi = brute_dftn(x, +1) / x.size
    assert np.max(np.abs(O.ifftn(x) - refi)) <= 1e-12 * np.max(np.abs(refi))


@pytest.mark.parametrize("shape", [(128, 128), (32, 48, 64), (384,), (4096,)])
def test_fft_vs_library(shape):
    x = rand_c(shape, 7)
    ref = np.fft.fftn(x)
    assert np.max(np.abs(O.fftn(x) - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_parseval_and_round_trip():
    x = rand_c((24, 32, 18), 3)
    X = O.fftn(x)
    assert abs(np.sum(np.abs(x) ** 2) - np.sum(np.abs(X) ** 2) / x.size) <= 1e-11 * np.sum(np.abs(x) ** 2)
    assert np.max(np.abs(O.ifftn(X) - x)) <= 1e-13 * np.max(np.abs(x))


def test_batch_matches_per_row():
    x = rand_c((5, 96), 11)
    B = O.fft_batch(x)
    for r in range(5):
        assert np.max(np.abs(B[r] - brute_dftn(x[r]))) <= 1e-12 * np.max(np.abs(B[r]))
    assert np.max(np.abs(O.ifft_batch(B) - x)) <= 1e-13 * np.max(np.abs(x))


def test_single_mode_lands_on_its_bin():
    n = 48
    m = 7
    t = np.arange(n)
    X = O.fftn(np.exp(2j * math.pi * m * t / n))
    expect = np.zeros(n, dtype=complex)
    expect[m] = n
    assert np.max(np.abs(X - expect)) <= 1e-12 * n


@pytest.mark.parametrize("n", [1 << 18, 3 * (1 << 13), 4096 * 27])
def test_long_transform_task_schedule_is_bit_identical(n):
    """A single long 1-D transform runs its recursion's sub-transforms as tasks;
    the batched entry point runs the same recursion serially.  Same operations,
    same order: the results must be identical bit for bit."""
    r = np.random.default_rng(n)
    x = r.standard_normal(n) + 1j * r.standard_normal(n)
    assert np.array_equal(O.fftn(x), O.fft_batch(x[None, :])[0])
    assert np.array_equal(O.ifftn(x), O.ifft_batch(x[None, :])[0])
