"""The identities the Hermitian half-spectrum passes rest on, checked with
numpy's FFT on small random fields (no GPU, no oracle arithmetic):

- c = Re(IFFT(c_hat)) equals the inverse transform of the Hermitian part
  h(k) = (c_hat(k) + conj(c_hat(-k))) / 2, which is real;
- the 3-D transform D of a real field satisfies D(-k) = conj(D(k)), so the z
  transform of a half pencil (ky, kx) also gives the mirror pencil
  (-ky, N2 - kx) at frequency -kz, conjugated (the paired z forward);
- two real rows x1, x2 share one complex transform W of x1 + i x2:
  X1[k] = (W[k] + conj W[-k]) / 2, X2[k] = (W[k] - conj W[-k]) / (2i)
  (the x pass).
"""
import numpy as np
import pytest

SHAPES = [(8, 6, 10), (4, 12, 16), (6, 6, 6)]


def _neg(a):
    """a(-k) on every axis (index -k mod N)."""
    return np.roll(np.flip(a, axis=tuple(range(a.ndim))), 1, axis=tuple(range(a.ndim)))


@pytest.mark.parametrize("shape", SHAPES)
def test_real_part_is_inverse_of_hermitian_part(shape):
    r = np.random.default_rng(11)
    c_hat = r.standard_normal(shape) + 1j * r.standard_normal(shape)   # not Hermitian
    h = 0.5 * (c_hat + np.conj(_neg(c_hat)))
    c = np.fft.ifftn(c_hat).real
    ch = np.fft.ifftn(h)
    assert np.max(np.abs(ch.imag)) <= 1e-13 * np.max(np.abs(ch.real))
    assert np.allclose(ch.real, c, rtol=0, atol=1e-13 * np.max(np.abs(c)))
    # h is the Hermitian part: h(-k) = conj(h(k)), and c_hat - h is anti-Hermitian
    assert np.allclose(_neg(h), np.conj(h), atol=1e-14)
    assert np.allclose(np.fft.ifftn(c_hat - h).real, 0.0, atol=1e-13)


@pytest.mark.parametrize("shape", SHAPES)
def test_mirror_pencils_from_half_pencils(shape):
    """z transform of the half array's pencil (ky, kx), kx <= N2/2, at frequency m
    gives the full transform at (m, ky, kx) and, conjugated, at (-m, -ky, N2 - kx)."""
    r = np.random.default_rng(12)
    g = r.standard_normal(shape)
    n0, n1, n2 = shape
    half = np.fft.fft(np.fft.fft(g, axis=1), axis=2)[:, :, : n2 // 2 + 1]   # y and x transforms, x <= N2/2
    full = np.fft.fftn(g)
    dz = np.fft.fft(half, axis=0)                                          # the z forward of the half array
    for ky in range(n1):
        for kx in range(n2 // 2 + 1):
            for m in range(n0):
                assert np.isclose(dz[m, ky, kx], full[m, ky, kx], atol=1e-11)
                mz, my, mx = (-m) % n0, (-ky) % n1, (n2 - kx) % n2
                assert np.isclose(np.conj(dz[m, ky, kx]), full[mz, my, mx], atol=1e-11)


@pytest.mark.parametrize("n", [8, 10, 64])
def test_two_real_rows_in_one_complex_transform(n):
    r = np.random.default_rng(13)
    x1, x2 = r.standard_normal(n), r.standard_normal(n)
    w = np.fft.fft(x1 + 1j * x2)
    wneg = np.conj(np.roll(w[::-1], 1))                                     # conj W[-k]
    assert np.allclose(0.5 * (w + wneg), np.fft.fft(x1), atol=1e-12)
    assert np.allclose((w - wneg) / 2j, np.fft.fft(x2), atol=1e-12)
    # and the inverse direction: half spectra k <= n/2 rebuild the packed row
    k = np.arange(n)
    z = np.where(k <= n // 2, np.fft.fft(x1)[np.minimum(k, n - k)], np.conj(np.fft.fft(x1)[(n - k) % n]))
    z = z + 1j * np.where(k <= n // 2, np.fft.fft(x2)[np.minimum(k, n - k)], np.conj(np.fft.fft(x2)[(n - k) % n]))
    assert np.allclose(np.fft.ifft(z), x1 + 1j * x2, atol=1e-12)
