"""Pins for the oracle's half-spectrum form: the spectrum of a real CH field
stored as kx = 0 .. N/2, block states on that half map, neighbours in the
omitted half activated through their conjugate counterparts (S1.2, Eq. S.4).

Each test checks the oracle against something other than itself: numpy's
real-to-complex transforms, the full-spectrum oracle where the two forms must
agree, or block maps and sigma values traced by hand from S1.1-S1.2.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

A, T, F = O.STATE_ACTIVE, O.STATE_TRANSITION, O.STATE_FROZEN


def _rng(seed):
    return np.random.default_rng(seed)


@pytest.mark.parametrize("dims", [(16,), (8, 12), (6, 8, 16), (4, 10, 12)])
def test_half_transforms_match_numpy_rfft(dims):
    x = _rng(1).standard_normal(dims)
    h = O.rfftn_half(x)
    assert h.shape == dims[:-1] + (dims[-1] // 2 + 1,)
    assert np.abs(h - np.fft.rfftn(x)).max() <= 1e-12 * np.abs(h).max()
    # Eq. S.4: the Hermitian extension of the stored half is the full DFT
    assert np.abs(O.hermitian_extend(h, dims) - np.fft.fftn(x)).max() <= 1e-12 * np.abs(h).max()
    assert np.abs(O.ch_real_field_half(h, dims) - x).max() <= 1e-13


@pytest.mark.parametrize("dims", [(8, 12), (6, 8, 16)])
def test_half_inverse_of_non_symmetric_planes_is_numpys_irfftn(dims):
    """Stored kx = 0 and kx = N/2 planes that are not conjugate-symmetric within
    themselves: c is what a complex-to-real transform gives (their Hermitian part)."""
    r = _rng(2)
    h = r.standard_normal(dims[:-1] + (dims[-1] // 2 + 1,)) + 1j * r.standard_normal(
        dims[:-1] + (dims[-1] // 2 + 1,))
    c = O.ch_real_field_half(h, dims)
    ref = np.fft.irfftn(h, s=dims, axes=tuple(range(len(dims))))
    assert np.abs(c - ref).max() <= 1e-13 * np.abs(ref).max()


def test_half_grid_wavenumbers_and_block_counts():
    dims = (16, 8, 32)
    k2h = O.k_squared_half(dims)
    assert k2h.shape == (16, 8, 17)
    assert np.array_equal(k2h, O.k_squared(dims)[..., :17])
    assert O.half_block_counts(dims, (8, 8, 8)) == (2, 1, 3)
    assert O.half_block_counts((64, 64, 64), (8, 8, 8)) == (8, 8, 5)
    with pytest.raises(ValueError):
        O.half_block_counts((16, 16, 24), (8, 8, 8))   # 2 B does not divide 24


def test_half_block_measures_put_the_nyquist_column_in_the_last_block():
    dims = (16, 32)
    h = np.zeros((16, 17), dtype=np.complex128)
    h[3, 16] = 3.0 + 4.0j     # kx = N/2: the last block, alone in it
    h[9, 7] = 1.0             # block (1, 0)
    mx, sm = O.half_block_measures(h, dims, (8, 8))
    assert mx.shape == (2, 3)
    assert mx[0, 2] == 25.0 and sm[0, 2] == 25.0
    assert mx[1, 0] == 1.0
    assert np.count_nonzero(mx) == 2


def test_half_neighbours_across_kx0_and_past_nyquist():
    nbs = (4, 6, 3)
    # inside the stored half: direct; other axes periodic
    assert O.half_neighbour((1, 2, 1), 2, -1, nbs) == (1, 2, 0)
    assert O.half_neighbour((1, 2, 1), 2, +1, nbs) == (1, 2, 2)
    assert O.half_neighbour((0, 5, 1), 0, -1, nbs) == (3, 5, 1)
    assert O.half_neighbour((0, 5, 1), 1, +1, nbs) == (0, 0, 1)
    # left of kx = 0: the conjugate block, mirrored (b -> nb - 1 - b), stays at x-block 0
    assert O.half_neighbour((1, 2, 0), 2, -1, nbs) == (2, 3, 0)
    assert O.half_neighbour((0, 0, 0), 2, -1, nbs) == (3, 5, 0)
    # right of the Nyquist block: the mirrored block just below it
    assert O.half_neighbour((1, 2, 2), 2, +1, nbs) == (2, 3, 1)
    # 1-D: the block across kx = 0 is block 0 itself
    assert O.half_neighbour((0,), 0, -1, (5,)) == (0,)
    assert O.half_neighbour((4,), 0, +1, (5,)) == (3,)


def test_classify_half_hand_traced_2d():
    """32 x 32 field, 8 x 8 blocks: half map 4 x 3 (x-blocks kx 0-7, 8-15, 16).
    ACTIVE (1,0) requests (0,0), (2,0), (1,1) and, across kx = 0, the conjugate of
    (1,-1): (2,0).  ACTIVE (3,2) (Nyquist) requests (2,2), (0,2) (periodic in y),
    (3,1) and, past kx = N/2, the conjugate block (0,1)."""
    m = np.zeros((4, 3))
    m[1, 0] = m[3, 2] = 2.0
    got = O.classify_half(m, 1.0)
    want = np.array([[T, T, T],
                     [A, T, F],
                     [T, F, T],
                     [F, T, A]], dtype=np.uint8)
    assert np.array_equal(got, want)
    # the pull of (0,1) alone would miss the request from (3,2): the relation is not symmetric
    assert all(m[O.half_neighbour((0, 1), ax, d, (4, 3))] < 1.0 for ax in (0, 1) for d in (-1, 1))


def test_classify_half_hand_traced_3d():
    """16 x 16 x 32 field, 8^3 blocks: half map 2 x 2 x 3.  ACTIVE (0,1,0) requests
    (1,1,0) (both z faces), (0,0,0) (both y faces), (0,1,1) and across kx = 0 the
    mirrored (1,0,0).  ACTIVE (1,0,2) requests (0,0,2), (1,1,2), (1,0,1) and past the
    Nyquist block the mirrored (0,1,1)."""
    m = np.zeros((2, 2, 3))
    m[0, 1, 0] = m[1, 0, 2] = 5.0
    got = O.classify_half(m, 1.0)
    want = np.array([[[T, F, T], [A, T, F]],
                     [[T, T, A], [T, F, T]]], dtype=np.uint8)
    assert np.array_equal(got, want)
    # DC forcing and no transitions
    assert np.array_equal(O.classify_half(np.zeros((2, 2, 3)), 1.0, force_dc=True, transitions=False),
                          np.where(np.arange(12).reshape(2, 2, 3) == 0, A, F).astype(np.uint8))


def test_sigma_half_hand_traced():
    """Sigma of the 2-D map above (B = 8, w = taper(8)): faces whose neighbour --
    the conjugate block across kx = 0 or past the Nyquist block -- is FROZEN."""
    states = np.array([[T, T, T],
                       [A, T, F],
                       [T, F, T],
                       [F, T, A]], dtype=np.uint8)
    dims = (32, 32)
    sig = O.sigma_field_half(states, dims, (8, 8))
    assert sig.shape == (32, 17)
    w = O.taper(8)
    iy = np.arange(8)[:, None]
    ix = np.arange(8)[None, :]
    # (0,0): y- (3,0) FROZEN, y+ ACTIVE, across kx = 0 the conjugate (3,0) FROZEN, x+ (0,1) T
    assert np.array_equal(sig[0:8, 0:8], w[iy] * w[ix])
    # (1,1): y+ (2,1) FROZEN, x+ (1,2) FROZEN, the rest not
    assert np.array_equal(sig[8:16, 8:16], w[7 - iy] * w[7 - ix])
    # (0,2), the Nyquist column: y+ (1,2) FROZEN; past kx = N/2 the conjugate (3,1) is T
    assert np.array_equal(sig[0:8, 16], w[7 - np.arange(8)])
    # (2,2): y- (1,2) FROZEN and x- (2,1) FROZEN: the column at the x- face gets w(0) = 0
    assert np.array_equal(sig[16:24, 16], np.zeros(8))
    # ACTIVE blocks 1, FROZEN blocks 0
    assert np.all(sig[8:16, 0:8] == 1.0) and np.all(sig[24:32, 0:8] == 0.0)


def test_regular_half_step_is_the_half_of_the_full_step():
    dims = (8, 16, 16)
    c = W.ch_initial_condition(dims, mean=0.1, seed=W.BASE_SEED + 900)
    full = O.ch_regular_step(O.fftn(c), O.k_squared(dims), 0.01, 1.0)
    half = O.ch_regular_step_half(O.rfftn_half(c), dims, O.k_squared_half(dims), 0.01, 1.0)
    assert np.abs(half - full[..., :9]).max() <= 1e-12 * np.abs(full).max()


def test_half_regular_run_equals_full_regular_run():
    dims = (16, 16, 16)
    c0 = W.ch_initial_condition(dims, mean=-0.05, seed=W.BASE_SEED + 901)
    cfg = O.CHConfig(dims, (8, 8, 8), mode=0)
    hf, _ = O.run_ch(c0, cfg, 6)
    hh, _ = O.run_ch_half(c0, cfg, 6)
    assert O.rel_l2(O.ch_real_field_half(hh, dims), O.ch_real_field(hf)) <= 1e-12


def test_half_threshold_zero_is_regular_bit_for_bit():
    dims = (8, 16, 32)
    c0 = W.ch_initial_condition(dims, mean=0.0, seed=W.BASE_SEED + 902)
    reg, _ = O.run_ch_half(c0, O.CHConfig(dims, (8, 8, 8), mode=0), 5)
    ada, hist = O.run_ch_half(c0, O.CHConfig(dims, (8, 8, 8), threshold=0.0, reassess=2), 5)
    assert all(np.all(st == A) for _, st, _ in hist)
    assert np.array_equal(reg, ada)


def test_half_frozen_modes_are_untouched_and_dc_is_conserved():
    dims = (16, 16, 32)
    c0 = W.ch_initial_condition(dims, mean=0.2, seed=W.BASE_SEED + 903)
    h0 = O.rfftn_half(c0)
    cfg = O.CHConfig(dims, (8, 8, 8), threshold=1e30, reassess=1, transitions=False)
    h, hist = O.run_ch_half(c0, cfg, 3)
    st = hist[-1][1]
    assert st.flat[0] == A and np.count_nonzero(st) == 1
    assert np.array_equal(h[8:, :, :], h0[8:, :, :])
    assert np.array_equal(h[:, :, 8:], h0[:, :, 8:])
    assert h[0, 0, 0] == h0[0, 0, 0]
    assert np.any(h[:8, :8, :8] != h0[:8, :8, :8])


def test_half_adaptive_run_stays_close_to_regular():
    """The adaptive half form at a small relative threshold tracks Regular."""
    dims = (32, 32, 32)
    c0 = W.ch_initial_condition(dims, mean=0.1, seed=W.BASE_SEED + 904)
    reg, _ = O.run_ch_half(c0, O.CHConfig(dims, (8, 8, 8), mode=0), 40)
    ada, hist = O.run_ch_half(c0, O.CHConfig(dims, (8, 8, 8), threshold=1e-3, reassess=5), 40)
    assert any(np.count_nonzero(st == F) >= 5 for _, st, _ in hist)
    assert O.rel_l2(O.ch_real_field_half(ada, dims), O.ch_real_field_half(reg, dims)) <= 1e-5
