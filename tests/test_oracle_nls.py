"""Pins for the oracle's split-step NLS (S5.1-S5.3 with M = 1, alpha = 0)."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


def test_cw_exact_solution():
    """A CW sitting on a bin evolves as A exp(i (beta2 w0^2 / 2 + gamma |A|^2) z)."""
    n, m, A = 1024, 37, 0.1
    beta2, gamma, h, steps = -21.7, 1.3, 0.1, 25
    E0 = W.nls_cw(n, m, A)
    H = O.nls_half_factor(O.nls_omega(n, 1.0), beta2, h)
    E = E0
    for _ in range(steps):
        E = O.nls_regular_step(E, H, gamma, h)
    w0 = 2 * math.pi * m / n
    z = steps * h
    expect = E0 * np.exp(1j * (beta2 * w0 * w0 / 2 + gamma * A * A) * z)
    assert np.max(np.abs(E - expect)) <= 1e-12 * A


def test_dispersion_only_gaussian_broadening():
    """gamma = 0: |E(z,t)|^2 = (T0/T) exp(-t^2/T^2), T = T0 sqrt(1 + (beta2 z / T0^2)^2)."""
    n, T0, beta2, h, steps = 4096, 20.0, -21.7, 0.1, 800
    E0 = W.gaussian_pulse(n, T0)
    cfg = O.NLSConfig(n, 64, beta2=beta2, gamma=0.0, h=h, mode=0)
    E, _ = O.run_nls(E0, cfg, steps)
    z = steps * h
    T = T0 * math.sqrt(1 + (beta2 * z / T0 ** 2) ** 2)
    t = np.arange(n) - n / 2.0
    expect = (T0 / T) * np.exp(-t * t / (T * T))
    assert np.max(np.abs(np.abs(E) ** 2 - expect)) <= 1e-10
    # the spectrum's magnitude is untouched by dispersion
    assert np.allclose(np.abs(O.fftn(E)), np.abs(O.fftn(E0)), rtol=0, atol=1e-9)


@pytest.mark.parametrize("mode,transitions", [(0, True), (1, False)])
def test_energy_conserved(mode, transitions):
    n = 2048
    E0 = W.nls_signal(n, seed=21)
    cfg = O.NLSConfig(n, n // 64, threshold=1e-3, reassess=5, mode=mode, transitions=transitions)
    E, _ = O.run_nls(E0, cfg, 40)
    e0 = np.sum(np.abs(E0) ** 2)
    assert abs(np.sum(np.abs(E) ** 2) - e0) <= 1e-12 * e0


def test_signal_occupies_eight_slots_exactly():
    n = 4096
    E = W.nls_signal(n, seed=3)
    S = np.abs(O.fftn(E))
    occ = [bool(np.any(S[s * 128:(s + 1) * 128] > 1e-9 * S.max())) for s in range(32)]
    assert sum(occ) == 8
    # each channel is scaled to 10 mW peak; the sum peaks at no more than 8 x (sqrt sum)^2
    assert np.max(np.abs(E) ** 2) <= 64 * 0.01 + 1e-12


def test_forward_then_adaptive_backward_recovers():
    """Dense forward propagation followed by sp-DBA back-propagation with the
    negated (beta2, gamma) recovers the transmitted field (S5.3: NMSE <= -20 dB)."""
    n, steps = 4096, 200
    E_tx = W.nls_signal(n, seed=8)
    fwd = O.NLSConfig(n, n // 64, mode=0)
    E_rx, _ = O.run_nls(E_tx, fwd, steps)
    # Kerr mixing spreads the received spectrum to ~1e-2 of its peak in every
    # slot, so a threshold of 1e-2 x max is the one that leaves blocks frozen.
    back = O.NLSConfig(n, n // 64, beta2=+21.7, gamma=-1.3, threshold=1e-2, reassess=10, mode=1)
    E_rec, hist = O.run_nls(E_rx, back, steps)
    assert O.nmse_db(E_rec, E_tx) <= -20.0
    assert O.field_corr(E_rec, E_tx) >= 0.998
    # activation follows the occupied bands: some blocks were frozen
    assert any(np.any(st == O.STATE_FROZEN) for _, st, _ in hist)


def test_metrics_closed_form():
    x = np.ones(10, dtype=complex)
    assert math.isclose(O.nmse_db(1.1 * x, x), 10 * math.log10(0.01), rel_tol=1e-12)
    assert math.isclose(O.field_corr(2j * x, x), 1.0, rel_tol=1e-15)
    assert math.isclose(O.rel_l2(1.5 * x, x), 0.5, rel_tol=1e-15)


def test_masked_half_step_transition_weights_by_hand():
    """One linear half-step on a 1-D map of 4 blocks of B = 4 bins with states
    (ACTIVE, TRANSITION, FROZEN, FROZEN): the ACTIVE block takes E H, the FROZEN
    blocks keep E, and the TRANSITION block (its lower neighbour ACTIVE, its upper
    neighbour FROZEN) takes E + w(B-1-i) (E H - E) with the taper
    w = (1 - cos(pi i / 3)) / 2 = (0, 1/4, 3/4, 1), so w(3 - i) = (1, 3/4, 1/4, 0)
    (S1.1, Eq. S.1-S.3)."""
    n, B = 16, 4
    E = (np.arange(n) + 1.0) * (1.0 + 0.5j)
    H = np.exp(1j * 0.1 * np.arange(n))
    states = np.array([O.STATE_ACTIVE, O.STATE_TRANSITION, O.STATE_FROZEN, O.STATE_FROZEN], dtype=np.uint8)
    out = O.nls_masked_half(E, states, (B,), H)
    new = E * H
    assert np.array_equal(out[0:4], new[0:4])
    assert np.array_equal(out[8:16], E[8:16])
    expect = [1.0, 0.75, 0.25, 0.0]
    for i in range(4):
        k = 4 + i
        assert abs(out[k] - (E[k] + expect[i] * (new[k] - E[k]))) <= 1e-15 * abs(E[k])
    # the mode touching the frozen face keeps its value exactly (w(0) = 0)
    assert out[7] == E[7]
    # periodic wrap: a TRANSITION block at the start whose lower neighbour (the last
    # block) is FROZEN takes w(i) = (0, 1/4, 3/4, 1) when its upper neighbour is ACTIVE
    states = np.array([O.STATE_TRANSITION, O.STATE_ACTIVE, O.STATE_FROZEN, O.STATE_FROZEN], dtype=np.uint8)
    out = O.nls_masked_half(E, states, (B,), H)
    for i, w in enumerate([0.0, 0.25, 0.75, 1.0]):
        assert abs(out[i] - (E[i] + w * (new[i] - E[i]))) <= 1e-15 * abs(E[i])
