"""Pins of the oracle's reaction-cross-diffusion workload (Supplementary S4.1-S4.3)."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


@pytest.mark.parametrize("M", [2, 3, 5, 8, 48])
def test_circulant_eigenvalues_closed_form(M):
    """D is symmetric circulant: its eigenvalues are d + 2c - 2c cos(2 pi j / M)
    (M >= 3); for M = 2 the matrix [[d + 2c, -c], [-c, d + 2c]] has d + c, d + 3c."""
    d, c = 0.5, 0.05
    D = O.rcd_diffusion_matrix(M, d, c)
    assert np.allclose(D, D.T)
    lam, V = O.rcd_eigen(D)
    if M == 2:
        expect = np.array([d + c, d + 3 * c])
    else:
        expect = np.sort(d + 2 * c - 2 * c * np.cos(2 * math.pi * np.arange(M) / M))
    assert np.max(np.abs(np.sort(lam) - expect)) <= 1e-14
    assert np.max(np.abs(V @ np.diag(lam) @ V.T - D)) <= 1e-14
    assert np.max(np.abs(V.T @ V - np.eye(M))) <= 1e-14


def test_reaction_hand_computed_values():
    A3 = O.rcd_interaction_matrix(3, 1.0, 0.3)
    # M = 3: every other component is a neighbour: alpha_ij = 1.3
    u = np.array([0.2, 0.3, 0.5])
    R = O.rcd_reaction(u, np.ones(3), np.ones(3), A3)
    # R0 = 0.2 (1 - 0.2 - 1.3 (0.3 + 0.5)) = -0.048, R1 = 0.3 (1 - 0.3 - 1.3 (0.7)) = -0.063,
    # R2 = 0.5 (1 - 0.5 - 1.3 (0.5)) = -0.075
    assert np.allclose(R, [-0.048, -0.063, -0.075], rtol=0, atol=1e-15)
    # M = 5: neighbours (periodic) 1.3, the two others 0.3
    u = np.array([0.1, 0.2, 0.3, 0.4, 0.5])
    R = O.rcd_reaction(u, np.ones(5), np.ones(5), O.rcd_interaction_matrix(5, 1.0, 0.3))
    # R0 = 0.1 (1 - 0.1 - (1.3 (0.2 + 0.5) + 0.3 (0.3 + 0.4))) = 0.1 (0.9 - 1.12) = -0.022
    # R2 = 0.3 (1 - 0.3 - (1.3 (0.2 + 0.4) + 0.3 (0.1 + 0.5))) = 0.3 (0.7 - 0.96) = -0.078
    assert abs(R[0] - (-0.022)) <= 1e-15 and abs(R[2] - (-0.078)) <= 1e-15
    # M = 2: the single other component, 1.3: R0 = 0.4 (1 - 0.4 - 1.3 * 0.6) = -0.072
    R = O.rcd_reaction(np.array([0.4, 0.6]), np.ones(2), np.ones(2), O.rcd_interaction_matrix(2, 1.0, 0.3))
    assert abs(R[0] - (-0.072)) <= 1e-15


@pytest.mark.parametrize("M", [2, 3, 8, 48])
def test_homogeneous_state_is_a_fixed_point(M):
    us = W.rcd_lv_homogeneous(M)
    assert us == pytest.approx(O.rcd_homogeneous_state(M, 1.0, 1.0, 1.0, 0.3), rel=1e-15)
    R = O.rcd_reaction(np.full(M, us), np.ones(M), np.ones(M), O.rcd_interaction_matrix(M, 1.0, 0.3))
    assert np.max(np.abs(R)) <= 1e-16


@pytest.mark.parametrize("M", [2, 5, 24])
def test_direct_solve_equals_eigen_form(M):
    r = np.random.default_rng(M)
    D = O.rcd_diffusion_matrix(M, 0.5, 0.05)
    lam, V = O.rcd_eigen(D)
    b = r.standard_normal((M, 6, 7)) + 1j * r.standard_normal((M, 6, 7))
    k2 = r.random((6, 7)) * 40.0
    x1 = O.rcd_update_direct(b, k2, 0.01, D)
    x2 = O.rcd_update_eigen(b, k2, 0.01, V, lam)
    assert np.max(np.abs(x1 - x2)) <= 1e-13 * np.max(np.abs(x1))
    # and x1 solves the system
    for i in range(6):
        for j in range(7):
            A = np.eye(M) + 0.01 * k2[i, j] * D
            assert np.allclose(A @ x1[:, i, j], b[:, i, j], rtol=0, atol=1e-13)


@pytest.mark.parametrize("M,eigen", [(3, True), (4, False)])
def test_linearised_single_mode_growth(M, eigen):
    """u = u* + eps v cos(k.x): each Regular step multiplies the mode's component
    vector by G = (I + dt k^2 D)^{-1} (I + dt J), J the reaction Jacobian at u*
    (J_ii = -a u*, J_ij = -u* alpha_ij), up to O(eps^2)."""
    dims = (16, 16)
    cfg = O.RCDConfig(dims, (4, 4), M, mode=0, eigen=eigen)
    us = W.rcd_lv_homogeneous(M)
    eps = 1e-7
    v = np.random.default_rng(1).standard_normal(M)
    kx, ky = 3, 2
    x = np.arange(dims[1]) * cfg.dx
    y = np.arange(dims[0]) * cfg.dx
    kvx = 2 * math.pi * kx / (dims[1] * cfg.dx)
    kvy = 2 * math.pi * ky / (dims[0] * cfg.dx)
    phase = np.cos(kvy * y[:, None] + kvx * x[None, :])
    u0 = us + eps * v[:, None, None] * phase[None]
    steps = 5
    u_hat, _ = O.run_rcd(u0, cfg, steps)
    # the cos mode's amplitude vector: 2 Re(u_hat[:, ky, kx]) / N
    amp = 2.0 * np.real(u_hat[:, ky, kx]) / (dims[0] * dims[1])
    A = O.rcd_interaction_matrix(M, cfg.alpha, cfg.beta)
    J = -us * A - cfg.a * us * np.eye(M)
    D = O.rcd_diffusion_matrix(M, cfg.d_diag, cfg.d_cross)
    k2 = kvx * kvx + kvy * kvy
    G = np.linalg.solve(np.eye(M) + cfg.dt * k2 * D, np.eye(M) + cfg.dt * J)
    expect = eps * np.linalg.matrix_power(G, steps) @ v
    assert np.max(np.abs(amp - expect)) <= 1e-6 * np.max(np.abs(expect))
    # the mean stays at u* to O(eps^2)
    assert np.max(np.abs(np.real(u_hat[:, 0, 0]) / (dims[0] * dims[1]) - us)) <= 1e-12


def test_threshold_zero_equals_regular_and_infinite_freezes():
    dims, M = (16, 16), 3
    us = W.rcd_lv_homogeneous(M)
    u0 = W.rcd_initial_condition(dims, M, us, 0.1, seed=5)
    reg, _ = O.run_rcd(u0, O.RCDConfig(dims, (4, 4), M, mode=0), 6)
    ada, hist = O.run_rcd(u0, O.RCDConfig(dims, (4, 4), M, threshold=0.0, reassess=2), 6)
    assert np.array_equal(ada, reg)
    assert all(np.all(st == O.STATE_ACTIVE) for _, st, _ in hist)
    inf, hist = O.run_rcd(u0, O.RCDConfig(dims, (4, 4), M, threshold=np.inf, reassess=2,
                                          transitions=False), 6)
    u_hat0 = np.stack([O.fftn(x) for x in u0])
    changed = np.any(inf != u_hat0, axis=0)
    assert changed[:4, :4].any() and not changed[4:, :].any() and not changed[:, 4:].any()


def test_activity_is_the_component_rms_amplitude():
    q = np.zeros((2, 8, 8), dtype=np.complex128)
    q[0, 1, 2] = 3 + 4j          # |q|^2 = 25
    q[1, 1, 2] = 1.0             # |q|^2 = 1  -> A^2 = 13
    q[1, 6, 6] = 2j              # A^2 = 2
    cfg = O.RCDConfig((8, 8), (4, 4), 2, threshold=0.5, force_dc=False, transitions=False)
    states, tau, measure = O.rcd_assess_states(q, cfg)
    assert measure[0, 0] == math.sqrt(13.0) and measure[1, 1] == math.sqrt(2.0)
    assert tau == 0.5 * math.sqrt(13.0)
    assert states[0, 0] == O.STATE_ACTIVE and states[1, 1] == O.STATE_FROZEN
