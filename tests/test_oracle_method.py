"""Pins for the oracle's sp-DBA logic and its Cahn-Hilliard step.

Each test checks the oracle against something other than itself: a closed
form, an invariant, a special case, or hand-derived values (tests/golden/).
"""
import math
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return rows


# ---------------------------------------------------------------- taper and sigma (S1.1)
def test_taper_matches_hand_values():
    for row in load_golden("taper_values.txt"):
        B = int(row[0])
        assert np.allclose(O.taper(B), row[1:], rtol=0, atol=1e-15)


def test_sigma_2d_worked_case():
    expect = np.array(load_golden("sigma_2d_B4.txt"))
    # 3x3 block map, B = 4; centre block TRANSITION, lower-x (left) and lower-y
    # neighbours FROZEN, the other two ACTIVE.
    st = np.full((3, 3), O.STATE_ACTIVE, dtype=np.uint8)
    st[1, 1] = O.STATE_TRANSITION
    st[1, 0] = O.STATE_FROZEN   # left: lower index along x (axis 1)
    st[0, 1] = O.STATE_FROZEN   # lower along y (axis 0)
    sig = O.sigma_field(st, (4, 4))
    assert np.allclose(sig[4:8, 4:8], expect, rtol=0, atol=1e-15)
    # active blocks carry sigma = 1, frozen ones 0
    assert np.all(sig[8:12, 4:8] == 1.0)
    assert np.all(sig[4:8, 0:4] == 0.0)


def test_sigma_upper_faces_and_3d():
    w = O.taper(8)
    st = np.full((3, 3, 3), O.STATE_ACTIVE, dtype=np.uint8)
    st[1, 1, 1] = O.STATE_TRANSITION
    st[1, 1, 2] = O.STATE_FROZEN   # upper x
    st[2, 1, 1] = O.STATE_FROZEN   # upper z
    sig = O.sigma_field(st, (8, 8, 8))[8:16, 8:16, 8:16]
    z, y, x = np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij")
    assert np.allclose(sig, w[7 - x] * w[7 - z], rtol=0, atol=1e-15)


# ---------------------------------------------------------------- states (Methods)
def test_classify_hand_built_with_wrap():
    m = np.zeros((4, 4))
    m[0, 3] = 5.0          # active at a corner: neighbours wrap around
    m[2, 1] = 1.0          # exactly at tau: active (>=)
    st = O.classify(m, tau=1.0, force_dc=False)
    A, T, F = O.STATE_ACTIVE, O.STATE_TRANSITION, O.STATE_FROZEN
    expect = np.array([[T, F, T, A],
                       [F, T, F, T],
                       [T, A, T, F],
                       [F, T, F, T]], dtype=np.uint8)
    assert np.array_equal(st, expect)


def test_classify_force_dc_and_no_transitions():
    m = np.zeros((3, 4, 5))
    st = O.classify(m, tau=1.0, force_dc=True, transitions=False)
    assert st[0, 0, 0] == O.STATE_ACTIVE and np.count_nonzero(st) == 1
    st = O.classify(m, tau=1.0, force_dc=True, transitions=True)
    assert np.count_nonzero(st == O.STATE_TRANSITION) == 6   # 6 face neighbours in 3-D


def test_block_measures_by_loops():
    q = np.random.default_rng(5).standard_normal((8, 12)) + 1j * np.random.default_rng(6).standard_normal((8, 12))
    mx, sm = O.block_measures(q, (4, 4))
    for by in range(2):
        for bx in range(3):
            blk = q[4 * by:4 * by + 4, 4 * bx:4 * bx + 4]
            vals = [abs(v) ** 2 for v in blk.ravel()]
            assert math.isclose(mx[by, bx], max(vals), rel_tol=1e-15)
            assert math.isclose(sm[by, bx], sum(vals), rel_tol=1e-13)


def test_effective_states_refresh_and_warmup():
    cfg = O.CHConfig((16, 16), (4, 4), refresh_every=5, warmup_steps=3)
    st = np.zeros((4, 4), dtype=np.uint8)
    for n in range(12):
        eff = O.effective_states(st, n, cfg)
        all_active = n < 3 or (n > 0 and n % 5 == 0)
        assert np.all(eff == O.STATE_ACTIVE) == all_active


# ---------------------------------------------------------------- CH step
@pytest.mark.parametrize("cbar,mode", [(0.3, (1, 2)), (0.3, (5, 3)), (0.0, (2, 0)), (0.55, (1, 1))])
def test_ch_single_mode_closed_form(cbar, mode):
    """Linearised about a uniform state, mode k grows by exactly
    G = (1 - dt k^2 (3 cbar^2 - 1)) / (1 + dt kappa k^4) per step."""
    N, dt, kappa, eps, steps = 32, 0.05, 1.0, 1e-6, 10
    y, x = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    kx, ky = 2 * math.pi * mode[1] / N, 2 * math.pi * mode[0] / N
    c0 = cbar + eps * np.cos(kx * x + ky * y)
    k2grid = O.k_squared((N, N))
    c_hat = O.fftn(c0)
    for _ in range(steps):
        c_hat = O.ch_regular_step(c_hat, k2grid, dt, kappa)
    k2 = kx * kx + ky * ky
    G = (1 - dt * k2 * (3 * cbar ** 2 - 1)) / (1 + dt * kappa * k2 * k2)
    amp = c_hat[mode[0], mode[1]].real * 2 / (N * N)
    assert abs(amp - eps * G ** steps) <= 1e-8 * eps * G ** steps
    growing = k2 < (1 - 3 * cbar ** 2) / kappa
    assert (G > 1) == growing


def test_ch_k0_conserved_bitwise():
    c0 = W.ch_initial_condition((32, 32), mean=0.1, seed=3)
    cfg = O.CHConfig((32, 32), (8, 8), threshold=1e-3, reassess=2, mode=1)
    c_hat0 = O.fftn(c0)
    c_hat, _ = O.run_ch(c0, cfg, 7)
    assert c_hat[0, 0] == c_hat0[0, 0]
    assert abs(O.ch_mass(c_hat) - c_hat0[0, 0].real) <= 1e-12 * abs(c_hat0[0, 0].real)


def test_threshold_zero_equals_regular_bitwise():
    c0 = W.ch_initial_condition((32, 48), mean=0.0, seed=4)
    a, hist = O.run_ch(c0, O.CHConfig((32, 48), (8, 8), threshold=0.0, reassess=3, mode=1), 9)
    b, _ = O.run_ch(c0, O.CHConfig((32, 48), (8, 8), mode=0), 9)
    assert np.array_equal(a, b)
    assert all(np.all(st == O.STATE_ACTIVE) for _, st, _ in hist)


@pytest.mark.parametrize("transitions", [False, True])
def test_infinite_threshold_freezes_all_but_dc(transitions):
    dims, block = (32, 32), (8, 8)
    c0 = W.ch_initial_condition(dims, mean=0.2, seed=5)
    cfg = O.CHConfig(dims, block, threshold=math.inf, tau_rule=O.TAU_ABS, reassess=1,
                     transitions=transitions)
    c_hat0 = O.fftn(c0)
    c_hat, hist = O.run_ch(c0, cfg, 4)
    st = hist[-1][1]
    changed = np.zeros(st.shape, dtype=bool)
    for by in range(4):
        for bx in range(4):
            sl = (slice(8 * by, 8 * by + 8), slice(8 * bx, 8 * bx + 8))
            changed[by, bx] = not np.array_equal(c_hat[sl], c_hat0[sl])
    assert np.array_equal(changed, st != O.STATE_FROZEN)
    assert st[0, 0] == O.STATE_ACTIVE
    assert np.count_nonzero(st == O.STATE_ACTIVE) == 1


def test_transition_edge_modes_next_to_frozen_face_unchanged():
    """w(0) = 0: the row of modes touching a frozen neighbour keeps its value."""
    dims, block = (32, 32), (8, 8)
    c0 = W.ch_initial_condition(dims, seed=6)
    c_hat = O.fftn(c0)
    st = np.zeros((4, 4), dtype=np.uint8)
    st[0, 0] = O.STATE_ACTIVE
    st[0, 1] = O.STATE_TRANSITION  # right of the DC block; its upper-x neighbour (0,2) is frozen
    new = O.ch_masked_step(c_hat, st, block, O.k_squared(dims), 0.01, 1.0)
    assert np.array_equal(new[0:8, 15], c_hat[0:8, 15])
    assert not np.array_equal(new[0:8, 12], c_hat[0:8, 12])


def test_energy_measure_is_block_l2_norm():
    q = W.ch_initial_condition((16, 16), seed=9) + 0j
    cfg = O.CHConfig((16, 16), (4, 4), measure=O.MEASURE_ENERGY, tau_rule=O.TAU_ABS, threshold=0.0)
    _, _, meas = O.assess_states(q, cfg, exclude_dc=True)
    blk = q[4:8, 8:12]
    assert math.isclose(meas[1, 2], math.sqrt(np.sum(np.abs(blk) ** 2)), rel_tol=1e-14)


def test_rel_max_threshold_excludes_dc():
    q = np.zeros((8, 8), dtype=complex)
    q[0, 0] = 1e6
    q[3, 5] = 2.0 + 0j
    assert O.threshold_value(q, 0.5, O.TAU_REL_MAX, exclude_dc=True) == 1.0
    assert O.threshold_value(q, 0.5, O.TAU_REL_MAX, exclude_dc=False) == 5e5
