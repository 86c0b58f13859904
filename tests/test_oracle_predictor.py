"""Pins for the CPU reference of the block-activity predictor (no paper counterpart)."""
import numpy as np
import pytest

from oracle import predictor_ref as R


def test_bf16_rounding_known_values():
    # bfloat16 has 7 fraction bits (ulp(1) = 2^-7): 1 + 2^-7 is exact; 1 + 2^-8 is a
    # tie and goes to the even neighbour 1; 1 + 3*2^-8 ties between 1 + 2^-7 (odd)
    # and 1 + 2^-6 (even); 1 + 2^-8 + 2^-12 is above the tie and rounds up
    x = np.array([1.0, 1 + 2 ** -7, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -8 + 2 ** -12, -2.5, 0.0])
    expect = np.array([1.0, 1 + 2 ** -7, 1.0, 1 + 2 ** -6, 1 + 2 ** -7, -2.5, 0.0])
    assert np.array_equal(R.bf16(x), expect)


def test_conv_matches_direct_loops():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 4, 5, 2))
    W = rng.standard_normal((3, 27, 2))
    y = R.conv(x, W)
    D, H, Wd = 3, 4, 5
    for z, yy, xx in [(0, 0, 0), (2, 3, 4), (1, 2, 0)]:
        for o in range(3):
            acc = 0.0
            for dz in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        tap = 9 * (dz + 1) + 3 * (dy + 1) + (dx + 1)
                        src = x[(z + dz) % D, (yy + dy) % H, (xx + dx) % Wd]
                        acc += W[o, tap] @ src
            assert abs(y[z, yy, xx, o] - acc) <= 1e-12


def _loss(P, x, y):
    p, _ = R.forward(P, x)
    return R.bce(p, y)


@pytest.mark.parametrize("name", ["W1", "b1", "W2", "b3", "wh", "bh"])
def test_backward_matches_central_differences(name):
    rng = np.random.default_rng(2)
    P = R.init_params(3)
    for k in P:
        if k.startswith("b"):
            P[k] = P[k] + 0.05 * rng.standard_normal(P[k].shape)
    x = rng.standard_normal((2, 4, 4, 4, 2))
    y = (rng.random((2, 4, 4, 4)) < 0.3).astype(float)
    _, G = R.backward(P, x, y)
    flat = P[name].reshape(-1)
    idx = rng.choice(flat.size, size=min(6, flat.size), replace=False)
    h = 1e-6
    for i in idx:
        old = flat[i]
        flat[i] = old + h
        lp = _loss(P, x, y)
        flat[i] = old - h
        lm = _loss(P, x, y)
        flat[i] = old
        fd = (lp - lm) / (2 * h)
        g = G[name].reshape(-1)[i]
        assert abs(fd - g) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (name, i, fd, g)


def test_adam_first_step_moves_by_lr():
    P = {"w": np.array([1.0, -2.0])}
    G = {"w": np.array([0.5, -3.0])}
    M = {"w": np.zeros(2)}
    V = {"w": np.zeros(2)}
    R.adam_step(P, G, M, V, 1, lr=0.1)
    # bias-corrected first step is lr * sign(g) (up to eps)
    assert np.allclose(P["w"], [0.9, -1.9], atol=1e-7)
