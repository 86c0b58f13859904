"""CPU reference of the block-activity predictor (TEST INFRASTRUCTURE ONLY).

The predictor has no counterpart in the paper: it is a small 3-D convolutional
network over the per-block activity map that predicts which blocks will be
non-frozen over the next K steps.  Network (periodic 3x3x3 convolutions over
the block map, channels-last arrays of shape (D, H, W, C)):

    a1 = conv(x, W1) + b1;  h1 = relu(a1)       2 -> 8 channels
    a2 = conv(h1, W2) + b2; h2 = relu(a2)       8 -> 16
    a3 = conv(h2, W3) + b3; h3 = relu(a3)       16 -> 8
    z  = h3 . wh + bh;      p = sigmoid(z)      8 -> 1
    L  = mean over voxels and samples of -[y log p + (1 - y) log(1 - p)]

conv(x, W)[v, o] = sum_{tap, i} W[o, tap, i] x[v + off(tap), i], with
off(tap) = (dz, dy, dx), tap = 9 (dz + 1) + 3 (dy + 1) + (dx + 1), indices
wrapping periodically (the block map of a periodic spectrum wraps).

`forward`/`backward` run in FP64.  With round_bf16=True they round to
bfloat16 (round to nearest even) at the points where the GPU kernels store
bfloat16: the input, the weights, h1..h3, and the pre-activation gradients
da1..da3 (the derivative of the rounding is taken as 1).
"""
import numpy as np

LAYERS = [(2, 8), (8, 16), (16, 8)]
OFFSETS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def shift(x, off):
    """y[z, y, x] = x[z + dz, y + dy, x + dx] (periodic)."""
    dz, dy, dx = off
    return np.roll(x, shift=(-dz, -dy, -dx), axis=(0, 1, 2))


def conv(x, W):
    """x: (D, H, W, Cin); W: (Cout, 27, Cin) -> (D, H, W, Cout)."""
    out = np.zeros(x.shape[:3] + (W.shape[0],))
    for tap, off in enumerate(OFFSETS):
        out += shift(x, off) @ W[:, tap, :].T
    return out


def conv_dgrad(dy, W):
    """Gradient of conv with respect to its input: sum over taps of dy shifted back."""
    out = np.zeros(dy.shape[:3] + (W.shape[2],))
    for tap, off in enumerate(OFFSETS):
        out += shift(dy, tuple(-o for o in off)) @ W[:, tap, :]
    return out


def conv_wgrad(dy, x):
    """dW[o, tap, i] = sum_v dy[v, o] x[v + off(tap), i]."""
    cout, cin = dy.shape[3], x.shape[3]
    dW = np.zeros((cout, 27, cin))
    dyf = dy.reshape(-1, cout)
    for tap, off in enumerate(OFFSETS):
        dW[:, tap, :] = dyf.T @ shift(x, off).reshape(-1, cin)
    return dW


def init_params(seed=0):
    """He-style random initialisation (FP64); a dict of arrays."""
    rng = np.random.default_rng(seed)
    P = {}
    for l, (ci, co) in enumerate(LAYERS, start=1):
        P["W%d" % l] = rng.standard_normal((co, 27, ci)) * np.sqrt(2.0 / (27 * ci))
        P["b%d" % l] = np.zeros(co)
    P["wh"] = rng.standard_normal(8) * np.sqrt(1.0 / 8)
    P["bh"] = np.zeros(1)
    return P


def forward(P, x, round_bf16=False):
    """x: (S, D, H, W, 2).  Returns (p, cache)."""
    R = bf16 if round_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    cache = {"x": [], "a": [], "h": []}
    ps = []
    for s in range(x.shape[0]):
        h = R(x[s])
        hs, As = [h], []
        for l in range(1, 4):
            a = conv(h, R(P["W%d" % l])) + P["b%d" % l]
            h = R(np.maximum(a, 0.0))
            As.append(a)
            hs.append(h)
        z = hs[3] @ P["wh"] + P["bh"][0]
        ps.append(1.0 / (1.0 + np.exp(-z)))
        cache["a"].append(As)
        cache["h"].append(hs)
    return np.stack(ps), cache


def bce(p, y):
    eps = 1e-12
    return float(-np.mean(y * np.log(p + eps) + (1 - y) * np.log(1 - p + eps)))


def backward(P, x, y, round_bf16=False):
    """Gradients of the mean BCE loss; returns (loss, grads dict)."""
    R = bf16 if round_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    p, cache = forward(P, x, round_bf16)
    n = p.size
    G = {k: np.zeros_like(v) for k, v in P.items()}
    for s in range(x.shape[0]):
        hs, As = cache["h"][s], cache["a"][s]
        dz = (p[s] - y[s]) / n
        G["wh"] += np.tensordot(dz, hs[3], axes=([0, 1, 2], [0, 1, 2]))
        G["bh"] += dz.sum()
        dh = dz[..., None] * P["wh"]
        for l in range(3, 0, -1):
            da = R(dh * (As[l - 1] > 0))
            G["W%d" % l] += conv_wgrad(da, hs[l - 1])
            G["b%d" % l] += da.sum(axis=(0, 1, 2))
            if l > 1:
                dh = conv_dgrad(da, R(P["W%d" % l]))
    return bce(p, y), G


def adam_step(P, G, M, V, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t counts from 1), in place on P, M, V."""
    for k in P:
        M[k] = b1 * M[k] + (1 - b1) * G[k]
        V[k] = b2 * V[k] + (1 - b2) * G[k] * G[k]
        mh = M[k] / (1 - b1 ** t)
        vh = V[k] / (1 - b2 ** t)
        P[k] = P[k] - lr * mh / (np.sqrt(vh) + eps)
