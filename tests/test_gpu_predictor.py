"""The predictor's BF16 tensor-core kernels against the CPU reference (FP64 with the
same BF16 rounding points), and its training on the GPU."""
import numpy as np
import pytest

from oracle import predictor_ref as R

pytestmark = pytest.mark.gpu


def _flat(P):
    return np.concatenate([P[k].reshape(-1) for k in ["W1", "b1", "W2", "b2", "W3", "b3", "wh", "bh"]])


def _unflat(v):
    P, o = {}, 0
    for k, shape in [("W1", (8, 27, 2)), ("b1", (8,)), ("W2", (16, 27, 8)), ("b2", (16,)), ("W3", (8, 27, 16)),
                     ("b3", (8,)), ("wh", (8,)), ("bh", (1,))]:
        n = int(np.prod(shape))
        P[k] = np.asarray(v[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return P


def _data(shape, nmaps, seed):
    r = np.random.default_rng(seed)
    x = R.bf16(r.standard_normal((nmaps,) + shape + (2,)))
    y = (r.random((nmaps,) + shape) < 0.35).astype(np.float64)
    return x, y


def _to_dev(x, y):
    import torch
    xd = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).cuda().contiguous()
    yd = torch.from_numpy(y.astype(np.float32)).cuda().contiguous()
    return xd, yd


@pytest.mark.parametrize("shape,nmaps", [((8, 8, 8), 2), ((6, 10, 12), 1), ((32, 32, 32), 1)])
def test_forward_matches_reference(shape, nmaps):
    import torch
    from paper_2609_03922_gb300 import spdba
    P = R.init_params(4)
    P["b1"] += 0.1
    params = _flat(P).astype(np.float32)
    pr = spdba.Predictor(shape, max_batch=nmaps, params=params)
    x, _ = _data(shape, nmaps, 5)
    xd, _ = _to_dev(x, np.zeros((nmaps,) + shape))
    prob = torch.empty((nmaps,) + shape, dtype=torch.float32, device="cuda")
    pr.forward(xd, prob, nmaps=nmaps)
    torch.cuda.synchronize()
    ref, _ = R.forward(_unflat(params), x, round_bf16=True)
    assert np.max(np.abs(prob.cpu().numpy() - ref)) <= 2e-3
    pr.close()


@pytest.mark.parametrize("shape", [(8, 8, 8), (6, 10, 12)])
def test_gradients_match_reference(shape):
    from paper_2609_03922_gb300 import spdba
    P = R.init_params(6)
    for k in ("b1", "b2", "b3"):
        P[k] = P[k] + 0.05
    params = _flat(P).astype(np.float32)
    pr = spdba.Predictor(shape, max_batch=2, params=params)
    x, y = _data(shape, 2, 7)
    xd, yd = _to_dev(x, y)
    loss, g = pr.gradients(xd, yd, nmaps=2)
    ref_loss, G = R.backward(_unflat(params), x, y, round_bf16=True)
    assert abs(loss - ref_loss) <= 1e-4 * abs(ref_loss)
    Gg = _unflat(g)
    for k in G:
        num = np.linalg.norm(Gg[k] - G[k])
        den = np.linalg.norm(G[k])
        assert num <= 1e-2 * den + 1e-9, (k, num / max(den, 1e-30))
    pr.close()


def test_training_reduces_loss_on_a_learnable_map():
    """Labels that are a fixed function of the inputs (a smoothed indicator of the
    activity channel) are learned by Adam on the GPU."""
    import torch
    from paper_2609_03922_gb300 import spdba
    shape = (16, 16, 16)
    r = np.random.default_rng(9)
    x = np.zeros((4,) + shape + (2,))
    x[..., 0] = R.bf16(r.uniform(-1, 1, (4,) + shape))
    x[..., 1] = (x[..., 0] > 0).astype(float)
    y = np.zeros((4,) + shape)
    for s in range(4):
        act = (x[s, ..., 0] > 0.2).astype(float)
        near = sum(np.roll(act, d, axis=a) for a in range(3) for d in (-1, 1))
        y[s] = ((act + near) > 0).astype(float)
    xd, yd = _to_dev(x, y)
    pr = spdba.Predictor(shape, max_batch=4, seed=1)
    first = pr.train_step(xd, yd, 3e-3, nmaps=4)
    for _ in range(300):
        last = pr.train_step(xd, yd, 3e-3, nmaps=4)
    prob = torch.empty((4,) + shape, dtype=torch.float32, device="cuda")
    pr.forward(xd, prob, nmaps=4)
    torch.cuda.synchronize()
    acc = float(((prob.cpu().numpy() > 0.5) == (y > 0.5)).mean())
    assert last < 0.5 * first
    assert acc >= 0.9
    pr.close()


def test_features_kernel_definition():
    import torch
    from paper_2609_03922_gb300 import spdba
    shape = (4, 4, 4)
    r = np.random.default_rng(3)
    maxsq = np.exp(r.uniform(-40, 10, (2,) + shape))
    maxsq[0, 0, 0, 0] = 0.0
    tau = np.array([1e-3, 2.0])
    states = r.integers(0, 3, (2,) + shape).astype(np.uint8)
    pr = spdba.Predictor(shape, max_batch=2)
    x = torch.empty((2,) + shape + (2,), dtype=torch.bfloat16, device="cuda")
    pr.features(torch.from_numpy(maxsq).cuda(), torch.from_numpy(tau).cuda(), torch.from_numpy(states).cuda(), x,
                nmaps=2)
    torch.cuda.synchronize()
    got = x.float().cpu().numpy()
    with np.errstate(divide="ignore"):
        f = np.log10(np.sqrt(maxsq) / tau[:, None, None, None]) / 8.0
    f = np.clip(f, -1, 1)
    assert np.allclose(got[..., 0], R.bf16(f), atol=0)
    assert np.array_equal(got[..., 1], (states != 0).astype(np.float32))
    pr.close()
