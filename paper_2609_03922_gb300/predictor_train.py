"""Training the block-activity predictor on traces that the method itself produces.

A trace is an adaptive Cahn-Hilliard run with exact reassessments every `R`
steps; at every reassessment it records the per-block activity (max |c_hat|^2,
FP64), tau and the block states.  A training sample at a prediction point t
(a multiple of the horizon K) pairs
  input  = features(activity of the last exact judge t0 <= t, states in force before t)
  label  = 1 where the block is non-frozen at any exact reassessment in [t, t + K)
which is what the attached predictor sees and must answer in the solver loop
(judges every J steps, predictions in between).  Features and all training
arithmetic run in the library's kernels; this module only moves arrays.
"""
import numpy as np

from . import spdba


def collect_trace(dims, block, c0, steps, reassess=10, threshold=1e-6, stream=None, **opts):
    """Run an exact adaptive CH run; returns dict with maxsq (n, nb...) float64,
    tau (n,), states (n, nb...) uint8 and the reassessment steps."""
    plan = spdba.Plan(dims, block, threshold=threshold, reassess=reassess, stream=stream, **opts)
    plan.set_field(np.ascontiguousarray(c0))
    maxsq, tau, states, at = [], [], [], []
    for s in range(0, steps, reassess):
        plan.step(1)            # the reassessment at step s happens at the start of this step
        m, t = plan.get_activity()
        maxsq.append(m)
        tau.append(t)
        states.append(plan.get_mask())
        at.append(s)
        plan.step(reassess - 1)
    plan.close()
    return {"maxsq": np.stack(maxsq), "tau": np.array(tau), "states": np.stack(states), "steps": np.array(at),
            "reassess": reassess}


def build_samples(trace, horizon=20, judge_every=100):
    """(activity index, state index, label) triples for every prediction point."""
    R = trace["reassess"]
    steps = trace["steps"]
    nonfrozen = trace["states"] != 0
    idx = {int(s): i for i, s in enumerate(steps)}
    out = []
    for t in range(horizon, int(steps[-1]) - horizon + R + 1, horizon):
        if t not in idx:
            continue
        t0 = (t // judge_every) * judge_every
        prev = t - R
        if t0 not in idx or prev not in idx:
            continue
        window = [idx[s] for s in range(t, t + horizon, R) if s in idx]
        if len(window) < horizon // R:
            continue
        label = np.any(nonfrozen[window], axis=0).astype(np.float32)
        out.append((idx[t0], idx[prev], label))
    return out


def make_inputs(predictor, trace, samples):
    """Device features (bf16) and labels for a list of samples, built by the
    library's feature kernel."""
    import torch
    n = len(samples)
    shape = trace["maxsq"].shape[1:]
    maxsq = torch.from_numpy(np.stack([trace["maxsq"][a] for a, _, _ in samples])).cuda()
    tau = torch.from_numpy(np.array([trace["tau"][a] for a, _, _ in samples])).cuda()
    states = torch.from_numpy(np.stack([trace["states"][b] for _, b, _ in samples])).cuda()
    labels = torch.from_numpy(np.stack([l for _, _, l in samples])).cuda()
    x = torch.empty((n,) + shape + (2,), dtype=torch.bfloat16, device="cuda")
    vox = int(np.prod(shape))
    for i in range(0, n, predictor.max_batch):
        k = min(predictor.max_batch, n - i)
        predictor.features(maxsq[i:i + k], tau[i:i + k], states[i:i + k], x[i:i + k], nmaps=k)
    torch.cuda.synchronize()
    return x, labels


def train(predictor, x, labels, epochs=40, lr=3e-3, seed=0):
    """Adam over mini-batches of maps; returns the per-epoch mean loss."""
    import torch
    n = x.shape[0]
    rng = np.random.default_rng(seed)
    hist = []
    B = predictor.max_batch
    for _ in range(epochs):
        order = rng.permutation(n)
        losses = []
        for i in range(0, n - B + 1, B):
            sel = torch.from_numpy(order[i:i + B]).cuda()
            xb = x.index_select(0, sel).contiguous()
            yb = labels.index_select(0, sel).contiguous()
            losses.append(predictor.train_step(xb, yb, lr, nmaps=B))
        hist.append(float(np.mean(losses)))
    return hist


class TrainedPredictor(spdba.Predictor):
    """A predictor with its map size and batch recorded (max_batch attribute)."""

    def __init__(self, map_dims, max_batch=8, **kw):
        super().__init__(map_dims, max_batch=max_batch, **kw)
        self.max_batch = max_batch
