"""Reaction-cross-diffusion (Supplementary S4.1-S4.3) on the GPU against the oracle.

Masks in lock-step: at every reassessment the GPU's M-component spectrum
(promoted to FP64) goes through the oracle's classifier (component RMS
amplitude, one state per block) and must give the GPU's states, tie band
excepted.  Fields: the oracle re-runs the steps in FP64 with the GPU's states
(its update through the eigendecomposition, pinned against the direct dense
solve), so the comparison measures arithmetic error only.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from _helpers import states_within_tie_band

pytestmark = pytest.mark.gpu


def _ic(dims, M, seed):
    return W.rcd_initial_condition(dims, M, W.rcd_lv_homogeneous(M), 0.1, seed=seed)


def run_gpu(dims, block, M, steps, precision, u0, R=5, threshold=1e-6, lockstep=True, **kw):
    from paper_2609_03922_gb300 import spdba
    rdt = np.float32 if precision == 0 else np.float64
    plan = spdba.Plan(dims, block, threshold=threshold, reassess=R, precision=precision, model=spdba.SPDBA_MODEL_RCD,
                      components=M, dx=0.5, **kw)
    plan.set_field(np.ascontiguousarray(u0.astype(rdt)))
    masks, spectra, coef = {}, {}, {}
    adaptive = kw.get("mode", 1) == 1
    for s in range(steps):
        if adaptive and lockstep and s % R == 0:
            spectra[s] = plan.get_spectrum()
            plan.step(1)
            masks[s] = plan.get_mask()
            coef[s] = plan.get_stats()["threshold"]
        else:
            plan.step(1)
    field = plan.get_field()
    stats = plan.get_stats()
    plan.close()
    return field, masks, spectra, coef, stats


def oracle_cfg(dims, block, M, R=5, threshold=1e-6, **kw):
    kw = dict(kw)
    kw.pop("use_graph", None)
    return O.RCDConfig(dims, block, M, threshold=threshold, reassess=R, **kw)


def check(dims, block, M, steps, precision, tol, seed, R=5, threshold=1e-6, **kw):
    u0 = _ic(dims, M, seed)
    field, masks, spectra, coef, stats = run_gpu(dims, block, M, steps, precision, u0, R=R, threshold=threshold, **kw)
    cfg = oracle_cfg(dims, block, M, R=R, threshold=threshold, **kw)
    for s, sp in spectra.items():
        st, tau, meas = O.rcd_assess_states(sp.astype(np.complex128), cfg, threshold=coef[s])
        ok, nties = states_within_tie_band(masks[s], meas, tau, cfg)
        assert ok, "step %d: GPU states differ from the oracle's (%d tie-band blocks)" % (s, nties)
    rdt = np.float32 if precision == 0 else np.float64
    ref_hat, _ = O.run_rcd(u0.astype(rdt).astype(np.float64), cfg, steps,
                           on_assess=lambda n, q, st, tau: masks.get(n))
    ref = O.rcd_real_field(ref_hat)
    err = O.rel_l2(field, ref)
    assert err <= tol, "rel-L2 %.3e > %.1e" % (err, tol)
    return field, masks, stats, err


@pytest.mark.parametrize("M", [3, 8])
def test_rcd_2d_fp64_lockstep(M):
    _, masks, stats, _ = check((32, 32), (4, 4), M, 100, 1, 1e-10, seed=W.BASE_SEED + 60 + M, threshold=1e-3)
    # the run does skip blocks, and every state setting was checked
    assert any(np.any(m == O.STATE_FROZEN) for m in masks.values())
    assert stats["assessments"] == 20


def test_rcd_3d_c64_lockstep():
    _, masks, _, err = check((32, 32, 32), (4, 4, 4), 8, 60, 0, 2e-5, seed=W.BASE_SEED + 70, threshold=1e-4)
    assert any(np.any(m == O.STATE_FROZEN) for m in masks.values())


@pytest.mark.parametrize("M", [1, 2, 5, 64])
def test_rcd_regular_fp64_edge_component_counts(M):
    """Regular mode for the special component counts: M = 1 (no coupling), M = 2
    (one off-diagonal entry), M = 64 (the largest)."""
    dims = (16, 16)
    u0 = _ic(dims, M, W.BASE_SEED + 80 + M)
    field, _, _, _, _ = run_gpu(dims, (4, 4), M, 20, 1, u0, mode=0)
    ref_hat, _ = O.run_rcd(u0, O.RCDConfig(dims, (4, 4), M, mode=0), 20)
    assert O.rel_l2(field, O.rcd_real_field(ref_hat)) <= 1e-11


def test_rcd_threshold_zero_equals_regular_on_gpu():
    dims, M = (32, 32, 32), 8
    u0 = _ic(dims, M, W.BASE_SEED + 90).astype(np.float32)
    a, masks, _, _, _ = run_gpu(dims, (8, 8, 8), M, 12, 0, u0, threshold=0.0, R=4)
    b, _, _, _, _ = run_gpu(dims, (8, 8, 8), M, 12, 0, u0, mode=0)
    assert np.array_equal(a, b)
    assert all(np.all(m == O.STATE_ACTIVE) for m in masks.values())


def test_rcd_control_lockstep():
    """Dynamic threshold control on an RCD run (S4.2: adjustment factor 0.1,
    interval 50; here 20): the GPU coefficient sequence equals the oracle
    controller's fed with the GPU's states, bit for bit."""
    dims, block, M, steps, R = (32, 32), (4, 4), 4, 120, 5
    kw = dict(target_ratio=0.3, control_every=20, control_eta=0.1)
    u0 = _ic(dims, M, W.BASE_SEED + 95)
    field, masks, spectra, coef, stats = run_gpu(dims, block, M, steps, 1, u0, R=R, threshold=1e-6, **kw)
    cfg = O.RCDConfig(dims, block, M, threshold=1e-6, reassess=R, **kw)
    ctl = O.ThresholdController(cfg, 64)
    cur = None
    for s in range(steps):
        thr = ctl.begin_step(s)
        if s in masks:
            assert coef[s] == thr
            st, tau, meas = O.rcd_assess_states(spectra[s].astype(np.complex128), cfg, threshold=thr)
            ok, _ = states_within_tie_band(masks[s], meas, tau, cfg)
            assert ok
            cur = masks[s]
        ctl.end_step(s, cur)
    assert stats["controls"] == len(ctl.log) == steps // 20 - 1
    ref_hat, _ = O.run_rcd(u0, cfg, steps, on_assess=lambda n, q, st, tau: masks.get(n))
    assert O.rel_l2(field, O.rcd_real_field(ref_hat)) <= 1e-10


def test_rcd_rejects_bad_component_counts():
    from paper_2609_03922_gb300 import spdba
    for M in (0, 65):
        with pytest.raises(spdba.SpdbaError) as ei:
            spdba.Plan((32, 32), (8, 8), model=spdba.SPDBA_MODEL_RCD, components=M)
        assert ei.value.status == spdba.SPDBA_ERR_UNSUPPORTED
    with pytest.raises(spdba.SpdbaError):
        spdba.Plan((64,), (8,), model=spdba.SPDBA_MODEL_RCD, components=4)


def test_rcd_graph_replay_equals_stepwise():
    import torch
    from paper_2609_03922_gb300 import spdba
    dims, M = (32, 32, 32), 8
    u0 = _ic(dims, M, W.BASE_SEED + 97).astype(np.float32)
    side = torch.cuda.Stream()
    out = []
    with torch.cuda.stream(side):
        for chunk in (60, 1):
            with spdba.Plan(dims, (8, 8, 8), threshold=1e-4, reassess=10, model=spdba.SPDBA_MODEL_RCD,
                            components=M, dx=0.5) as pl:
                pl.set_field(u0)
                for _ in range(60 // chunk):
                    pl.step(chunk)
                out.append(pl.get_spectrum())
    assert np.array_equal(out[0], out[1])
