"""Dynamic threshold control (Supplementary S1.3) on the GPU against the oracle.

Lock-step: at every reassessment the GPU's spectrum (promoted to FP64) goes
through the oracle's classifier with the oracle controller's coefficient, and
must give the GPU's states (tie band excepted).  The oracle controller is fed
the GPU's own states, so its coefficient sequence must equal the GPU's bit
for bit (both form r from exact integer counts and take the same FP64
decisions).  The oracle then re-runs the steps with the GPU's states (control
steps all-active on both sides) and the fields must agree to rounding.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from _helpers import states_within_tie_band

pytestmark = pytest.mark.gpu


def _lockstep(plan, cfg, steps, run=0):
    """Step `plan` one step at a time; returns (masks, spectra, coefficient per reassessment)."""
    R = cfg.reassess
    masks, spectra, coef = {}, {}, {}
    for s in range(steps):
        if s % R == 0:
            spectra[s] = plan.get_spectrum(run=run)
            plan.step(1)
            masks[s] = plan.get_mask(run=run)
            coef[s] = plan.get_stats(run=run)["threshold"]
        else:
            plan.step(1)
    return masks, spectra, coef


def _check_lockstep(cfg, masks, spectra, coef, steps, nblocks, exclude_dc):
    ctl = O.ThresholdController(cfg, nblocks)
    cur = None
    for s in range(steps):
        thr = ctl.begin_step(s)
        if s in masks:
            assert coef[s] == thr, "step %d: GPU coefficient %.17g, oracle %.17g" % (s, coef[s], thr)
            st, tau, meas = O.assess_states(spectra[s].astype(np.complex128), cfg, exclude_dc=exclude_dc,
                                            threshold=thr)
            ok, nties = states_within_tie_band(masks[s], meas, tau, cfg)
            assert ok, "step %d: GPU states differ from the oracle's (%d tie-band blocks)" % (s, nties)
            cur = masks[s]
        ctl.end_step(s, cur)
    return ctl


@pytest.mark.parametrize("precision,dims,block,tol", [
    (1, (128, 128), (8, 8), 1e-11),
    (0, (64, 64, 64), (8, 8, 8), 2e-5),
])
def test_ch_control_lockstep(precision, dims, block, tol):
    from paper_2609_03922_gb300 import spdba
    steps, R = 240, 5
    kw = dict(target_ratio=0.2, control_every=20, control_eta=0.05)
    c0 = W.ch_initial_condition(dims, mean=0.1 if len(dims) == 3 else 0.0, seed=W.BASE_SEED + 7)
    rdt = np.float32 if precision == 0 else np.float64
    c0 = c0.astype(rdt)
    nb = int(np.prod([d // b for d, b in zip(dims, block)]))
    cfg = O.CHConfig(dims, block, threshold=1e-6, reassess=R, **kw)
    with spdba.Plan(dims, block, threshold=1e-6, reassess=R, precision=precision, **kw) as plan:
        plan.set_field(np.ascontiguousarray(c0))
        masks, spectra, coef = _lockstep(plan, cfg, steps)
        field = plan.get_field()
        stats = plan.get_stats()
    ctl = _check_lockstep(cfg, masks, spectra, coef, steps, nb, exclude_dc=True)
    assert stats["controls"] == len(ctl.log) == steps // 20 - 1
    assert stats["threshold"] == ctl.threshold
    assert ctl.threshold > 1e-6          # the ratio started far above the target: raised
    ref_hat, _ = O.run_ch(c0.astype(np.float64), cfg, steps, on_assess=lambda n, ch, st, tau: masks.get(n))
    err = O.rel_l2(field, O.ch_real_field(ref_hat))
    assert err <= tol, "rel-L2 %.3e > %.1e" % (err, tol)


def test_ch_control_graph_replay_equals_stepwise():
    """Free-running steps (graph-replayed segments, control steps launched directly)
    give the same field and coefficient as one-step-at-a-time stepping."""
    import torch
    from paper_2609_03922_gb300 import spdba
    dims, block = (64, 64, 64), (8, 8, 8)
    c0 = W.ch_initial_condition(dims, mean=0.1, seed=W.BASE_SEED + 8).astype(np.float32)
    kw = dict(target_ratio=0.1, control_every=50, control_eta=0.05, precision=spdba.SPDBA_C64)
    side = torch.cuda.Stream()
    out = []
    with torch.cuda.stream(side):
        for chunk in (300, 1):
            with spdba.Plan(dims, block, threshold=1e-6, reassess=10, **kw) as pl:
                pl.set_field(c0)
                for _ in range(300 // chunk):
                    pl.step(chunk)
                out.append((pl.get_spectrum(), pl.get_stats()))
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1]["threshold"] == out[1][1]["threshold"] and out[0][1]["controls"] == 5


@pytest.mark.parametrize("precision,tol", [(1, 1e-10), (0, 2e-4)])
def test_nls_control_lockstep(precision, tol):
    """Batch of a short (single-kernel) and a long (row/column) signal, each run
    with its own coefficient."""
    from paper_2609_03922_gb300 import spdba
    lengths = [4096, 16384]
    steps, R = 120, 5
    kw = dict(target_ratio=0.1, control_every=20, control_eta=0.05)
    cdt = np.complex64 if precision == 0 else np.complex128
    sigs = [W.nls_signal(n, seed=W.BASE_SEED + 40 + i).astype(cdt) for i, n in enumerate(lengths)]
    plan = spdba.Plan(None, (-64,), threshold=1e-6, reassess=R, batch_dims=[(n,) for n in lengths],
                      model=spdba.SPDBA_MODEL_NLS, precision=precision, **kw)
    for r, E in enumerate(sigs):
        plan.set_field(np.ascontiguousarray(E), run=r)
    masks = [dict() for _ in lengths]
    spectra = [dict() for _ in lengths]
    coef = [dict() for _ in lengths]
    for s in range(steps):
        if s % R == 0:
            for r in range(len(lengths)):
                spectra[r][s] = plan.get_spectrum(run=r)
            plan.step(1)
            for r in range(len(lengths)):
                masks[r][s] = plan.get_mask(run=r)
                coef[r][s] = plan.get_stats(run=r)["threshold"]
        else:
            plan.step(1)
    fields = [plan.get_field(run=r) for r in range(len(lengths))]
    plan.close()
    for r, n in enumerate(lengths):
        cfg = O.NLSConfig(n, n // 64, threshold=1e-6, reassess=R, **kw)
        ctl = _check_lockstep(cfg, masks[r], spectra[r], coef[r], steps, 64, exclude_dc=False)
        assert len(ctl.log) == steps // 20 - 1
        ref, _ = O.run_nls(sigs[r].astype(np.complex128), cfg, steps, on_assess=lambda s, E, st, tau, r=r: masks[r].get(s))
        err = O.rel_l2(fields[r], ref)
        assert err <= tol, "signal %d: rel-L2 %.3e > %.1e" % (r, err, tol)


def test_control_rejects_bad_options_and_predictor():
    from paper_2609_03922_gb300 import spdba
    with pytest.raises(spdba.SpdbaError):
        spdba.Plan((32, 32), (8, 8), target_ratio=1.5)
    with pytest.raises(spdba.SpdbaError):
        spdba.Plan((32, 32), (8, 8), target_ratio=0.1, control_eta=0.0)
    with pytest.raises(spdba.SpdbaError):
        spdba.Plan((32, 32), (8, 8), target_ratio=0.1, control_every=0)
    pr = spdba.Predictor((4, 4, 4), max_batch=1)
    with spdba.Plan((32, 32, 32), (8, 8, 8), target_ratio=0.1) as pl:
        with pytest.raises(spdba.SpdbaError) as ei:
            pl.attach_predictor(pr, 20, 100, 0.5)
        assert ei.value.status == spdba.SPDBA_ERR_STATE
