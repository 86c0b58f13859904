"""Adaptive and Regular Cahn-Hilliard on the GPU against the oracle, through the C ABI.

Masks: at every reassessment the GPU's spectrum (promoted to FP64) goes
through the oracle's classifier and must give the GPU's states, blocks in
the 1e-6 tie band excepted (lock-step).  Fields: the oracle re-runs the same
steps in FP64 with the GPU's (checked) states, so the comparison measures
arithmetic error only.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from _helpers import states_within_tie_band

pytestmark = pytest.mark.gpu


def run_gpu(dims, block, steps, precision, c0, **kw):
    from paper_2609_03922_gb300 import spdba
    R = kw.pop("reassess", 10)
    thr = kw.pop("threshold", 1e-6)
    rdt = np.float32 if precision == 0 else np.float64
    plan = spdba.Plan(dims, block, threshold=thr, reassess=R, precision=precision, **kw)
    plan.set_field(np.ascontiguousarray(c0.astype(rdt)))
    masks, spectra = {}, {}
    mode = kw.get("mode", 1)
    for s in range(steps):
        if mode == 1 and s % R == 0:
            spectra[s] = plan.get_spectrum()
            plan.step(1)
            masks[s] = plan.get_mask()
        else:
            plan.step(1)
    field = plan.get_field()
    stats = plan.get_stats()
    spec = plan.get_spectrum()
    plan.close()
    return field, spec, masks, spectra, stats


def oracle_cfg(dims, block, **kw):
    kw = dict(kw)
    kw.pop("precision", None)
    kw.pop("use_graph", None)
    return O.CHConfig(dims, block, **kw)


def check_run(dims, block, steps, precision, c0, tol, **kw):
    field, spec, masks, spectra, stats = run_gpu(dims, block, steps, precision, c0, **kw)
    cfg = oracle_cfg(dims, block, **kw)
    # lock-step masks on the GPU's own spectrum
    for s, sp in spectra.items():
        st, tau, meas = O.assess_states(sp.astype(np.complex128), cfg, exclude_dc=True)
        ok, nties = states_within_tie_band(masks[s], meas, tau, cfg)
        assert ok, "step %d: GPU block states differ from the oracle's (%d tie-band blocks)" % (s, nties)
    # oracle with the GPU's states
    rdt = np.float32 if precision == 0 else np.float64
    c0r = c0.astype(rdt).astype(np.float64)
    ref_hat, _ = O.run_ch(c0r, cfg, steps, on_assess=lambda n, ch, st, tau: masks[n] if n in masks else None)
    ref = O.ch_real_field(ref_hat)
    err = O.rel_l2(field, ref)
    assert err <= tol, "rel-L2 %.3e > %.1e" % (err, tol)
    return field, spec, stats, err, spectra


def test_config1_2d_128_fp64_full_run():
    """2-D CH 128^2, FP64, 16^2 blocks, tau = 1e-6 max|c_hat|, R = 10, 200 steps."""
    dims, block = (128, 128), (16, 16)
    c0 = W.ch_initial_condition(dims, mean=0.0, amplitude=0.05, seed=W.BASE_SEED)
    check_run(dims, block, 200, 1, c0, 1e-10)


@pytest.mark.parametrize("precision,tol1,side", [(0, 1e-5, 64), (1, 1e-12, 64), (0, 1e-5, 128), (0, 1e-5, 32)])
def test_one_step_3d(precision, tol1, side):
    dims, block = (side, side, side), (8, 8, 8)
    c0 = W.ch_initial_condition(dims, mean=0.1, seed=W.BASE_SEED + 1)
    check_run(dims, block, 1, precision, c0, tol1)


def test_3d_fp32_many_steps_with_fp64_norms():
    dims, block = (64, 64, 64), (8, 8, 8)
    c0 = W.ch_initial_condition(dims, mean=0.1, seed=W.BASE_SEED + 2)
    _, spec, stats, _, spectra = check_run(dims, block, 120, 0, c0, 1e-4)
    # k = 0 is never touched by the update: bit-identical to its value after set_field
    assert spec[0, 0, 0] == spectra[0][0, 0, 0]
    c0r = c0.astype(np.float32).astype(np.float64)
    assert abs(spec[0, 0, 0].real - np.sum(c0r)) <= 1e-6 * abs(np.sum(c0r))
    # FP64 mass of the real field at the last reassessment
    assert abs(stats["mass"] - np.sum(c0r)) <= 1e-6 * abs(np.sum(c0r))
    assert stats["assessments"] == 12


@pytest.mark.parametrize("opts", [dict(transitions=0), dict(measure=1), dict(reassess=1),
                                  dict(refresh_every=7, warmup_steps=3), dict(force_dc=0, threshold=1e-3)])
def test_options_2d(opts):
    dims, block = (64, 128), (16, 16)
    c0 = W.ch_initial_condition(dims, mean=0.2, seed=W.BASE_SEED + 3)
    check_run(dims, block, 25, 1, c0, 1e-11, **opts)


@pytest.mark.parametrize("precision", [0, 1])
def test_threshold_zero_equals_regular_on_gpu(precision):
    dims, block = (32, 32, 32), (8, 8, 8)
    c0 = W.ch_initial_condition(dims, mean=0.0, seed=W.BASE_SEED + 4)
    a = run_gpu(dims, block, 15, precision, c0, threshold=0.0, reassess=4)
    b = run_gpu(dims, block, 15, precision, c0, mode=0)
    assert np.array_equal(a[1], b[1])
    assert all(np.all(m == 2) for m in a[2].values())


def test_zero_field_stays_zero():
    dims, block = (32, 32), (8, 8)
    field, spec, masks, _, stats = run_gpu(dims, block, 5, 0, np.zeros(dims))
    assert not np.any(field) and not np.any(spec)
    assert all(np.all(m == 2) for m in masks.values())   # tau = 0 * 0: every block meets it


@pytest.mark.parametrize("shape,block", [((192, 384), (16, 16)), ((512, 512), (16, 16)), ((32, 192, 64), (8, 8, 8))])
def test_ragged_radix3_and_large_2d(shape, block):
    c0 = W.ch_initial_condition(shape, mean=0.05, seed=W.BASE_SEED + 5)
    check_run(shape, block, 12, 0, c0, 1e-5)


def test_full_size_256cubed_fp32():
    """The benchmark workload: 3-D CH 256^3, complex64, 8^3 blocks, R = 10."""
    dims, block = (256, 256, 256), (8, 8, 8)
    c0 = W.ch_initial_condition(dims, mean=0.1, seed=W.BASE_SEED)
    check_run(dims, block, 11, 0, c0, 1e-5)


def test_fp32_full_step_count_at_64cubed():
    """Precision form over the configuration's full 2000 steps (at 64^3, where the
    FP64 oracle finishes): rel-L2 <= 1e-4 against FP64 with the same states."""
    dims, block = (64, 64, 64), (8, 8, 8)
    c0 = W.ch_initial_condition(dims, mean=0.1, seed=W.BASE_SEED + 7)
    check_run(dims, block, 2000, 0, c0, 1e-4)


def test_uneven_ensemble_plan_matches_per_run_oracle():
    """One plan holding runs of different sizes (the ensemble form) steps each run
    exactly like the oracle would."""
    from paper_2609_03922_gb300 import spdba
    sizes = [(128, 128), (192, 192), (256, 256)]
    means = [0.1, -0.15, 0.0]
    c0s = [W.ch_initial_condition(s, mean=m, seed=W.BASE_SEED + 10 + i) for i, (s, m) in enumerate(zip(sizes, means))]
    plan = spdba.Plan(None, (16, 16), threshold=1e-6, reassess=5, batch_dims=sizes, precision=0)
    for r, c0 in enumerate(c0s):
        plan.set_field(np.ascontiguousarray(c0.astype(np.float32)), run=r)
    steps = 20
    masks = [dict() for _ in sizes]
    for s in range(steps):
        plan.step(1)
        if s % 5 == 0:
            for r in range(len(sizes)):
                masks[r][s] = plan.get_mask(run=r)
    for r, (dims, c0) in enumerate(zip(sizes, c0s)):
        got = plan.get_field(run=r)
        cfg = O.CHConfig(dims, (16, 16), threshold=1e-6, reassess=5)
        ref_hat, hist = O.run_ch(c0.astype(np.float32).astype(np.float64), cfg, steps,
                                 on_assess=lambda n, ch, st, tau, r=r: masks[r][n])
        assert O.rel_l2(got, O.ch_real_field(ref_hat)) <= 1e-5
    plan.close()


@pytest.mark.parametrize("shape,block,batch", [((64, 64, 64), (8, 8, 8), 1), ((128, 128), (16, 16), 3)])
def test_fused_update_equals_staged_update(shape, block, batch):
    """The update applied inside the last forward FFT pass gives exactly the values of
    the separate list/dense update kernels (same arithmetic, same states)."""
    from paper_2609_03922_gb300 import spdba
    outs = []
    for fuse in (1, 0):
        dims = [shape] * batch
        plan = spdba.Plan(None, block, threshold=1e-2, reassess=3, batch_dims=dims, precision=0, fuse_update=fuse)
        for r in range(batch):
            c0 = W.ch_initial_condition(shape, mean=0.1 * r, seed=W.BASE_SEED + 40 + r)
            plan.set_field(np.ascontiguousarray(c0.astype(np.float32)), run=r)
        plan.step(14)
        outs.append([(plan.get_spectrum(run=r), plan.get_mask(run=r), plan.get_stats(run=r)) for r in range(batch)])
        plan.close()
    for (sa, ma, ta), (sb, mb, tb) in zip(*outs):
        assert np.array_equal(sa, sb)
        assert np.array_equal(ma, mb)
        assert abs(ta["active_ratio_sum"] - tb["active_ratio_sum"]) < 1e-9
    assert any(np.any(m == 0) for _, m, _ in outs[0])   # some blocks were frozen


@pytest.mark.parametrize("model", ["ch", "nls"])
def test_graph_replay_equals_direct_launches(model):
    """Reassessment segments captured once in a CUDA graph and replayed give the
    same fields, masks and statistics as launching every kernel directly."""
    import torch
    from paper_2609_03922_gb300 import spdba
    outs = []
    for use_graph in (1, 0):
        side = torch.cuda.Stream()
        with torch.cuda.stream(side):
            if model == "ch":
                dims = [(128, 128), (128, 128), (192, 192)]
                plan = spdba.Plan(None, (16, 16), threshold=1e-3, reassess=5, batch_dims=dims, precision=0,
                                  use_graph=use_graph)
                inputs = [W.ch_initial_condition(d, mean=0.05 * i, seed=W.BASE_SEED + 60 + i).astype(np.float32)
                          for i, d in enumerate(dims)]
            else:
                dims = [(4096,), (8192,), (4096,)]
                plan = spdba.Plan(None, (-64,), threshold=1e-3, reassess=5, batch_dims=dims,
                                  model=spdba.SPDBA_MODEL_NLS, precision=0, use_graph=use_graph)
                inputs = [W.nls_signal(d[0], seed=W.BASE_SEED + 70 + i).astype(np.complex64) for i, d in enumerate(dims)]
            for r, x in enumerate(inputs):
                plan.set_field(x, run=r)
            plan.step(3)       # off the segment grid: direct launches
            plan.step(2)
            plan.step(17)      # three whole segments (graph) and two single steps
            res = [(plan.get_spectrum(run=r), plan.get_mask(run=r), plan.get_stats(run=r)) for r in range(len(dims))]
            plan.close()
        side.synchronize()
        outs.append(res)
    for (sa, ma, ta), (sb, mb, tb) in zip(*outs):
        assert np.array_equal(sa, sb)
        assert np.array_equal(ma, mb)
        assert ta["step"] == tb["step"] == 22 and ta["assessments"] == tb["assessments"]


def test_autotune_mid_run_restores_half_form_state():
    """3-D 128^3 in the half-spectrum form, tuned after 15 steps (frozen blocks,
    a live-tile list for the paired z forward in force): the trial steps leave
    no trace (spectrum, mask and statistics bit for bit), and 12 more steps
    match an untuned half-form plan bit for bit when the half form is chosen
    (its update forms and graph replay agree bit for bit), else to rounding."""
    import torch
    from paper_2609_03922_gb300 import spdba
    dims = (128, 128, 128)
    c0 = W.ch_initial_condition(dims, mean=0.1, seed=W.BASE_SEED + 85).astype(np.float32)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        plan = spdba.Plan(dims, (8, 8, 8), threshold=1e-2, reassess=5, precision=0, half_spectrum=1)
        plan.set_field(c0)
        plan.step(15)
        before = (plan.get_spectrum(), plan.get_mask(), plan.get_stats())
        rep = plan.autotune(5)
        chosen = rep["candidates"][rep["chosen"]]
        after = (plan.get_spectrum(), plan.get_mask(), plan.get_stats())
        plan.step(12)
        tuned = (plan.get_spectrum(), plan.get_mask(), plan.get_stats())
        plan.close()
        ref = spdba.Plan(dims, (8, 8, 8), threshold=1e-2, reassess=5, precision=0, half_spectrum=1)
        ref.set_field(c0)
        ref.step(27)
        untuned = (ref.get_spectrum(), ref.get_mask(), ref.get_stats())
        ref.close()
    side.synchronize()
    assert np.any(before[1] == 0)
    assert np.array_equal(after[0], before[0]) and np.array_equal(after[1], before[1])
    assert after[2]["step"] == before[2]["step"] == 15
    assert after[2]["assessments"] == before[2]["assessments"]
    assert tuned[2]["step"] == untuned[2]["step"] == 27
    if chosen["half_spectrum"] == 1:
        assert np.array_equal(tuned[0], untuned[0]), chosen
        assert np.array_equal(tuned[1], untuned[1]), chosen
    else:
        assert O.rel_l2(tuned[0], untuned[0]) <= 1e-5, chosen


def test_autotune_restores_state_and_keeps_results():
    """The autotuner tries every launch configuration from the same state and
    leaves no trace: after it, the plan's step count, fields, masks and
    statistics evolve exactly as in an untuned plan."""
    import torch
    from paper_2609_03922_gb300 import spdba
    dims = [(128, 128), (192, 192)]
    inputs = [W.ch_initial_condition(d, mean=0.05, seed=W.BASE_SEED + 80 + i).astype(np.float32)
              for i, d in enumerate(dims)]
    outs = []
    for tune in (True, False):
        side = torch.cuda.Stream()
        with torch.cuda.stream(side):
            plan = spdba.Plan(None, (16, 16), threshold=1e-3, reassess=5, batch_dims=dims, precision=0)
            for r, x in enumerate(inputs):
                plan.set_field(x, run=r)
            if tune:
                rep = plan.autotune(10)
                assert rep["chosen"] in range(len(rep["candidates"]))
                assert {(c["fuse_update"], c["use_graph"]) for c in rep["candidates"]} == {(1, 1), (1, 0), (0, 1), (0, 0)}
                assert all(c["ms_per_step"] > 0 for c in rep["candidates"])
                assert plan.get_stats(run=0)["step"] == 0
            plan.step(23)
            res = [(plan.get_spectrum(run=r), plan.get_mask(run=r), plan.get_stats(run=r)) for r in range(len(dims))]
            plan.close()
        side.synchronize()
        outs.append(res)
    for (sa, ma, ta), (sb, mb, tb) in zip(*outs):
        assert np.array_equal(sa, sb)
        assert np.array_equal(ma, mb)
        assert ta["step"] == tb["step"] == 23 and ta["assessments"] == tb["assessments"]
        assert ta["active_ratio_sum"] == tb["active_ratio_sum"]


def test_tma_list_update_equals_warp_list_update():
    """The staged update moved by TMA boxes (3-D complex64, 8^3 blocks) gives the
    values of the per-warp list kernel bit for bit, through several state settings."""
    from paper_2609_03922_gb300 import spdba
    dims = (64, 64, 64)
    c0 = W.ch_initial_condition(dims, mean=0.1, seed=W.BASE_SEED + 44).astype(np.float32)
    outs = []
    for tma in (0, 1):
        with spdba.Plan(dims, (8, 8, 8), threshold=1e-3, reassess=4, precision=0, fuse_update=0,
                        tma_update=tma) as plan:
            plan.set_field(c0)
            plan.step(23)
            outs.append((plan.get_spectrum(), plan.get_mask(), plan.get_stats()))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])
    assert np.any(outs[0][1] == 0)
    assert outs[1][2]["active_ratio_sum"] == outs[0][2]["active_ratio_sum"]
