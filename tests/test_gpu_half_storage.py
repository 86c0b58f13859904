"""Half-spectrum storage of 3-D complex64 Cahn-Hilliard runs (S1.2, Eq. S.4):
the spectrum of the real field kept as its half kx = 0 .. N2/2, block states
on the half map with neighbours in the omitted half activated through their
conjugate counterparts, every transform and the update on the stored half.
Checked against the oracle's half-spectrum form (run_ch_half) in lock-step,
and the launch forms against one another bit for bit."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from _helpers import states_within_tie_band

pytestmark = pytest.mark.gpu

B = (8, 8, 8)
SHAPES = [(64, 64, 64), (128, 64, 128), (64, 128, 256), (256, 128, 64)]


def _plan(dims, **kw):
    from paper_2609_03922_gb300 import spdba
    return spdba.Plan(dims, B, threshold=kw.pop("threshold", 0.1), reassess=kw.pop("reassess", 2), precision=0,
                      half_storage=1, **kw)


def _f32(c0):
    return np.ascontiguousarray(c0.astype(np.float32))


def _run(dims, steps, c0, **kw):
    plan = _plan(dims, **kw)
    assert plan.get_config()["half_storage"] == 1
    plan.set_field(_f32(c0))
    masks = {}
    for s in range(steps):
        plan.step(1)
        if s % plan_reassess(kw) == 0:
            masks[s] = plan.get_mask()
    out = (plan.get_field().astype(np.float64), plan.get_spectrum(), masks, plan.get_stats())
    plan.close()
    return out


def plan_reassess(kw):
    return kw.get("reassess", 2)


@pytest.mark.parametrize("fuse", [1, 0])
@pytest.mark.parametrize("dims", SHAPES)
def test_half_storage_against_oracle(dims, fuse):
    """Three steps, reassessments at steps 0 and 2 (the second mixes FROZEN,
    TRANSITION and ACTIVE blocks): the GPU's half-map states against the
    oracle's half-map classifier, the stored half and the field against the
    FP64 oracle advanced with the GPU's states; update fused and staged."""
    c0 = W.ch_initial_condition(dims, mean=0.1, seed=W.BASE_SEED + 700)
    plan = _plan(dims, fuse_update=fuse)
    plan.set_field(_f32(c0))
    spec0 = plan.get_spectrum()
    assert spec0.shape == dims[:2] + (dims[2] // 2 + 1,)
    ref0 = O.rfftn_half(c0.astype(np.float32).astype(np.float64))
    assert O.rel_l2(spec0, ref0) <= 2e-6
    plan.step(1)
    masks = {0: plan.get_mask()}
    plan.step(2)
    masks[2] = plan.get_mask()
    field = plan.get_field()
    spec = plan.get_spectrum()
    plan.close()
    assert masks[2].shape == O.half_block_counts(dims, B)
    assert {0, 1, 2} <= set(np.unique(masks[2]).tolist())
    cfg = O.CHConfig(dims, B, threshold=0.1, reassess=2)
    checked = []

    def on_assess(n, h, st, tau):
        _, _, meas = O.assess_states_half(h, cfg, exclude_dc=True)
        checked.append(states_within_tie_band(masks[n], meas, tau, cfg, classifier=O.classify_half)[0])
        return masks[n]

    ref_h, _ = O.run_ch_half(c0.astype(np.float32).astype(np.float64), cfg, 3, on_assess=on_assess)
    assert checked == [True, True]
    assert O.rel_l2(field, O.ch_real_field_half(ref_h, dims)) <= 1e-5
    assert O.rel_l2(spec, ref_h) <= 1e-5


def test_half_storage_lockstep_many_steps():
    """64^3 over 40 steps (eight reassessments, blocks freezing as the high modes
    decay) in lock-step with the oracle's half form."""
    dims = (64, 64, 64)
    c0 = W.ch_initial_condition(dims, mean=0.1, seed=W.BASE_SEED + 701)
    f, spec, masks, st = _run(dims, 40, c0, threshold=1e-3, reassess=5)
    cfg = O.CHConfig(dims, B, threshold=1e-3, reassess=5)
    checked = []

    def on_assess(n, h, s_, tau):
        _, _, meas = O.assess_states_half(h, cfg, exclude_dc=True)
        checked.append(states_within_tie_band(masks[n], meas, tau, cfg, classifier=O.classify_half)[0])
        return masks[n]

    ref_h, _ = O.run_ch_half(c0.astype(np.float32).astype(np.float64), cfg, 40, on_assess=on_assess)
    assert checked == [True] * 8
    assert any(np.count_nonzero(m == O.STATE_FROZEN) > 0 for m in masks.values())
    assert O.rel_l2(f, O.ch_real_field_half(ref_h, dims)) <= 1e-5
    # the statistics count the half map's live blocks only
    nb = int(np.prod(O.half_block_counts(dims, B)))
    assert st["nblocks"] == nb
    last = masks[35]
    assert st["n_active"] == np.count_nonzero(last == O.STATE_ACTIVE)
    assert st["n_transition"] == np.count_nonzero(last == O.STATE_TRANSITION)


@pytest.mark.parametrize("tma", [0, 1])
def test_half_storage_fused_equals_staged(tma):
    dims = (128, 128, 128)
    c0 = W.ch_initial_condition(dims, mean=0.1, seed=W.BASE_SEED + 702)
    a = _run(dims, 11, c0, fuse_update=1, threshold=1e-2)
    b = _run(dims, 11, c0, fuse_update=0, tma_update=tma, threshold=1e-2)
    assert np.array_equal(a[1], b[1])
    assert all(np.array_equal(a[2][s], b[2][s]) for s in a[2])
    assert any(np.any(m == O.STATE_FROZEN) for m in a[2].values())


def test_half_storage_threshold_zero_equals_regular():
    dims = (128, 64, 128)
    c0 = W.ch_initial_condition(dims, mean=0.0, seed=W.BASE_SEED + 703)
    a = _run(dims, 7, c0, threshold=0.0, reassess=3)
    b = _run(dims, 7, c0, mode=0)
    assert np.array_equal(a[1], b[1])
    assert all(np.all(m == O.STATE_ACTIVE) for m in a[2].values())


def test_half_storage_regular_matches_full_storage():
    """Regular steps need no block states: the stored half and the full spectrum
    give the same field up to FP32 rounding."""
    from paper_2609_03922_gb300 import spdba
    dims = (128, 128, 128)
    c0 = W.ch_initial_condition(dims, mean=0.1, seed=W.BASE_SEED + 704)
    fh = _run(dims, 10, c0, mode=0)[0]
    plan = spdba.Plan(dims, B, threshold=0.1, reassess=2, precision=0, mode=0)
    plan.set_field(_f32(c0))
    plan.step(10)
    ff = plan.get_field().astype(np.float64)
    plan.close()
    assert O.rel_l2(fh, ff) <= 2e-6


def test_half_storage_spectrum_round_trip_and_activity_shape():
    dims = (64, 64, 128)
    plan = _plan(dims)
    r = np.random.default_rng(5)
    shape = (64, 64, 65)
    h = (r.standard_normal(shape) + 1j * r.standard_normal(shape)).astype(np.complex64)
    plan.set_spectrum(h)
    assert np.array_equal(plan.get_spectrum(), h)
    plan.step(1)
    mx, tau = plan.get_activity()
    assert mx.shape == O.half_block_counts(dims, B)
    # the GPU's exact FP64 block maxima of the stored half it started from
    ref, _ = O.half_block_measures(h.astype(np.complex128), dims, B)
    assert np.array_equal(mx, ref)
    plan.close()


def test_half_storage_graph_replay_equals_direct_launches():
    dims = (64, 128, 64)
    c0 = W.ch_initial_condition(dims, mean=-0.1, seed=W.BASE_SEED + 705)
    out = []
    for graph in (1, 0):
        import torch
        side = torch.cuda.Stream()
        with torch.cuda.stream(side):
            plan = _plan(dims, threshold=1e-2, reassess=5, use_graph=graph)
            plan.set_field(_f32(c0))
            plan.step(30)
            out.append((plan.get_spectrum(), plan.get_mask()))
            plan.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_half_storage_where_it_applies():
    from paper_2609_03922_gb300 import spdba
    with pytest.raises(spdba.SpdbaError):
        spdba.Plan((64, 64), (8, 8), half_storage=1)                       # 2-D
    with pytest.raises(spdba.SpdbaError):
        spdba.Plan((64, 64, 24), B, half_storage=1)                        # 2 B does not divide 24
    with pytest.raises(spdba.SpdbaError):
        spdba.Plan((64, 64, 64), B, half_storage=1, precision=1)           # complex128
    with spdba.Plan((64, 64, 64), B) as p:
        assert p.get_config()["half_storage"] == 0


def test_half_storage_threshold_control_lockstep():
    """Dynamic threshold control (S1.3) with half-spectrum storage: the ratio of
    non-frozen blocks is counted over the half map's live blocks, so the GPU's
    coefficient sequence equals the oracle controller's (fed the GPU's states)
    bit for bit; states through the oracle's half-map classifier, the field
    against the oracle's half form run with the GPU's states."""
    dims = (64, 64, 64)
    steps, R = 240, 5
    kw = dict(target_ratio=0.2, control_every=20, control_eta=0.05)
    c0 = _f32(W.ch_initial_condition(dims, mean=0.1, seed=W.BASE_SEED + 706))
    cfg = O.CHConfig(dims, B, threshold=1e-6, reassess=R, **kw)
    masks, spectra, coef = {}, {}, {}
    plan = _plan(dims, threshold=1e-6, reassess=R, **kw)
    plan.set_field(c0)
    for s in range(steps):
        if s % R == 0:
            spectra[s] = plan.get_spectrum()
            plan.step(1)
            masks[s] = plan.get_mask()
            coef[s] = plan.get_stats()["threshold"]
        else:
            plan.step(1)
    field = plan.get_field()
    stats = plan.get_stats()
    plan.close()
    nb = int(np.prod(O.half_block_counts(dims, B)))
    assert stats["nblocks"] == nb
    ctl = O.ThresholdController(cfg, nb)
    cur = None
    for s in range(steps):
        thr = ctl.begin_step(s)
        if s in masks:
            assert coef[s] == thr, "step %d: GPU coefficient %.17g, oracle %.17g" % (s, coef[s], thr)
            _, tau, meas = O.assess_states_half(spectra[s].astype(np.complex128), cfg, exclude_dc=True,
                                                threshold=thr)
            ok, nties = states_within_tie_band(masks[s], meas, tau, cfg, classifier=O.classify_half)
            assert ok, "step %d: GPU states differ from the oracle's (%d tie-band blocks)" % (s, nties)
            cur = masks[s]
        ctl.end_step(s, cur)
    assert stats["controls"] == len(ctl.log) == steps // 20 - 1
    assert stats["threshold"] == ctl.threshold and ctl.threshold > 1e-6
    ref_h, _ = O.run_ch_half(c0.astype(np.float64), cfg, steps, on_assess=lambda n, h, st, tau: masks.get(n))
    assert O.rel_l2(field, O.ch_real_field_half(ref_h, dims)) <= 2e-5


@pytest.mark.parametrize("hs", [1, 0])
def test_autotune_between_reassessments_keeps_results(hs):
    """Tuned at step 17 with R = 5 (between reassessments, blocks frozen): the
    trial steps pass a reassessment, so the forward passes' pencil and column
    liveness must come back with the snapshot's states.  The next steps equal an
    untuned plan's bit for bit (every candidate of these forms gives the same
    values: fused, staged, TMA staged, graph replay, direct launches)."""
    import torch
    from paper_2609_03922_gb300 import spdba
    dims = (128, 128, 128)
    c0 = _f32(W.ch_initial_condition(dims, mean=0.1, seed=W.BASE_SEED + 707))
    kw = dict(threshold=1e-2, reassess=5, precision=0)
    if hs:
        kw["half_storage"] = 1
    else:
        kw["half_spectrum"] = 1
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        plan = spdba.Plan(dims, B, **kw)
        plan.set_field(c0)
        plan.step(17)
        before = (plan.get_spectrum(), plan.get_mask())
        rep = plan.autotune(4)
        after = (plan.get_spectrum(), plan.get_mask())
        plan.step(13)
        tuned = (plan.get_spectrum(), plan.get_mask())
        chosen = rep["candidates"][rep["chosen"]]
        plan.close()
        ref = spdba.Plan(dims, B, **kw)
        ref.set_field(c0)
        ref.step(30)
        untuned = (ref.get_spectrum(), ref.get_mask())
        ref.close()
    side.synchronize()
    assert np.any(before[1] == O.STATE_FROZEN)
    assert np.array_equal(after[0], before[0]) and np.array_equal(after[1], before[1])
    if hs or chosen["half_spectrum"] == 1:
        assert np.array_equal(tuned[0], untuned[0]), chosen
        assert np.array_equal(tuned[1], untuned[1]), chosen
    else:
        assert O.rel_l2(tuned[0], untuned[0]) <= 1e-5, chosen
