"""Pins of the oracle's dynamic threshold control (Supplementary S1.3).

The rule: with q = r / r_tar, q > 2 doubles the threshold and q < 0.5 halves
it; otherwise a deviation outside the relative deadband eta scales it by
1 + eta or 1 - eta; inside the deadband it stays.  Each check is followed by
one full-activation step.  The sequences below are traced by hand with
exactly representable numbers, so every comparison is exact.
"""
import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("r,expect", [
    (0.75, 2.0),        # q = 3: factor-of-two correction up
    (0.5, 1.25),        # q = 2 exactly: not "> 2", so 1 + eta
    (0.375, 1.25),      # q = 1.5: above the deadband
    (0.3125, 1.0),      # q = 1.25 = 1 + eta: deadband edge, kept
    (0.25, 1.0),        # on target
    (0.1875, 1.0),      # q = 0.75 = 1 - eta: deadband edge, kept
    (0.15625, 0.75),    # q = 0.625: below the deadband
    (0.125, 0.75),      # q = 0.5 exactly: not "< 0.5", so 1 - eta
    (0.0625, 0.5),      # q = 0.25: factor-of-two correction down
])
def test_threshold_control_branches(r, expect):
    assert O.threshold_control(1.0, r, 0.25, 0.25) == expect


def _cfg(**kw):
    c = O.CHConfig((16, 16), (4, 4), threshold=1.0, target_ratio=0.25, control_every=4, control_eta=0.25,
                   warmup_steps=2)
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def _drive(cfg, counts, nblocks=8):
    """Feed a controller a synthetic history of non-frozen block counts per step."""
    ctl = O.ThresholdController(cfg, nblocks)
    in_force = []
    for step, nf in enumerate(counts):
        in_force.append(ctl.begin_step(step))
        states = np.array([2] * nf + [0] * (nblocks - nf), dtype=np.uint8)
        ctl.end_step(step, states)
    return ctl, in_force


def test_controller_hand_traced_sequence():
    # steps 0, 1: warm-up (not counted); 4, 8, 12: control steps (not counted)
    counts = [8, 8, 4, 2, 8, 1, 1, 2, 8, 6, 6, 6, 8]
    ctl, in_force = _drive(_cfg(), counts)
    # step 4: r = (4 + 2) / (2 * 8) = 0.375, q = 1.5 -> x 1.25
    # step 8: r = (1 + 1 + 2) / (3 * 8) = 1/6, q = 2/3 < 0.75 -> x 0.75
    # step 12: r = (6 + 6 + 6) / (3 * 8) = 0.75, q = 3 -> x 2
    assert ctl.log == [(4, 1.25), (8, 0.9375), (12, 1.875)]
    assert in_force == [1.0] * 4 + [1.25] * 4 + [0.9375] * 4 + [1.875]


def test_controller_skips_refresh_steps_and_empty_intervals():
    # refresh every 3 steps: steps 3, 6, 9 are full-activation steps and do not count
    counts = [8, 8, 2, 8, 8, 2, 8, 2, 2]
    ctl, _ = _drive(_cfg(refresh_every=3), counts)
    # step 4: counted step 2 only: r = 2 / 8 = 0.25 -> kept (logged)
    # step 8: counted steps 5, 7: r = 4 / 16 = 0.25 -> kept
    assert ctl.log == [(4, 1.0), (8, 1.0)]
    # refresh on every step: no step is ever counted, so the control steps 4 and 8
    # see empty intervals and make no decision
    ctl, in_force = _drive(_cfg(refresh_every=1), [8, 1, 1, 1, 1, 1, 1, 1, 1, 1])
    assert ctl.log == [] and in_force == [1.0] * 10


def test_control_steps_are_full_activation_steps():
    """At a control step every block is updated: the step equals a Regular step bit for bit."""
    dims, block = (32, 32), (4, 4)
    rng = np.random.default_rng(3)
    c0 = 0.05 * (rng.random(dims) - 0.5)
    cfg = O.CHConfig(dims, block, threshold=0.5, reassess=2, target_ratio=0.2, control_every=4)
    k2 = O.k_squared(dims)
    ctl = O.ThresholdController(cfg, 64)
    c_hat, hist = O.run_ch(c0, cfg, 4, controller=ctl)
    states = hist[-1][1]
    assert np.count_nonzero(states == O.STATE_FROZEN) > 0      # the adaptive steps do skip blocks
    nxt, _ = O.run_ch(None, cfg, 1, start_step=4, c_hat=c_hat, states=states, controller=ctl)
    assert np.array_equal(nxt, O.ch_regular_step(c_hat, k2, cfg.dt, cfg.kappa))
    # and the step after it is adaptive again (differs from Regular)
    nxt2, _ = O.run_ch(None, cfg, 1, start_step=5, c_hat=nxt, states=states, controller=ctl)
    assert not np.array_equal(nxt2, O.ch_regular_step(nxt, k2, cfg.dt, cfg.kappa))


def test_run_threshold_follows_the_controller_fed_with_its_own_states():
    """The run's reassessments use the threshold the rule produced from the
    states the run itself had in force (integration order: decision before the
    step's reassessment, counting after the step)."""
    dims, block = (32, 32), (4, 4)
    rng = np.random.default_rng(7)
    c0 = 0.05 * (rng.random(dims) - 0.5)
    cfg = O.CHConfig(dims, block, threshold=1e-3, reassess=5, target_ratio=0.3, control_every=10,
                     control_eta=0.05)
    ctl = O.ThresholdController(cfg, 64)
    seen = {}

    def watch(step, c_hat, states, tau):
        seen[step] = (c_hat.copy(), tau)
    c_hat, hist = O.run_ch(c0, cfg, 60, controller=ctl, on_assess=watch)
    assert len(ctl.log) == 5
    # replay: states in force per step from the history, fed to a fresh controller
    by_step = dict((s, st) for s, st, _ in hist)
    replay = O.ThresholdController(cfg, 64)
    cur = None
    for step in range(60):
        replay.begin_step(step)
        cur = by_step.get(step, cur)
        replay.end_step(step, cur)
    assert replay.log == ctl.log
    # each reassessment at a decision step uses the new coefficient:
    # tau = threshold * max_{k != 0} |c_hat(k)| of that step's field
    for step, thr in ctl.log:
        q, tau = seen[step]
        assert tau == thr * np.sqrt(O.global_max_sq(q, exclude_dc=True))
    assert any(thr != 1e-3 for _, thr in ctl.log)


def test_control_drives_the_ratio_toward_the_target():
    """Property: after a few intervals the measured share sits within the x2 band of the target."""
    dims, block = (32, 32), (4, 4)
    rng = np.random.default_rng(11)
    c0 = 0.05 * (rng.random(dims) - 0.5)
    cfg = O.CHConfig(dims, block, threshold=1e-8, reassess=1, target_ratio=0.25, control_every=5,
                     control_eta=0.1)
    ctl = O.ThresholdController(cfg, 64)
    ratios = []

    def watch(step, c_hat, states, tau):
        ratios.append((step, np.count_nonzero(states) / states.size))
    O.run_ch(c0, cfg, 150, on_assess=watch, controller=ctl)
    assert ctl.log[0][1] > 1e-8          # starts far too low (everything active): raised
    late = [r for s, r in ratios if s >= 100]
    assert 0.125 <= np.mean(late) <= 0.5
