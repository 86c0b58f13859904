"""The Hermitian half-spectrum form of 3-D complex64 Cahn-Hilliard steps
(transforms on x frequencies 0 .. N2/2 of the Hermitian part of c_hat) against
the full complex transforms and against the oracle.  c = Re(IFFT(c_hat)) is
exactly the inverse transform of (c_hat(k) + conj(c_hat(-k))) / 2, so both
forms compute the method's step; they differ by rounding only."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from _helpers import states_within_tie_band

pytestmark = pytest.mark.gpu


def _run(dims, steps, c0, **kw):
    from paper_2609_03922_gb300 import spdba
    plan = spdba.Plan(dims, (8, 8, 8), threshold=kw.pop("threshold", 1e-6), reassess=kw.pop("reassess", 5),
                      precision=0, **kw)
    plan.set_field(np.ascontiguousarray(c0.astype(np.float32)))
    masks = {}
    for s in range(steps):
        plan.step(1)
        if s % 5 == 0:
            masks[s] = plan.get_mask()
    out = (plan.get_field().astype(np.float64), plan.get_spectrum(), masks, plan.get_stats())
    plan.close()
    return out


@pytest.mark.parametrize("side", [128, 256])
def test_half_matches_full_transforms(side):
    dims = (side,) * 3
    c0 = W.ch_initial_condition(dims, mean=0.1, seed=W.BASE_SEED + 120)
    fh, _, mh, sh = _run(dims, 12, c0, half_spectrum=1)
    ff, _, mf, sf = _run(dims, 12, c0, half_spectrum=0)
    assert O.rel_l2(fh, ff) <= 2e-6
    for s in mh:
        assert np.mean(mh[s] != mf[s]) <= 1e-3          # tie-band flips only
    assert abs(sh["mass"] - sf["mass"]) <= 1e-6 * abs(sf["mass"])


def test_half_one_step_and_masks_against_oracle():
    """One reassessment step at 128^3 in the half form: the GPU's states through
    the oracle's classifier, and the field against the FP64 oracle."""
    dims = (128,) * 3
    c0 = W.ch_initial_condition(dims, mean=0.1, seed=W.BASE_SEED + 121)
    from paper_2609_03922_gb300 import spdba
    plan = spdba.Plan(dims, (8, 8, 8), threshold=1e-6, reassess=10, precision=0, half_spectrum=1)
    plan.set_field(np.ascontiguousarray(c0.astype(np.float32)))
    spec0 = plan.get_spectrum()
    plan.step(1)
    mask = plan.get_mask()
    field = plan.get_field()
    plan.close()
    cfg = O.CHConfig(dims, (8, 8, 8), threshold=1e-6, reassess=10)
    st, tau, meas = O.assess_states(spec0.astype(np.complex128), cfg, exclude_dc=True)
    ok, _ = states_within_tie_band(mask, meas, tau, cfg)
    assert ok
    ref_hat, _ = O.run_ch(c0.astype(np.float32).astype(np.float64), cfg, 1, on_assess=lambda n, ch, s_, t_: mask)
    assert O.rel_l2(field, O.ch_real_field(ref_hat)) <= 1e-5


def test_half_fused_equals_staged():
    dims = (128,) * 3
    c0 = W.ch_initial_condition(dims, mean=0.1, seed=W.BASE_SEED + 122)
    a = _run(dims, 11, c0, half_spectrum=1, fuse_update=1, threshold=1e-2)
    b = _run(dims, 11, c0, half_spectrum=1, fuse_update=0, threshold=1e-2)
    assert np.array_equal(a[1], b[1])
    assert any(np.any(m == 0) for m in a[2].values())


def test_half_threshold_zero_equals_regular():
    dims = (128,) * 3
    c0 = W.ch_initial_condition(dims, mean=0.0, seed=W.BASE_SEED + 123)
    a = _run(dims, 7, c0, half_spectrum=1, threshold=0.0, reassess=3)
    b = _run(dims, 7, c0, half_spectrum=1, mode=0)
    assert np.array_equal(a[1], b[1])
    assert all(np.all(m == 2) for m in a[2].values())


# Shapes for the z forward pass of the half form: one transform per half pencil
# serving x frequencies kx and N2 - kx (z lengths 64, 128, 256, with one or
# several tiles of the column N2/2), and z length 384, which takes one
# transform per full pencil.
SHAPES = [(64, 256, 64), (128, 256, 128), (256, 128, 256), (256, 256, 64), (384, 128, 128)]


@pytest.mark.parametrize("dims", SHAPES)
def test_half_shapes_have_half_kernels(dims):
    """Every shape of this set runs in the half form (the autotuner offers it)."""
    from paper_2609_03922_gb300 import spdba
    plan = spdba.Plan(dims, (8, 8, 8), threshold=3e-3, reassess=10, precision=0, half_spectrum=1)
    plan.set_field(np.zeros(dims, dtype=np.float32))
    rep = plan.autotune(1)
    plan.close()
    assert any(c["half_spectrum"] == 1 for c in rep["candidates"])


@pytest.mark.parametrize("fuse", [1, 0])
@pytest.mark.parametrize("dims", SHAPES)
def test_half_shapes_against_oracle(dims, fuse):
    """Three steps with reassessments at steps 0 and 2: the second assessment,
    after the stiff damping of the high modes, mixes FROZEN, TRANSITION and
    ACTIVE blocks.  Both GPU assessments against the oracle's classifier, the
    field against the FP64 oracle advanced with the GPU's states; the update
    fused into the z forward pass and staged after the (paired) z forward."""
    c0 = W.ch_initial_condition(dims, mean=0.1, seed=W.BASE_SEED + 124)
    from paper_2609_03922_gb300 import spdba
    plan = spdba.Plan(dims, (8, 8, 8), threshold=0.1, reassess=2, precision=0, half_spectrum=1, fuse_update=fuse)
    plan.set_field(np.ascontiguousarray(c0.astype(np.float32)))
    plan.step(1)
    masks = {0: plan.get_mask()}
    plan.step(2)
    masks[2] = plan.get_mask()
    field = plan.get_field()
    plan.close()
    assert {0, 1, 2} <= set(np.unique(masks[2]).tolist())
    cfg = O.CHConfig(dims, (8, 8, 8), threshold=0.1, reassess=2)
    checked = []

    def on_assess(n, ch, st, tau):
        _, _, meas = O.assess_states(ch, cfg, exclude_dc=True)
        checked.append(states_within_tie_band(masks[n], meas, tau, cfg)[0])
        return masks[n]

    ref_hat, _ = O.run_ch(c0.astype(np.float32).astype(np.float64), cfg, 3, on_assess=on_assess)
    assert checked == [True, True]
    assert O.rel_l2(field, O.ch_real_field(ref_hat)) <= 1e-5


@pytest.mark.parametrize("dims", SHAPES)
def test_half_shapes_match_full_transforms(dims):
    c0 = W.ch_initial_condition(dims, mean=0.1, seed=W.BASE_SEED + 125)
    fh, sph, mh, _ = _run(dims, 8, c0, half_spectrum=1, threshold=0.1, reassess=2)
    ff, spf, mf, _ = _run(dims, 8, c0, half_spectrum=0, threshold=0.1, reassess=2)
    assert any(np.any(m == 0) for m in mh.values())
    assert O.rel_l2(fh, ff) <= 2e-6
    assert O.rel_l2(sph, spf) <= 2e-6


TMA_SHAPES = SHAPES + [(512, 128, 128), (256, 256, 256)]


@pytest.mark.parametrize("dims", TMA_SHAPES)
def test_tma_z_inverse_equals_cp_async_z_inverse(dims):
    """The half form's z inverse with its direct and mirror tiles moved as TMA
    boxes (where the x rows are whole tiles) gives the cp.async kernel's
    values bit for bit, over steps with frozen, transition and active blocks."""
    c0 = W.ch_initial_condition(dims, mean=0.1, seed=W.BASE_SEED + 126)
    from paper_2609_03922_gb300 import spdba
    out, used = [], []
    for tma in (1, 0):
        plan = spdba.Plan(dims, (8, 8, 8), threshold=0.1, reassess=2, precision=0, half_spectrum=1, fuse_update=0,
                          tma_passes=tma)
        used.append(plan.get_config()["tma_passes"])
        plan.set_field(np.ascontiguousarray(c0.astype(np.float32)))
        plan.step(7)
        out.append((plan.get_spectrum(), plan.get_mask(), plan.get_stats()))
        plan.close()
    assert used[1] == 0
    # x rows of whole tiles: every shape here but the two whose rows (48 and 80
    # entries) are not multiples of the z tile (64 and 32 pencils)
    assert used[0] == (0 if dims in [(64, 256, 64), (128, 256, 128)] else 1)
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert out[0][2]["n_active"] == out[1][2]["n_active"]
