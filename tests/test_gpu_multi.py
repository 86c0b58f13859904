"""The multi-size form of batched 2-D complex64 Cahn-Hilliard plans: each pass
phase of a step is one persistent launch whose CTAs drain a queue of every
group's tiles.  It runs the same per-tile arithmetic as the one-launch-per-group
form, so fields, block states and statistics must agree bit for bit with it
(the per-group form is itself checked against the oracle); one case also goes
to the oracle directly, in lock-step."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

# uneven ensemble: every side the multi-size kernels serve, 1-3 runs each
SIZES = [(64, 64), (128, 128), (128, 128), (192, 192), (256, 256), (256, 256), (384, 384), (512, 512)]


def _c0s(sizes, seed0):
    return [np.ascontiguousarray(W.ch_initial_condition(s, mean=0.12 * ((i % 3) - 1), seed=seed0 + i)
                                 .astype(np.float32)) for i, s in enumerate(sizes)]


def _run(sizes, c0s, steps, multi, threshold=1e-3, reassess=5, use_graph=1, chunk=None, **kw):
    import torch
    from paper_2609_03922_gb300 import spdba
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        plan = spdba.Plan(None, (16, 16), threshold=threshold, reassess=reassess, batch_dims=sizes, precision=0,
                          multi_pass=multi, use_graph=use_graph, **kw)
        cfg = plan.get_config()
        for r, c0 in enumerate(c0s):
            plan.set_field(c0, run=r)
        chunk = chunk or steps
        for _ in range(steps // chunk):
            plan.step(chunk)
        out = [(plan.get_spectrum(run=r), plan.get_mask(run=r), plan.get_stats(run=r)) for r in range(len(sizes))]
        plan.close()
    return out, cfg


def _same(a, b):
    for (sa, ma, ta), (sb, mb, tb) in zip(a, b):
        assert np.array_equal(sa, sb)
        assert np.array_equal(ma, mb)
        for k in ("step", "assessments", "n_active", "n_transition", "active_ratio_sum", "tau", "max_amp"):
            assert ta[k] == tb[k], k
        # mass: each thread sums its tile's values of c in FP32 before the FP64
        # reduction, and the tile widths differ between the forms; |c| < 2, at most
        # 32 values a thread: |error| <= 2 * 32 * 2^-24 * points
        assert abs(ta["mass"] - tb["mass"]) <= 64 * 2.0 ** -24 * sa.size


@pytest.mark.parametrize("multi", [1, 2])
def test_multi_size_launches_equal_per_group_launches(multi):
    c0s = _c0s(SIZES, W.BASE_SEED + 300)
    ref, cfg0 = _run(SIZES, c0s, 40, 0)
    got, cfg = _run(SIZES, c0s, 40, multi)
    assert cfg0["multi_pass"] == 0 and cfg["multi_pass"] == multi
    # some blocks were frozen (the update skipped tiles) and some were not
    assert any(np.any(m == O.STATE_FROZEN) for _, m, _ in got)
    assert any(np.any(m != O.STATE_FROZEN) for _, m, _ in got)
    _same(got, ref)


def test_multi_size_graph_replay_and_direct_launches_agree():
    """Replayed reassessment segments (graphs) and direct launches; the queue
    counters return to zero after every launch, so replays see a full queue."""
    sizes = SIZES[:5]
    c0s = _c0s(sizes, W.BASE_SEED + 320)
    a, _ = _run(sizes, c0s, 60, 1, use_graph=1, chunk=20)
    b, _ = _run(sizes, c0s, 60, 1, use_graph=0, chunk=1)
    c, _ = _run(sizes, c0s, 60, 0, use_graph=0, chunk=1)
    _same(a, b)
    _same(a, c)


def test_multi_size_dense_and_regular_steps():
    """Regular mode (every step dense) and threshold 0 (everything ACTIVE) in the
    multi-size form equal the per-group form."""
    sizes = SIZES[:4]
    c0s = _c0s(sizes, W.BASE_SEED + 340)
    _same(_run(sizes, c0s, 12, 1, mode=0)[0], _run(sizes, c0s, 12, 0, mode=0)[0])
    _same(_run(sizes, c0s, 12, 2, threshold=0.0)[0], _run(sizes, c0s, 12, 0, threshold=0.0)[0])


def test_multi_size_against_oracle_lockstep():
    """Three sizes in one plan, multi-size form: every run against the FP64
    oracle advanced with the GPU's block states."""
    from paper_2609_03922_gb300 import spdba
    sizes = [(64, 64), (192, 192), (128, 128)]
    c0s = _c0s(sizes, W.BASE_SEED + 360)
    plan = spdba.Plan(None, (16, 16), threshold=1e-4, reassess=5, batch_dims=sizes, precision=0, multi_pass=1,
                      use_graph=0)
    assert plan.get_config()["multi_pass"] == 1
    for r, c0 in enumerate(c0s):
        plan.set_field(c0, run=r)
    steps = 30
    masks = [dict() for _ in sizes]
    for s in range(steps):
        plan.step(1)
        if s % 5 == 0:
            for r in range(len(sizes)):
                masks[r][s] = plan.get_mask(run=r)
    for r, (dims, c0) in enumerate(zip(sizes, c0s)):
        got = plan.get_field(run=r)
        cfg = O.CHConfig(dims, (16, 16), threshold=1e-4, reassess=5)
        ref_hat, _ = O.run_ch(c0.astype(np.float64), cfg, steps, on_assess=lambda n, ch, st, tau, r=r: masks[r][n])
        assert O.rel_l2(got, O.ch_real_field(ref_hat)) <= 1e-5
    plan.close()


def test_multi_size_form_only_where_it_applies():
    from paper_2609_03922_gb300 import spdba
    cases = [
        dict(dims=None, batch_dims=[(64, 64), (128, 128)], precision=1),         # complex128
        dict(dims=None, batch_dims=[(64, 64), (128, 128)], fuse_update=0),       # staged update
        dict(dims=None, batch_dims=[(128, 128), (128, 128)]),                    # one group
        dict(dims=(64, 64, 64), batch_dims=None),                                # 3-D
        dict(dims=None, batch_dims=[(32, 32), (64, 64)]),                        # 32 has no multi-size kernel
    ]
    for c in cases:
        dims, bd = c.pop("dims"), c.pop("batch_dims")
        block = (8, 8, 8) if dims is not None and len(dims) == 3 else (16, 16)
        with spdba.Plan(dims, block, batch_dims=bd, multi_pass=1, **c) as pl:
            assert pl.get_config()["multi_pass"] == 0, c
    with pytest.raises(spdba.SpdbaError):
        spdba.Plan(None, (16, 16), batch_dims=[(64, 64), (128, 128)], multi_pass=3)


def test_autotune_offers_multi_size_form_and_caches_its_choice():
    from paper_2609_03922_gb300 import spdba
    sizes = [(128, 128), (256, 256), (256, 256), (512, 512)]
    c0s = _c0s(sizes, W.BASE_SEED + 380)
    spdba.tune_cache_clear()

    def plan():
        p = spdba.Plan(None, (16, 16), threshold=1e-3, reassess=5, batch_dims=sizes, precision=0)
        for r, c0 in enumerate(c0s):
            p.set_field(c0, run=r)
        return p

    import torch
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        p1 = plan()
        p1.step(10)
        rep = p1.autotune(5)
        assert rep["cached"] == 0
        assert {c["multi_pass"] for c in rep["candidates"]} == {0, 1, 2}
        chosen = rep["candidates"][rep["chosen"]]
        cfg1 = p1.get_config()
        assert cfg1["multi_pass"] == chosen["multi_pass"] and cfg1["use_graph"] == chosen["use_graph"]
        p1.step(10)
        f1 = [p1.get_spectrum(run=r) for r in range(len(sizes))]
        p1.close()
        # same signature: the stored choice, no timing
        p2 = plan()
        p2.step(10)
        rep2 = p2.autotune(5, cached=True)
        assert rep2["cached"] == 1 and rep2["candidates"][0]["multi_pass"] == chosen["multi_pass"]
        assert p2.get_config()["multi_pass"] == cfg1["multi_pass"]
        p2.step(10)
        # the tuning (timed or cached) leaves no trace in the results
        for r in range(len(sizes)):
            assert np.array_equal(p2.get_spectrum(run=r), f1[r])
        p2.close()
        spdba.tune_cache_clear()
        p3 = plan()
        assert p3.autotune(2, cached=True)["cached"] == 0
        p3.close()
