"""Parity at each configuration's stated scale, against the FP64 oracle.

- 512-signal NLS batch: a 32-signal seeded subset covering every length
  2^12..2^18, all 800 steps, in complex128 and complex64;
- uneven 2-D CH ensemble: every run of side <= 256 of the 64-run set, all
  1000 steps, inside the full 64-run grouped plan;
- 3-D CH with the learned predictor: K = 20, judge every J = 100, the full
  5000 steps at 64^3 (8^3 blocks), with a network trained on the method's own
  traces of other seeds.  Over 5000 complex64 steps the coarsening amplifies
  FP32 rounding past 1e-4 in any FP32 implementation; there the GPU must stay
  within 2x of an independent FP32 run (as for the NLS batch).
Masks are checked in lock-step at every state setting (the GPU's spectrum
promoted to FP64 through the oracle's classifier, tie band excepted); the
oracle then re-runs the steps in FP64 with the GPU's states in worker
processes (spawned), so the field error measures arithmetic only.  Each
result's error is printed.
"""
import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle as O
import workloads as W
import _oracle_jobs as J
from _helpers import states_within_tie_band

pytestmark = pytest.mark.gpu

NLS_COMPOSITION = {4096: 10, 8192: 8, 16384: 6, 32768: 4, 65536: 2, 131072: 1, 262144: 1}


@pytest.fixture(scope="module")
def pool():
    cores = os.cpu_count() or 4
    workers = max(1, min(8, cores // 4))
    ex = cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"),
                                initializer=J.init_worker, initargs=(max(1, cores // workers),))
    yield ex
    ex.shutdown()


def nls_subset():
    """(index in the seeded 512-signal set, length): the first signals of each length."""
    need = dict(NLS_COMPOSITION)
    picked = []
    for i, n in enumerate(W.nls_lengths(512)):
        if need.get(n, 0) > 0:
            picked.append((i, n))
            need[n] -= 1
    assert not any(need.values())
    return picked


def _nls_gpu(sub, precision, steps, R):
    from paper_2609_03922_gb300 import spdba
    cdt = np.complex64 if precision == 0 else np.complex128
    plan = spdba.Plan(None, (-64,), threshold=1e-6, reassess=R, batch_dims=[(n,) for _, n in sub],
                      model=spdba.SPDBA_MODEL_NLS, precision=precision)
    for r, (i, n) in enumerate(sub):
        # both precisions start from the complex64-rounded samples
        E0 = W.nls_signal(n, seed=W.BASE_SEED + 1 + i).astype(np.complex64).astype(cdt)
        plan.set_field(np.ascontiguousarray(E0), run=r)
    masks = [dict() for _ in sub]
    for s in range(steps):
        if s % R == 0:
            specs = [plan.get_spectrum(run=r) for r in range(len(sub))]
            plan.step(1)
            for r, (i, n) in enumerate(sub):
                m = plan.get_mask(run=r)
                cfg = O.NLSConfig(n, n // 64, threshold=1e-6, reassess=R)
                st, tau, meas = O.assess_states(specs[r].astype(np.complex128), cfg, exclude_dc=False)
                ok, nties = states_within_tie_band(m, meas, tau, cfg)
                assert ok, "signal %d (n=%d) step %d: states differ (%d tie-band blocks)" % (i, n, s, nties)
                masks[r][s] = m
        else:
            plan.step(1)
    fields = [plan.get_field(run=r) for r in range(len(sub))]
    plan.close()
    return masks, fields


def test_nls_config_subset_full_run(pool):
    steps, R = 800, 10
    sub = nls_subset()
    m128, f128 = _nls_gpu(sub, 1, steps, R)
    m64, f64 = _nls_gpu(sub, 0, steps, R)
    jobs = []
    for r, (i, n) in enumerate(sub):
        seed = W.BASE_SEED + 1 + i
        same = all(np.array_equal(m128[r][s], m64[r][s]) for s in m128[r])
        if same:
            jobs.append((r, pool.submit(J.nls_job, n, seed, steps, R, m128[r], {"c128": f128[r], "c64": f64[r]},
                                        True)))
        else:
            jobs.append((r, pool.submit(J.nls_job, n, seed, steps, R, m128[r], {"c128": f128[r]}, False)))
            jobs.append((r, pool.submit(J.nls_job, n, seed, steps, R, m64[r], {"c64": f64[r]}, True)))
    errs = {r: {} for r in range(len(sub))}
    floors = {}
    for r, f in jobs:
        e, fl = f.result()
        errs[r].update(e)
        if fl is not None:
            floors[r] = fl
    worst128, worst64 = 0.0, 0.0
    for r, (i, n) in enumerate(sub):
        e128, e64, fl = errs[r]["c128"], errs[r]["c64"], floors[r]
        print("NLS signal %3d n=%6d: rel-L2 c128 %.2e, c64 %.2e (FP32 floor %.2e)" % (i, n, e128, e64, fl))
        worst128 = max(worst128, e128)
        worst64 = max(worst64, e64 / max(fl, 1e-4))
        assert e128 <= 1e-4, "signal %d: c128 rel-L2 %.3e" % (i, e128)
        # complex64 meets 1e-4, or, where FP32 arithmetic itself leaves more
        # (modulation instability), stays within 2x of an independent FP32 run
        assert e64 <= max(1e-4, 2.0 * fl), "signal %d: c64 rel-L2 %.3e, FP32 floor %.3e" % (i, e64, fl)
    print("worst c128 rel-L2 %.2e; worst c64 / max(floor, 1e-4) %.2f" % (worst128, worst64))


def test_ensemble_runs_up_to_256_full_run(pool):
    from paper_2609_03922_gb300 import spdba
    members = W.ensemble_members(64)
    steps, R, block = 1000, 10, (16, 16)
    plan = spdba.Plan(None, block, threshold=1e-6, reassess=R, batch_dims=[(sd, sd) for sd, _, _ in members],
                      precision=spdba.SPDBA_C64)
    for r, (sd, m, seed) in enumerate(members):
        plan.set_field(W.ch_initial_condition((sd, sd), mean=m, seed=seed).astype(np.float32), run=r)
    check = [r for r, (sd, _, _) in enumerate(members) if sd <= 256]
    masks = {r: {} for r in check}
    for s in range(steps):
        if s % R == 0:
            specs = {r: plan.get_spectrum(run=r) for r in check}
            plan.step(1)
            for r in check:
                sd = members[r][0]
                mk = plan.get_mask(run=r)
                cfg = O.CHConfig((sd, sd), block, threshold=1e-6, reassess=R)
                st, tau, meas = O.assess_states(specs[r].astype(np.complex128), cfg, exclude_dc=True)
                ok, nties = states_within_tie_band(mk, meas, tau, cfg)
                assert ok, "run %d step %d: states differ (%d tie-band blocks)" % (r, s, nties)
                masks[r][s] = mk
        else:
            plan.step(1)
    fields = {r: plan.get_field(run=r) for r in check}
    plan.close()
    futs = {r: pool.submit(J.ch_job, (members[r][0],) * 2, block, members[r][1], members[r][2], steps, R, masks[r],
                           fields[r]) for r in check}
    worst = 0.0
    for r in check:
        e = futs[r].result()
        print("ensemble run %2d side %3d: rel-L2 %.2e" % (r, members[r][0], e))
        worst = max(worst, e)
        assert e <= 1e-4, "run %d: rel-L2 %.3e" % (r, e)
    print("ensemble: %d runs, worst rel-L2 %.2e" % (len(check), worst))


def test_predictor_config_full_run(pool):
    """The predictor-driven run against the oracle advanced with the same states."""
    import torch
    from paper_2609_03922_gb300 import spdba
    from paper_2609_03922_gb300 import predictor_train as PT
    dims, block, K, Jv, steps = (64, 64, 64), (8, 8, 8), 20, 100, 5000
    mp_ = tuple(d // b for d, b in zip(dims, block))
    traces = [PT.collect_trace(dims, block, W.ch_initial_condition(dims, mean=0.1, seed=W.BASE_SEED + 300 + i)
                               .astype(np.float32), 1000) for i in range(2)]
    pr = PT.TrainedPredictor(mp_, max_batch=4, seed=0)
    xs, ys = [], []
    for tr in traces:
        x, y = PT.make_inputs(pr, tr, PT.build_samples(tr, K, Jv))
        xs.append(x)
        ys.append(y)
    PT.train(pr, torch.cat(xs), torch.cat(ys), epochs=30, lr=3e-3)
    seed = W.BASE_SEED + 310
    c0 = W.ch_initial_condition(dims, mean=0.1, seed=seed).astype(np.float32)
    plan = spdba.Plan(dims, block, threshold=1e-6, reassess=10)
    plan.attach_predictor(pr, K, Jv, 0.5)
    plan.set_field(c0)
    masks = {}
    cfg = O.CHConfig(dims, block, threshold=1e-6, reassess=10)
    for t in range(0, steps, K):
        judge = t % Jv == 0
        spec = plan.get_spectrum() if judge else None
        plan.step(1)
        masks[t] = plan.get_mask()
        if judge:
            st, tau, meas = O.assess_states(spec.astype(np.complex128), cfg, exclude_dc=True)
            ok, nties = states_within_tie_band(masks[t], meas, tau, cfg)
            assert ok, "judge at step %d: states differ (%d tie-band blocks)" % (t, nties)
        plan.step(K - 1)
    f_pred = plan.get_field()
    s_pred = plan.get_stats()
    plan.close()
    fut = pool.submit(J.ch_job, dims, block, 0.1, seed, steps, K, masks, f_pred)
    fut_floor = pool.submit(J.ch_fp32_floor, dims, 0.1, seed, steps)
    f_exact = None
    with spdba.Plan(dims, block, threshold=1e-6, reassess=10) as ex:
        ex.set_field(c0)
        ex.step(steps)
        f_exact = ex.get_field()
    err = fut.result()
    floor = fut_floor.result()
    d = float(np.linalg.norm(f_pred.astype(np.float64) - f_exact) / np.linalg.norm(f_exact.astype(np.float64)))
    nb = int(np.prod(mp_))
    print("predictor 64^3, %d steps: rel-L2 vs oracle (same states) %.2e (FP32 floor %.2e); vs exact adaptive "
          "GPU run %.2e; exact scans %d, predictions %d, missed blocks %d" %
          (steps, err, floor, d, s_pred["assessments"] - s_pred["predictions"], s_pred["predictions"],
           s_pred["missed_blocks"]))
    # complex64 meets 1e-4, or, where FP32 arithmetic itself leaves more over the
    # 5000 steps (coarsening amplifies rounding), stays within 2x of an
    # independent FP32 implementation of the same steps
    assert err <= max(1e-4, 2.0 * floor)
    assert d <= 1e-5          # the predictor's own effect against the exact method
    assert s_pred["assessments"] - s_pred["predictions"] == steps // Jv
    assert s_pred["missed_blocks"] <= 0.05 * nb * (steps // Jv)
