"""Out-of-memory path, injected on the host (no GPU fault, no real exhaustion).

spdba_debug_fail_alloc(k) makes the k-th device allocation of the library
fail as cudaMalloc would when the device is full.  Every allocation a plan
creation makes is failed in turn: the creation must return SPDBA_ERR_OOM with
a message naming the allocation, free everything it had allocated, and leave
the process able to create, step and destroy a fresh plan.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _create(L, spdba, dims, block, **kw):
    o = spdba.options_default()
    for k, v in kw.items():
        setattr(o, k, v)
    p = ctypes.c_void_p()
    d = (ctypes.c_int64 * len(dims))(*dims)
    b = (ctypes.c_int32 * len(block))(*block)
    st = L.spdba_plan_create(ctypes.byref(p), len(dims), d, b, 1e-6, 10, ctypes.byref(o))
    return st, p


@pytest.mark.parametrize("dims,block,prec", [((32, 32, 32), (8, 8, 8), 0), ((64, 64), (16, 16), 1)])
def test_every_failed_allocation_returns_oom_and_frees_everything(dims, block, prec):
    import torch
    from paper_2609_03922_gb300 import spdba
    import workloads as W
    torch.cuda.set_device(0)
    L = spdba.lib()
    L.spdba_debug_fail_alloc(0)
    live0 = L.spdba_debug_live_allocs()
    st, p = _create(L, spdba, dims, block, precision=prec)
    assert st == spdba.SPDBA_OK, L.spdba_last_error()
    n_alloc = L.spdba_debug_live_allocs() - live0
    assert n_alloc > 5
    L.spdba_plan_destroy(p)
    assert L.spdba_debug_live_allocs() == live0
    for k in range(1, n_alloc + 1):
        L.spdba_debug_fail_alloc(k)
        st, p = _create(L, spdba, dims, block, precision=prec)
        assert st == spdba.SPDBA_ERR_OOM, (k, st, L.spdba_last_error())
        assert b"device allocation" in L.spdba_last_error()
        assert not p.value
        assert L.spdba_debug_live_allocs() == live0, "allocation %d leaked buffers" % k
    # the injection ended with the failing allocation: a fresh plan works
    L.spdba_debug_fail_alloc(0)
    c0 = W.ch_initial_condition(dims, mean=0.0, seed=W.BASE_SEED)
    with spdba.Plan(dims, block, threshold=1e-6, reassess=10, precision=prec) as pl:
        pl.set_field(np.ascontiguousarray(c0, dtype=np.float32 if prec == 0 else np.float64))
        pl.step(3)
        out = pl.get_field()
    assert np.all(np.isfinite(out))
    assert L.spdba_debug_live_allocs() == live0


def test_failed_autotune_snapshot_leaves_the_plan_usable():
    import torch
    from paper_2609_03922_gb300 import spdba
    import workloads as W
    torch.cuda.set_device(0)
    L = spdba.lib()
    dims = (32, 32, 32)
    c0 = W.ch_initial_condition(dims, mean=0.1, seed=W.BASE_SEED).astype(np.float32)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        with spdba.Plan(dims, (8, 8, 8), threshold=1e-6, reassess=10, precision=spdba.SPDBA_C64) as pl:
            pl.set_field(c0)
            pl.step(10)
            live = L.spdba_debug_live_allocs()
            L.spdba_debug_fail_alloc(3)     # the third buffer of the tuner's snapshot
            with pytest.raises(spdba.SpdbaError) as ei:
                pl.autotune(10)
            assert ei.value.status == spdba.SPDBA_ERR_OOM
            L.spdba_debug_fail_alloc(0)
            assert L.spdba_debug_live_allocs() == live
            pl.step(10)
            assert np.all(np.isfinite(pl.get_field()))


@pytest.mark.parametrize("kind", ["z_inverse", "list_update"])
def test_tma_wait_timeout_is_reported_and_the_context_stays_usable(kind):
    """The TMA kernels' mbarrier waits are bounded.  With the first wait of every
    CTA pointed at a barrier nothing arrives on (a host switch), the wait runs
    out after its limit, the kernel counts the timeout, lets its real copies
    land and returns; spdba_get_stats then reports SPDBA_ERR_TIMEOUT.  The
    context stays usable: with the switch off a new plan steps and its results
    equal those of a plan that never saw a timeout."""
    import workloads as W
    from paper_2609_03922_gb300 import spdba
    lib = spdba.lib()
    if kind == "z_inverse":
        dims, kw = (128, 128, 128), dict(half_spectrum=1, tma_passes=1)
        key = "tma_passes"
    else:
        dims, kw = (64, 64, 64), dict(half_spectrum=0, tma_update=1)
        key = "tma_update"
    c0 = W.ch_initial_condition(dims, mean=0.1, seed=W.BASE_SEED + 7).astype(np.float32)

    def run(steps):
        with spdba.Plan(dims, (8, 8, 8), threshold=1e-2, reassess=2, precision=0, fuse_update=0, use_graph=0,
                        **kw) as pl:
            assert pl.get_config()[key] == 1
            pl.set_field(c0)
            pl.step(steps)
            pl.sync()
            try:
                return pl.get_stats(), pl.get_spectrum(), None
            except spdba.SpdbaError as e:
                return None, None, e

    try:
        lib.spdba_debug_set_wait_limit(64)
        lib.spdba_debug_stall_waits(1)
        _, _, err = run(3)
        assert err is not None and err.status == spdba.SPDBA_ERR_TIMEOUT
    finally:
        lib.spdba_debug_stall_waits(0)
        lib.spdba_debug_set_wait_limit(0)
    st_a, sp_a, err_a = run(6)
    st_b, sp_b, err_b = run(6)
    assert err_a is None and err_b is None and st_a["step"] == 6
    assert np.array_equal(sp_a, sp_b)
