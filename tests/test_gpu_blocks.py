"""GPU block activity and classification/compaction against the oracle, through the C ABI."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


def _rand(shape, seed, dtype, scale_blocks=None):
    r = np.random.default_rng(seed)
    x = (r.standard_normal(shape) + 1j * r.standard_normal(shape))
    if scale_blocks is not None:
        # give blocks wildly different magnitudes, like a decaying spectrum
        x = x * scale_blocks
    return x.astype(dtype)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("shape,block", [((64, 64), (16, 16)), ((32, 32, 32), (8, 8, 8)), ((4096,), (64,)),
                                         ((48, 96), (16, 8)), ((256, 256, 256), (8, 8, 8)),
                                         ((256, 320, 96), (8, 8, 8)), ((256, 256, 128), (8, 8, 16))])
def test_block_activity_matches_oracle(shape, block, precision):
    import torch
    from paper_2609_03922_gb300 import spdba
    if precision == 1 and np.prod(shape) > 1 << 20:
        pytest.skip("full-size case runs in complex64 only")
    cdt = np.complex64 if precision == 0 else np.complex128
    r = np.random.default_rng(3)
    scale = np.exp(-6 * r.random(shape))
    q = _rand(shape, 1, cdt, scale)
    nb = tuple(s // b for s, b in zip(shape, block))
    qd = torch.from_numpy(q).cuda()
    maxsq = torch.empty(nb, dtype=torch.float64, device="cuda")
    sumsq = torch.empty(nb, dtype=torch.float64, device="cuda")
    gmax = torch.empty(2, dtype=torch.float64, device="cuda")
    spdba.block_activity(qd, block, maxsq, sumsq, gmax, precision=precision)
    torch.cuda.synchronize()
    q64 = q.astype(np.complex128)
    mx, sm = O.block_measures(q64, block)
    assert np.array_equal(maxsq.cpu().numpy(), mx)            # same FP64 formula: bit-exact
    assert np.allclose(sumsq.cpu().numpy(), sm, rtol=1e-12, atol=0)
    g = gmax.cpu().numpy()
    assert g[0] == O.global_max_sq(q64, exclude_dc=False)
    assert g[1] == O.global_max_sq(q64, exclude_dc=True)


@pytest.mark.parametrize("shape,block", [((256, 256, 256), (8, 8, 8)), ((256, 320, 96), (8, 8, 8)),
                                         ((256, 256, 128), (8, 8, 16)), ((128, 160, 512), (8, 4, 8))])
def test_block_max_only_matches_oracle(shape, block):
    """The maximum alone (no energy sum): complex64 fields with enough rows of
    blocks take the streaming rows kernel (whole rows of blocks per CTA, lane
    groups of 4 or 8 per block); bit-exact FP64 maxima, the global maxima with
    and without k = 0."""
    import torch
    from paper_2609_03922_gb300 import spdba
    r = np.random.default_rng(4)
    scale = np.exp(-6 * r.random(shape))
    q = _rand(shape, 2, np.complex64, scale)
    nb = tuple(s // b for s, b in zip(shape, block))
    qd = torch.from_numpy(q).cuda()
    maxsq = torch.empty(nb, dtype=torch.float64, device="cuda")
    gmax = torch.zeros(2, dtype=torch.float64, device="cuda")
    spdba.block_activity(qd, block, maxsq, None, gmax, precision=0)
    torch.cuda.synchronize()
    q64 = q.astype(np.complex128)
    mx, _ = O.block_measures(q64, block)
    assert np.array_equal(maxsq.cpu().numpy(), mx)
    g = gmax.cpu().numpy()
    assert g[0] == O.global_max_sq(q64, exclude_dc=False)
    assert g[1] == O.global_max_sq(q64, exclude_dc=True)


def _screen_field(shape, block, seed):
    """A complex64 field whose blocks each hold one hard case for the FP32 screen
    of the activity scan: exact zeros, one subnormal mode, all modes below the
    screen floor 2^-99 (in |q|^2), modes straddling it, near-ties within 2^-22
    of each other, exact ties, a dominant k = 0 mode, huge dynamic range, and
    plain random blocks."""
    r = np.random.default_rng(seed)
    nb = tuple(s // b for s, b in zip(shape, block))
    bm = int(np.prod(block))
    q = np.zeros(shape, dtype=np.complex64)
    view = q.reshape(nb[0], block[0], nb[1], block[1], nb[2], block[2])
    for b0 in range(nb[0]):
        for b1 in range(nb[1]):
            for b2 in range(nb[2]):
                kind = r.integers(0, 9)
                v = np.zeros(bm, dtype=np.complex64)
                if kind == 1:
                    v[r.integers(0, bm)] = np.float32(1e-40) * (1 + 1j)
                elif kind == 2:
                    v = ((r.standard_normal(bm) + 1j * r.standard_normal(bm)) * 1e-20).astype(np.complex64)
                elif kind == 3:
                    v = ((r.standard_normal(bm) + 1j * r.standard_normal(bm)) * 2.0 ** -50).astype(np.complex64)
                elif kind == 4:
                    ang = r.random(bm) * 2 * np.pi
                    mag = 1.0 + r.integers(-4, 5, size=bm) * 2.0 ** -24
                    v = (mag * np.exp(1j * ang)).astype(np.complex64)
                elif kind == 5:
                    v = (r.integers(-3, 4, size=bm) + 1j * r.integers(-3, 4, size=bm)).astype(np.complex64)
                elif kind == 6:
                    v = ((r.standard_normal(bm) + 1j * r.standard_normal(bm)) * 10.0 ** r.uniform(-30, 15, bm)
                         ).astype(np.complex64)
                elif kind >= 7:
                    v = (r.standard_normal(bm) + 1j * r.standard_normal(bm)).astype(np.complex64)
                view[b0, :, b1, :, b2, :] = v.reshape(block)
    q[(0,) * len(shape)] = np.complex64(3e9 + 1e9j)   # dominant k = 0
    return q


@pytest.mark.parametrize("shape,block", [((256, 256, 64), (8, 8, 8)), ((64, 64, 64), (8, 8, 8)),
                                         ((128, 256, 32), (4, 4, 8))])
def test_block_max_screen_hard_cases(shape, block):
    """Both scan kernels (rows of blocks, warp per block) on blocks built to
    defeat an FP32 screen: the FP64 maxima stay bit-exact, and the maximum over
    k != 0 ignores the dominant k = 0 mode."""
    import torch
    from paper_2609_03922_gb300 import spdba
    q = _screen_field(shape, block, 11)
    nb = tuple(s // b for s, b in zip(shape, block))
    maxsq = torch.empty(nb, dtype=torch.float64, device="cuda")
    gmax = torch.zeros(2, dtype=torch.float64, device="cuda")
    spdba.block_activity(torch.from_numpy(q).cuda(), block, maxsq, None, gmax, precision=0)
    torch.cuda.synchronize()
    q64 = q.astype(np.complex128)
    mx, _ = O.block_measures(q64, block)
    assert np.array_equal(maxsq.cpu().numpy(), mx)
    g = gmax.cpu().numpy()
    assert g[0] == O.global_max_sq(q64, exclude_dc=False)
    assert g[1] == O.global_max_sq(q64, exclude_dc=True)


def _expected_chi(states):
    d = states.ndim
    chi = np.zeros(states.shape, dtype=np.uint8)
    for a in range(d):
        lo = np.roll(states, 1, axis=a) == O.STATE_FROZEN
        hi = np.roll(states, -1, axis=a) == O.STATE_FROZEN
        chi |= (lo.astype(np.uint8) << (2 * a)) | (hi.astype(np.uint8) << (2 * a + 1))
    return chi


@pytest.mark.parametrize("nb", [(4, 4), (8, 8), (1, 8), (64,), (3, 5, 7), (32, 32, 32), (48, 48, 48)])
@pytest.mark.parametrize("force_dc,transitions", [(1, 1), (0, 1), (1, 0)])
def test_classify_matches_oracle(nb, force_dc, transitions):
    import torch
    from paper_2609_03922_gb300 import spdba
    r = np.random.default_rng(sum(nb))
    meas = np.exp(-8 * r.random(nb))
    tau = float(np.quantile(meas, 0.9))
    meas.flat[r.integers(0, meas.size)] = tau          # an exact tie: >= makes it active
    n = meas.size
    md = torch.from_numpy(meas).cuda()
    td = torch.tensor([tau], dtype=torch.float64, device="cuda")
    states = torch.empty(n, dtype=torch.uint8, device="cuda")
    chi = torch.empty(n, dtype=torch.uint8, device="cuda")
    lst = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    cnt = torch.empty(1, dtype=torch.int32, device="cuda")
    scratch = torch.empty(spdba.classify_scratch_bytes(n), dtype=torch.uint8, device="cuda")
    spdba.classify(nb, md, td, force_dc, transitions, states, chi, lst, cnt, scratch)
    torch.cuda.synchronize()
    ref = O.classify(meas, tau, force_dc=bool(force_dc), transitions=bool(transitions))
    got = states.cpu().numpy().reshape(nb)
    assert np.array_equal(got, ref)
    assert np.array_equal(chi.cpu().numpy().reshape(nb)[ref == O.STATE_TRANSITION],
                          _expected_chi(ref)[ref == O.STATE_TRANSITION])
    ids = np.flatnonzero(ref.ravel() != O.STATE_FROZEN)
    c = int(cnt.item())
    assert c == ids.size
    assert np.array_equal(lst.cpu().numpy()[:c], ids)


def test_classify_all_frozen_and_all_active():
    import torch
    from paper_2609_03922_gb300 import spdba
    nb = (16, 16)
    n = 256
    for tau, expect_count in [(np.inf, 0), (0.0, n)]:
        md = torch.zeros(n, dtype=torch.float64, device="cuda")
        td = torch.tensor([tau], dtype=torch.float64, device="cuda")
        states = torch.empty(n, dtype=torch.uint8, device="cuda")
        chi = torch.empty(n, dtype=torch.uint8, device="cuda")
        lst = torch.empty(n, dtype=torch.int32, device="cuda")
        cnt = torch.empty(1, dtype=torch.int32, device="cuda")
        scratch = torch.empty(spdba.classify_scratch_bytes(n), dtype=torch.uint8, device="cuda")
        spdba.classify(nb, md, td, 0, 1, states, chi, lst, cnt, scratch)
        torch.cuda.synchronize()
        assert int(cnt.item()) == expect_count
