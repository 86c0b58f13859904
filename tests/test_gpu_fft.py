"""GPU FFT (Stockham passes) against the oracle's FP64 FFT, through the C ABI."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

TOL = {0: 2e-6, 1: 1e-13}   # rel-L2: complex64 (FP32 arithmetic) / complex128


def _rand(shape, seed, dtype):
    r = np.random.default_rng(seed)
    return (r.standard_normal(shape) + 1j * r.standard_normal(shape)).astype(dtype)


CASES_ND = [(16, 16), (32, 64), (128, 128), (192, 256), (384, 128), (512, 512), (16, 32, 64), (64, 64, 64),
            (32, 192, 16), (384, 16, 16), (128, 128, 128), (256, 64, 32)]
CASES_1D = [16, 256, 1024, 4096, 8192, 65536, 262144]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("shape", CASES_ND + [(n,) for n in CASES_1D])
def test_fft_matches_oracle(shape, precision):
    import torch
    from paper_2609_03922_gb300 import spdba
    cdt = np.complex64 if precision == 0 else np.complex128
    batch = 3 if np.prod(shape) <= 1 << 16 else 1
    x = _rand((batch,) + tuple(shape), sum(shape) + precision, cdt)
    plan = spdba.FFTPlan(shape, batch=batch, precision=precision)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    plan.exec(xd, yd, spdba.SPDBA_FORWARD)
    zd = torch.empty_like(xd)
    plan.exec(yd, zd, spdba.SPDBA_INVERSE)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    z = zd.cpu().numpy()
    x64 = x.astype(np.complex128)
    for b in range(batch):
        ref = O.fftn(x64[b])
        assert O.rel_l2(y[b], ref) <= TOL[precision], "forward %s b=%d" % (shape, b)
        refi = O.ifftn(x64[b])
        assert O.rel_l2(z[b], x64[b]) <= 2 * TOL[precision], "round trip %s" % (shape,)
        # inverse of x itself against the oracle's inverse
    plan.exec(xd, yd, spdba.SPDBA_INVERSE)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    assert O.rel_l2(y[0], O.ifftn(x64[0])) <= TOL[precision]
    plan.close()


def test_fft_in_place():
    import torch
    from paper_2609_03922_gb300 import spdba
    x = _rand((64, 128), 5, np.complex64)
    xd = torch.from_numpy(x).cuda()
    plan = spdba.FFTPlan((64, 128))
    plan.exec(xd, xd, spdba.SPDBA_FORWARD)
    torch.cuda.synchronize()
    assert O.rel_l2(xd.cpu().numpy(), O.fftn(x.astype(np.complex128))) <= 2e-6


def test_fft_rejects_unsupported():
    from paper_2609_03922_gb300 import spdba
    with pytest.raises(spdba.SpdbaError) as e:
        spdba.FFTPlan((96, 100))
    assert e.value.status == spdba.SPDBA_ERR_UNSUPPORTED
    with pytest.raises(spdba.SpdbaError):
        spdba.FFTPlan((1024, 64))   # multi-D axes are limited to 512
