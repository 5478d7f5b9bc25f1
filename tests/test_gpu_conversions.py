"""The integer-pipe binary32 <-> binary64 conversions of the FP32 deviation
kernels agree bit for bit with the hardware conversions (torch's casts) over
random values of every magnitude in range, signed zeros, ties, inf and NaN."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def test_conversions_bitwise():
    from paper_0912_2913_gb300 import _native as N

    rng = np.random.default_rng(3)
    n = 1 << 20
    # binary32 inputs: random bit patterns restricted to normal numbers, plus specials
    fb = rng.integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
    e = (fb >> 23) & 0xFF
    fb = np.where((e == 0) | (e == 255), fb ^ (0x40 << 23), fb).astype(np.uint32)
    f = fb.view(np.float32).copy()
    f[:6] = [0.0, -0.0, np.inf, -np.inf, np.nan, 1.0]
    # binary64 inputs whose binary32 rounding is normal: exponents within range,
    # mantissas with all tail patterns, exact ties included
    mant = rng.integers(0, 2**52, size=n, dtype=np.uint64)
    ex = rng.integers(1023 - 125, 1023 + 127, size=n, dtype=np.uint64)
    sign = rng.integers(0, 2, size=n, dtype=np.uint64) << np.uint64(63)
    db = sign | (ex << np.uint64(52)) | mant
    tie = np.arange(n) % 7 == 0
    db[tie] = (db[tie] & ~np.uint64(0x1FFFFFFF)) | np.uint64(0x10000000)
    d = db.view(np.float64).copy()
    d[:6] = [0.0, -0.0, np.inf, -np.inf, np.nan, 3.4028234663852886e38 * 2]
    fi = torch.from_numpy(f).cuda()
    di = torch.from_numpy(d).cuda()
    fo = torch.empty(n, dtype=torch.float64, device="cuda")
    do = torch.empty(n, dtype=torch.float32, device="cuda")
    N.rlb_selftest_conversions(fi, di, n, fo, do)
    ref_f2d = fi.double()
    ref_d2f = di.float()
    nan_f = torch.isnan(ref_f2d)
    assert torch.equal(torch.isnan(fo), nan_f)
    assert torch.equal(fo[~nan_f].view(torch.int64), ref_f2d[~nan_f].view(torch.int64))
    nan_d = torch.isnan(ref_d2f)
    assert torch.equal(torch.isnan(do), nan_d)
    assert torch.equal(do[~nan_d].view(torch.int32), ref_d2f[~nan_d].view(torch.int32))
