"""Tensor-core convolution of the warm-start network against the FP64 direct convolution."""
import numpy as np
import pytest
import torch

from oracle import conv3d as C

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def U():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2211_03516_gb300 import unet
    return unet


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("shape,cin,cout,taps", [
    ((5, 7, 37), 16, 16, 27),     # ragged: 1295 positions = 10 full tiles + a tail
    ((4, 6, 9), 32, 48, 27),
    ((3, 5, 11), 16, 128, 27),
    ((2, 3, 70), 64, 32, 27),
    ((6, 6, 6), 16, 16, 1),
    ((4, 4, 8), 128, 16, 1),
])
def test_conv3d_matches_direct_convolution(U, shape, cin, cout, taps):
    rng = np.random.default_rng(cin + cout + taps)
    D, H, W = shape
    x = torch.from_numpy(rng.standard_normal((D, H, W, cin)).astype(np.float32)).to(torch.bfloat16)
    w = torch.from_numpy((rng.standard_normal((cout, taps, cin)) / np.sqrt(taps * cin)).astype(np.float32)).to(
        torch.bfloat16)
    b = torch.from_numpy(rng.standard_normal(cout).astype(np.float32))
    ref = C.conv3d(x.float().numpy(), w.float().numpy(), b.numpy(), relu=False)
    y32 = U.conv3d(x.to(DEV), w.to(DEV), b.to(DEV), relu=False, out_dtype=torch.float32)
    yr = U.conv3d(x.to(DEV), w.to(DEV), b.to(DEV), relu=True, out_dtype=torch.bfloat16)
    torch.cuda.synchronize()
    U.check_errors(DEV)
    assert rel_l2(y32.cpu().numpy(), ref) <= 1e-5
    assert rel_l2(yr.float().cpu().numpy(), np.maximum(ref, 0)) <= 4e-3
