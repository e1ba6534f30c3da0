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


# W % 8 != 0 runs the gather kernel, W % 8 == 0 the halo-tile kernel (both checked below)
@pytest.mark.parametrize("shape,cin,cout,taps", [
    ((5, 7, 37), 16, 16, 27),     # gather: 1295 positions = 10 full tiles + a tail
    ((4, 6, 9), 32, 48, 27),
    ((3, 5, 11), 16, 128, 27),
    ((2, 3, 70), 64, 32, 27),
    ((6, 6, 6), 16, 16, 1),
    ((4, 4, 8), 128, 16, 1),      # halo from here on
    ((5, 7, 40), 16, 16, 27),     # tiles run through the rows of a plane; ragged regions
    ((4, 6, 24), 48, 48, 27),     # three 16-channel chunks per region
    ((3, 5, 128), 16, 32, 27),    # one tile per 128-voxel row
    ((3, 5, 200), 16, 32, 27),    # rows longer than a tile
    ((2, 3, 16), 16, 256, 27),    # output channels in slices
    ((5, 6, 32), 16, 16, 1),
    ((48, 128, 128), 16, 16, 27),  # several regions per block: both stages, both accumulators cycle
    ((24, 64, 64), 48, 128, 27),
    ((20, 32, 32), 64, 192, 27),
])
def test_conv3d_matches_direct_convolution(U, shape, cin, cout, taps):
    rng = np.random.default_rng(cin + cout + taps)
    D, H, W = shape
    x = torch.from_numpy(rng.standard_normal((D, H, W, cin)).astype(np.float32)).to(torch.bfloat16)
    w = torch.from_numpy((rng.standard_normal((cout, taps, cin)) / np.sqrt(taps * cin)).astype(np.float32)).to(
        torch.bfloat16)
    b = torch.from_numpy(rng.standard_normal(cout).astype(np.float32))
    ref = C.conv3d(x.float().numpy(), w.float().numpy(), b.numpy(), relu=False)
    kind, tz, ty, nt = U.conv3d_tiling(D, H, W, cin, cout, taps)
    assert kind == (1 if W % 8 == 0 and W + 16 <= 256 else 0)   # halo rows are one TMA box dimension
    if kind == 1:
        assert 1 <= tz <= D and 1 <= ty <= H and cout % nt == 0
    y32 = U.conv3d(x.to(DEV), w.to(DEV), b.to(DEV), relu=False, out_dtype=torch.float32)
    yr = U.conv3d(x.to(DEV), w.to(DEV), b.to(DEV), relu=True, out_dtype=torch.bfloat16)
    torch.cuda.synchronize()
    U.check_errors(DEV)
    assert rel_l2(y32.cpu().numpy(), ref) <= 1e-5
    assert rel_l2(yr.float().cpu().numpy(), np.maximum(ref, 0)) <= 4e-3


@pytest.mark.parametrize("shape,cin,cout,taps", [
    ((3, 5, 32), 16, 16, 27), ((3, 5, 32), 48, 16, 27), ((3, 5, 32), 16, 32, 27), ((3, 5, 32), 16, 16, 1),
    ((2, 3, 16), 16, 16, 27),        # W = 16: a 32-position stage is two 16-position boxes
    ((1, 1, 16), 32, 48, 27),        # a single stage; 32-byte dY rows at Cout = 48
    ((2, 2, 48), 192, 64, 27),       # W = 48: 16-position boxes; 128-byte X rows
    ((2, 3, 16), 128, 256, 27),      # N = 256
    ((5, 4, 64), 16, 16, 27),        # W = 64: stages of 64 positions
    ((4, 3, 32), 96, 32, 27),        # 64-byte rows
    ((2, 2, 16), 1024, 16, 1),       # 1^3 taps, wide Cin
    ((1, 2, 16), 512, 16, 27),       # many tile groups
    ((24, 32, 64), 16, 16, 27),      # hundreds of blocks, several stages each
])
def test_conv3d_weight_gradient_matches_direct_sum(U, shape, cin, cout, taps):
    rng = np.random.default_rng(cin * 7 + cout + shape[2])
    D, H, W = shape
    x = torch.from_numpy(rng.standard_normal((D, H, W, cin)).astype(np.float32)).to(torch.bfloat16)
    dy = torch.from_numpy(rng.standard_normal((D, H, W, cout)).astype(np.float32)).to(torch.bfloat16)
    xs, dys = x.double().numpy(), dy.double().numpy()
    xp = np.zeros((D + 2, H + 2, W + 2, cin))
    xp[1:-1, 1:-1, 1:-1] = xs
    ref = np.zeros((cout, taps, cin))
    for t, (dz, dyy, dx) in enumerate(C.tap_offsets(taps)):
        sh = xp[1 + dz:1 + dz + D, 1 + dyy:1 + dyy + H, 1 + dx:1 + dx + W].reshape(-1, cin)
        ref[:, t, :] = dys.reshape(-1, cout).T @ sh
    dw = torch.zeros((cout, taps, cin), device=DEV)
    U.conv3d_wgrad(x.to(DEV), dy.to(DEV), dw, taps)
    torch.cuda.synchronize()
    U.check_errors(DEV)
    assert rel_l2(dw.cpu().numpy(), ref) <= 1e-5


def test_unet_forward_backward_matches_fp64_reference(U):
    """Whole network: output, loss and every layer's weight and bias gradient against the
    FP64 autograd reference at the same (BF16-rounded) weights and input.  BF16 activation
    and gradient storage bounds the agreement at a few 1e-2."""
    from oracle import unet_ref
    net = U.UNet3D(device=DEV, seed=1)
    rng = np.random.default_rng(2)
    Dp, Vv, Uu, A = 8, 16, 128, 6
    proj = torch.from_numpy(rng.random((A, Vv, Uu), dtype=np.float32)).to(DEV)
    target = torch.from_numpy(rng.random((A, Vv, Uu), dtype=np.float32)).to(DEV)
    x0 = net.prepare(proj, 1.0, Dp)
    net.zero_grad()
    z = net.forward(x0)
    out, loss, dz = net.head(z, proj, 0.5, target=target, want_grad=True)
    net.backward(dz)
    torch.cuda.synchronize()
    U.check_errors(DEV)
    weights = {n: (L.Wb.float().cpu().numpy(), L.b.cpu().numpy()) for n, L in net.layers.items()}
    L_ref, z_ref, g_ref = unet_ref.loss_and_grads(U.ARCH, weights, x0.float().cpu().numpy(), target.cpu().numpy(), A,
                                                  proj.cpu().numpy(), 0.5)
    assert rel_l2(z.cpu().numpy()[..., 0], z_ref[..., 0]) <= 2e-2
    assert abs(loss.item() - L_ref) <= 2e-2 * L_ref
    for n, L in net.layers.items():
        gw, gb = g_ref[n]
        assert rel_l2(L.gW.cpu().numpy(), gw) <= 5e-2, n
        assert rel_l2(L.gb.cpu().numpy(), gb) <= 5e-2, n


def _offset_copy(x):
    """The same values at a 2-byte offset (not 16-byte aligned): the ops then take their
    one-element-per-thread kernels instead of the 16-byte ones."""
    buf = torch.empty(x.numel() + 8, device=x.device, dtype=x.dtype)
    v = buf[1:1 + x.numel()].view(x.shape)
    v.copy_(x)
    return v


def test_glue_ops_vector_and_scalar_kernels_agree_bitwise(U):
    """Pooling, upsampling, their backwards, concatenation, split and the ReLU backward:
    the 16-byte kernels against the scalar kernels (bit for bit) and against numpy."""
    nn = U._nn()
    s = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(5)
    D, H, W, C = 6, 10, 24, 16
    x = torch.from_numpy(rng.standard_normal((D, H, W, C)).astype(np.float32)).to(torch.bfloat16).to(DEV)
    c = torch.from_numpy(rng.standard_normal((D // 2, H // 2, W // 2, C)).astype(np.float32)).to(torch.bfloat16).to(DEV)
    for op, src, out_shape in ((0, x, c.shape), (1, c, x.shape), (2, c, x.shape), (3, x, c.shape)):
        y_vec = torch.empty(out_shape, device=DEV, dtype=torch.bfloat16)
        y_sca = _offset_copy(torch.zeros(out_shape, device=DEV, dtype=torch.bfloat16))
        src_sca = _offset_copy(src)
        assert nn.vamrt_nn_resample(op, src.data_ptr(), y_vec.data_ptr(), D, H, W, C, s) == 0
        assert nn.vamrt_nn_resample(op, src_sca.data_ptr(), y_sca.data_ptr(), D, H, W, C, s) == 0
        torch.cuda.synchronize()
        assert torch.equal(y_vec, y_sca), op
    xf = x.float().cpu().numpy()
    pooled = xf.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).mean(axis=(1, 3, 5))
    np.testing.assert_allclose(U.avgpool2(x).float().cpu().numpy(), pooled, rtol=1e-2, atol=1e-2)
    up = U.upsample2(c).float().cpu().numpy()
    np.testing.assert_array_equal(up, np.repeat(np.repeat(np.repeat(c.float().cpu().numpy(), 2, 0), 2, 1), 2, 2))
    b = torch.from_numpy(rng.standard_normal((D, H, W, 32)).astype(np.float32)).to(torch.bfloat16).to(DEV)
    ab = U.concat(x, b)
    ab_sca = _offset_copy(torch.zeros_like(ab))
    xs, bs = _offset_copy(x), _offset_copy(b)
    assert nn.vamrt_nn_concat(xs.data_ptr(), C, bs.data_ptr(), 32, ab_sca.data_ptr(), D * H * W, 0, s) == 0
    torch.cuda.synchronize()
    assert torch.equal(ab, ab_sca) and torch.equal(ab, torch.cat([x, b], dim=-1))
    a2, b2 = U.split(ab, C)
    assert torch.equal(a2, x) and torch.equal(b2, b)
    dy = torch.from_numpy(rng.standard_normal((D, H, W, C)).astype(np.float32)).to(torch.bfloat16).to(DEV)
    dy_vec, dy_sca = dy.clone(), _offset_copy(dy)
    x_sca = _offset_copy(x)
    assert nn.vamrt_nn_relu_backward(x.data_ptr(), dy_vec.data_ptr(), dy.numel(), s) == 0
    assert nn.vamrt_nn_relu_backward(x_sca.data_ptr(), dy_sca.data_ptr(), dy.numel(), s) == 0
    torch.cuda.synchronize()
    assert torch.equal(dy_vec, dy_sca) and torch.equal(dy_vec, torch.where(x > 0, dy, torch.zeros_like(dy)))
    for ch in (16, 48, 128):
        g = torch.from_numpy(rng.standard_normal((D * H * W, ch)).astype(np.float32)).to(torch.bfloat16).to(DEV)
        db = torch.zeros(ch, device=DEV)
        assert nn.vamrt_nn_bias_grad(g.data_ptr(), db.data_ptr(), D * H * W, ch, s) == 0
        torch.cuda.synchronize()
        np.testing.assert_allclose(db.cpu().numpy(), g.double().sum(0).cpu().numpy(), rtol=1e-4, atol=1e-3)
    # many positions per thread: the four-deep unrolled loop and its tail
    for npos, ch in ((1 << 20, 16), (300001, 48)):
        g = torch.from_numpy(rng.standard_normal((npos, ch)).astype(np.float32)).to(torch.bfloat16).to(DEV)
        db = torch.zeros(ch, device=DEV)
        assert nn.vamrt_nn_bias_grad(g.data_ptr(), db.data_ptr(), npos, ch, s) == 0
        torch.cuda.synchronize()
        np.testing.assert_allclose(db.cpu().numpy(), g.double().sum(0).cpu().numpy(), rtol=1e-4, atol=1e-2)
