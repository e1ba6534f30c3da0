"""FP64 CPU reference of the warm-start network (test infrastructure only): the same
layers as the CUDA path -- 3^3 convolutions (zero padding) + ReLU, 2x average pool,
nearest 2x upsample, channel concatenation, 1^3 head added to the (scaled) input
projections, mean 0.5 squared error --
written with plain PyTorch CPU ops in float64, differentiated by autograd."""
import numpy as np
import torch
import torch.nn.functional as F


def _w5(W, taps):
    """[cout][taps][cin] (taps in dz, dy, dx order) -> [cout][cin][k][k][k]."""
    W = torch.as_tensor(np.asarray(W, dtype=np.float64))
    cout, _, cin = W.shape
    k = 3 if taps == 27 else 1
    return W.permute(0, 2, 1).reshape(cout, cin, k, k, k)


def loss_and_grads(arch, weights, x, target, n_angles, base, in_scale):
    """arch: [(name, cin, cout, taps)]; weights: name -> (W, b) numpy; x [Dp][V][U][16];
    target, base [n_angles][V][U].  Returns (loss, z [Dp][V][U][16], grads name -> (gW, gb))."""
    params = {}
    for (n, ci, co, t) in arch:
        W, b = weights[n]
        params[n] = (_w5(W, t).requires_grad_(True), torch.as_tensor(np.asarray(b, np.float64)).requires_grad_(True))
    taps = {n: t for (n, ci, co, t) in arch}

    def conv(n, v, relu=True):
        W, b = params[n]
        y = F.conv3d(v, W, b, padding=1 if taps[n] == 27 else 0)
        return F.relu(y) if relu else y

    xin = torch.as_tensor(np.asarray(x, np.float64)).permute(3, 0, 1, 2).unsqueeze(0)
    s0 = conv("enc0b", conv("enc0a", xin))
    s1 = conv("enc1b", conv("enc1a", F.avg_pool3d(s0, 2)))
    s2 = conv("enc2b", conv("enc2a", F.avg_pool3d(s1, 2)))
    b2 = conv("botb", conv("bota", F.avg_pool3d(s2, 2)))
    up = lambda v: F.interpolate(v, scale_factor=2, mode="nearest")
    d2 = conv("dec2b", conv("dec2a", torch.cat([up(b2), s2], 1)))
    d1 = conv("dec1b", conv("dec1a", torch.cat([up(d2), s1], 1)))
    d0 = conv("dec0b", conv("dec0a", torch.cat([up(d1), s0], 1)))
    z = conv("head", d0, relu=False)
    out = in_scale * torch.as_tensor(np.asarray(base, np.float64)) + z[0, 0, :n_angles]
    t = torch.as_tensor(np.asarray(target, np.float64))
    loss = 0.5 * ((out - t) ** 2).mean()
    loss.backward()
    grads = {}
    for (n, ci, co, tp) in arch:
        W, b = params[n]
        gW = W.grad.reshape(co, ci, tp).permute(0, 2, 1).numpy()
        grads[n] = (gW, b.grad.numpy())
    return float(loss), z[0].permute(1, 2, 3, 0).detach().numpy(), grads
