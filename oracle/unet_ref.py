"""FP64 CPU reference of the warm-start network (TEST INFRASTRUCTURE ONLY).

Plain PyTorch CPU ops in float64; gradients come from autograd.  Only tests
import this module.  It shares no code with the CUDA path; the architecture
below is written out from its description:

  input 7 channels (log10 Ra, Pr, and the coarse u, v, w, T and density
  deviation trilinearly upsampled); 4 levels with 16, 32, 48, 64 channels; two 3x3x3 convolutions
  with ReLU per level; average pooling by 2 (ceil sizes) down, nearest
  upsampling by 2 (cropped to the skip's size) up; skip connections
  concatenated after the upsampled channels; a 3x3x3 head to 5 channels added
  to the upsampled coarse (u, v, w, T, density deviation).

Weights are FP64 copies of the BF16-rounded weights the GPU uses; the tap
order of a weight row [Cout][Cin][27] is dz, dy, dx in -1, 0, 1 with dx
fastest, i.e. torch's [Cout][Cin][3][3][3].
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

CH = (16, 32, 48, 64)
IN_CH, OUT_CH = 7, 5


def layer_shapes():
    """(name, Cin, Cout) of every convolution, in a fixed order."""
    s = []
    cin = IN_CH
    for l, c in enumerate(CH):
        s.append((f"e{l}a", cin, c))
        s.append((f"e{l}b", c, c))
        cin = c
    for l in (2, 1, 0):
        s.append((f"d{l}a", CH[l + 1] + CH[l], CH[l]))
        s.append((f"d{l}b", CH[l], CH[l]))
    s.append(("head", CH[0], OUT_CH))
    return s


def conv(x, w, b):
    cout, cin = w.shape[0], w.shape[1]
    return F.conv3d(x[None], w.reshape(cout, cin, 3, 3, 3), b, padding=1)[0]


def pool(x):
    """Average over 2x2x2 windows with ceil sizes; a window at an odd edge
    averages the voxels it has."""
    C, D, H, W = x.shape
    pad = (0, W % 2, 0, H % 2, 0, D % 2)
    xs = F.pad(x, pad)
    ones = F.pad(torch.ones((1, D, H, W), dtype=x.dtype), pad)
    def sum2(t):
        c, d, h, w = t.shape
        return t.reshape(c, d // 2, 2, h // 2, 2, w // 2, 2).sum(dim=(2, 4, 6))
    return sum2(xs) / sum2(ones)


def up(x, size):
    """Nearest upsampling by 2, cropped to `size` = (D, H, W)."""
    y = x.repeat_interleave(2, dim=1).repeat_interleave(2, dim=2).repeat_interleave(2, dim=3)
    return y[:, : size[0], : size[1], : size[2]]


def forward(params, x):
    """params: dict name -> (w [Cout][Cin][27], b [Cout]) float64; x [7][D][H][W]."""
    def block(name, t):
        w, b = params[name]
        return F.relu(conv(t, w, b))

    skips = []
    t = x
    for l in range(4):
        t = block(f"e{l}b", block(f"e{l}a", t))
        if l < 3:
            skips.append(t)
            t = pool(t)
    for l in (2, 1, 0):
        s = skips[l]
        t = torch.cat([up(t, s.shape[1:]), s], dim=0)
        t = block(f"d{l}b", block(f"d{l}a", t))
    w, b = params["head"]
    return conv(t, w, b) + x[2:7]


def loss_and_grads(params, x, target):
    """Mean squared error over all output values and its parameter gradients."""
    p = {k: (w.detach().clone().requires_grad_(True), b.detach().clone().requires_grad_(True))
         for k, (w, b) in params.items()}
    out = forward(p, x)
    loss = ((out - target) ** 2).mean()
    loss.backward()
    return out.detach(), loss.item(), {k: (w.grad, b.grad) for k, (w, b) in p.items()}


def trilinear(x, size):
    """Node-centred trilinear interpolation of [C][d][h][w] to `size`
    (source coordinate (j + 1/2) n_in/n_out - 1/2, clamped at the walls)."""
    return F.interpolate(x[None], size=tuple(size), mode="trilinear", align_corners=False)[0]


def adam(w, g, m, v, lr, t, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba, 2015), in FP64 numpy; returns new w, m, v."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1**t)
    vh = v / (1 - beta2**t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
