"""The warm-start network on the GPU: a 3D U-Net driven through the kernels of
include/lbm_nn.h.

Architecture: input 7 channels (log10 Ra, Pr and the coarse steady u, v, w, T
and density deviation, trilinearly upsampled to the fine lattice); four levels with 16, 32, 48 and
64 channels, each two 3x3x3 convolutions with ReLU; average pooling by 2
(ceil sizes) on the way down and nearest upsampling by 2 on the way up, the
skip of each level concatenated after the upsampled channels; a 3x3x3 head
to 5 channels added to the upsampled coarse (u, v, w, T, density deviation),
so the network learns the fine-minus-coarse correction.  BF16 weights, FP32 accumulation,
FP32 master weights for Adam.

This module only allocates buffers (PyTorch tensors: device memory) and
sequences kernel calls; every arithmetic operation runs in the CUDA library.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import lbm as _lbm

CH = (16, 32, 48, 64)
IN_CH, OUT_CH = 7, 5

_fp, _u16p, _dp = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p


_i, _f, _i64, _v = ctypes.c_int, ctypes.c_float, ctypes.c_int64, ctypes.c_void_p
# argument types of every entry point of include/lbm_nn.h
NN_SIGNATURES = {
    "lbm_nn_conv3d_forward": [_v, _i, _i, _i, _i, _v, _v, _i, _v, _i, _v],
    "lbm_nn_conv3d_backward_data": [_v, _i, _i, _i, _i, _v, _v, _i, _v, _i, _v],
    "lbm_nn_conv3d_backward_weight": [_v, _i, _i, _i, _i, _v, _i, _v, _v, _v],
    "lbm_nn_relu_backward": [_v, _v, _i64, _v],
    "lbm_nn_avgpool2_forward": [_v, _i, _i, _i, _i, _v, _v],
    "lbm_nn_avgpool2_backward": [_v, _i, _i, _i, _i, _v, _i, _v],
    "lbm_nn_upsample2_forward": [_v, _i, _i, _i, _i, _v, _v],
    "lbm_nn_upsample2_backward": [_v, _i, _i, _i, _i, _v, _v],
    "lbm_nn_trilinear": [_v, _i, _i, _i, _i, _v, _i, _i, _i, _v],
    "lbm_nn_axpy": [_f, _v, _v, _i64, _v],
    "lbm_nn_mse": [_v, _v, _i64, _v, _v, _v],
    "lbm_nn_adam": [_v, _v, _v, _v, _v, _i64, _f, _f, _f, _f, _i, _v],
    "lbm_nn_to_bf16": [_v, _v, _i64, _v],
}


def _sig():
    L = _lbm.lib()
    if getattr(L, "_nn_ready", False):
        return L
    for name, args in NN_SIGNATURES.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L._nn_ready = True
    return L


def _call(name, *args):
    st = getattr(_sig(), name)(*args)
    if st != _lbm.LBM_OK:
        raise _lbm.LbmError(st, _lbm.lib().lbm_last_error(None).decode())


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream():
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream or None)


# ------------------------------------------------------------- kernel ops --
# Thin wrappers over the C ABI (PyTorch tensors supply device pointers).

def conv_forward(x, w_bf16, b, cout, y, relu):
    cin, D, H, W = x.shape
    _call("lbm_nn_conv3d_forward", _p(x), cin, D, H, W, _p(w_bf16), _p(b), cout, _p(y), int(relu), _stream())


def conv_backward_data(dy, w_bf16, wt_scratch, cin, dx, accumulate=False):
    cout, D, H, W = dy.shape
    _call("lbm_nn_conv3d_backward_data", _p(dy), cout, D, H, W, _p(w_bf16), _p(wt_scratch), cin, _p(dx),
          int(accumulate), _stream())


def conv_backward_weight(x, dy, dw, db):
    cin, D, H, W = x.shape
    _call("lbm_nn_conv3d_backward_weight", _p(x), cin, D, H, W, _p(dy), dy.shape[0], _p(dw), _p(db), _stream())


def relu_backward(dy, y):
    _call("lbm_nn_relu_backward", _p(dy), _p(y), dy.numel(), _stream())


def pool_forward(x, y):
    C, D, H, W = x.shape
    _call("lbm_nn_avgpool2_forward", _p(x), C, D, H, W, _p(y), _stream())


def pool_backward(dy, dx, accumulate=False):
    C, D, H, W = dx.shape
    _call("lbm_nn_avgpool2_backward", _p(dy), C, D, H, W, _p(dx), int(accumulate), _stream())


def up_forward(x, y):
    C, D, H, W = y.shape
    _call("lbm_nn_upsample2_forward", _p(x), C, D, H, W, _p(y), _stream())


def up_backward(dy, dx):
    C, D, H, W = dy.shape
    _call("lbm_nn_upsample2_backward", _p(dy), C, D, H, W, _p(dx), _stream())


def trilinear(x, y):
    C, d, h, w = x.shape
    _, D, H, W = y.shape
    _call("lbm_nn_trilinear", _p(x), C, d, h, w, _p(y), D, H, W, _stream())


def axpy(a, x, y):
    _call("lbm_nn_axpy", ctypes.c_float(a), _p(x), _p(y), x.numel(), _stream())


def mse(p, t, loss, grad):
    _call("lbm_nn_mse", _p(p), _p(t), p.numel(), _p(loss), _p(grad), _stream())


def adam(w, w_bf16, g, m, v, lr, t, beta1=0.9, beta2=0.999, eps=1e-8):
    _call("lbm_nn_adam", _p(w), _p(w_bf16), _p(g), _p(m), _p(v), w.numel(), ctypes.c_float(lr),
          ctypes.c_float(beta1), ctypes.c_float(beta2), ctypes.c_float(eps), int(t), _stream())


def to_bf16(x, y):
    _call("lbm_nn_to_bf16", _p(x), _p(y), x.numel(), _stream())


def layer_shapes():
    s = []
    cin = IN_CH
    for l, c in enumerate(CH):
        s += [(f"e{l}a", cin, c), (f"e{l}b", c, c)]
        cin = c
    for l in (2, 1, 0):
        s += [(f"d{l}a", CH[l + 1] + CH[l], CH[l]), (f"d{l}b", CH[l], CH[l])]
    s.append(("head", CH[0], OUT_CH))
    return s


class UNet:
    """Parameters, Adam state and activation buffers for one lattice size."""

    def __init__(self, size, seed=0, device="cuda"):
        import torch

        self.torch = torch
        self.size = tuple(size)  # (D, H, W)
        gen = torch.Generator().manual_seed(seed)
        self.params = {}
        for name, cin, cout in layer_shapes():
            bound = float(np.sqrt(6.0 / (cin * 27)))
            if name == "head":
                bound *= 0.1
            w = ((torch.rand((cout, cin, 27), generator=gen, dtype=torch.float64) * 2 - 1) * bound).float()
            w = w.to(device)
            p = dict(w=w, b=torch.zeros(cout, device=device), wb=torch.empty(w.shape, dtype=torch.int16, device=device),
                     gw=torch.zeros_like(w), gb=torch.zeros(cout, device=device), mw=torch.zeros_like(w),
                     vw=torch.zeros_like(w), mb=torch.zeros(cout, device=device), vb=torch.zeros(cout, device=device),
                     cin=cin, cout=cout)
            to_bf16(w, p["wb"])
            self.params[name] = p
        self.wt = torch.empty(max(p["w"].numel() for p in self.params.values()), dtype=torch.int16, device=device)
        self.step_count = 0
        self._alloc(device)

    def _alloc(self, device):
        torch = self.torch
        sizes = [self.size]
        for _ in range(3):
            sizes.append(tuple((s + 1) // 2 for s in sizes[-1]))
        self.sizes = sizes
        E = lambda c, l: torch.empty((c,) + sizes[l], device=device)  # noqa: E731
        b = {}
        for l, c in enumerate(CH):
            b[f"a{l}"] = E(c, l)  # first conv of the level (encoder)
        # concat buffers: upsampled channels first, then the skip (the level's encoder output)
        for l in (0, 1, 2):
            b[f"c{l}"] = E(CH[l + 1] + CH[l], l)
            b[f"p{l}"] = E(CH[l], l + 1)  # pooled skip
            b[f"da{l}"] = E(CH[l], l)
            b[f"d{l}"] = E(CH[l], l)
        b["bott"] = E(CH[3], 3)
        b["out"] = E(OUT_CH, 0)
        self.buf = b
        self.grad = {k: torch.empty_like(v) for k, v in b.items()}
        self.loss = torch.zeros(1, dtype=torch.float64, device=device)

    def skip(self, l, grad=False):
        t = (self.grad if grad else self.buf)[f"c{l}"]
        return t[CH[l + 1]:]

    def forward(self, x):
        """x: [7][D][H][W] float32 on the GPU; returns the output buffer."""
        b, P = self.buf, self.params
        t = x
        for l in range(4):
            pa, pb = P[f"e{l}a"], P[f"e{l}b"]
            conv_forward(t, pa["wb"], pa["b"], pa["cout"], b[f"a{l}"], True)
            out = self.skip(l) if l < 3 else b["bott"]
            conv_forward(b[f"a{l}"], pb["wb"], pb["b"], pb["cout"], out, True)
            if l < 3:
                pool_forward(out, b[f"p{l}"])
                t = b[f"p{l}"]
        t = b["bott"]
        for l in (2, 1, 0):
            c = b[f"c{l}"]
            up_forward(t, c[: CH[l + 1]])
            pa, pb = P[f"d{l}a"], P[f"d{l}b"]
            conv_forward(c, pa["wb"], pa["b"], pa["cout"], b[f"da{l}"], True)
            conv_forward(b[f"da{l}"], pb["wb"], pb["b"], pb["cout"], b[f"d{l}"], True)
            t = b[f"d{l}"]
        ph = P["head"]
        conv_forward(t, ph["wb"], ph["b"], OUT_CH, b["out"], False)
        axpy(1.0, x[2:7].contiguous() if not x[2:7].is_contiguous() else x[2:7], b["out"])
        return b["out"]

    def _conv_back(self, name, x, y, gy, gx, relu=True, accumulate=False):
        """Backward of y = relu(conv(x)): gradient wrt weights (accumulated) and,
        when gx is given, wrt x."""
        p = self.params[name]
        if relu:
            relu_backward(gy, y)
        conv_backward_weight(x, gy, p["gw"], p["gb"])
        if gx is not None:
            conv_backward_data(gy, p["wb"], self.wt, p["cin"], gx, accumulate)

    def backward(self, x, target):
        """Adds the parameter gradients of mean((out - target)^2); returns the
        loss as a device scalar (forward must have run on x)."""
        b, g = self.buf, self.grad
        self.loss.zero_()
        mse(b["out"], target, self.loss, g["out"])
        self._conv_back("head", b["d0"], None, g["out"], g["d0"], relu=False)
        for l in (0, 1, 2):
            self._conv_back(f"d{l}b", b[f"da{l}"], b[f"d{l}"], g[f"d{l}"], g[f"da{l}"])
            self._conv_back(f"d{l}a", b[f"c{l}"], b[f"da{l}"], g[f"da{l}"], g[f"c{l}"])
            # the upsampled channels send their gradient to the level below
            below = g["bott"] if l == 2 else g[f"d{l + 1}"]
            up_backward(g[f"c{l}"][: CH[l + 1]], below)
        # bottleneck and encoder, from the bottom up; skip gradients already
        # hold the decoder's share, the pooled path adds the rest
        for l in (3, 2, 1, 0):
            out = b["bott"] if l == 3 else self.skip(l)
            gout = g["bott"] if l == 3 else self.skip(l, grad=True)
            if l < 3:
                pool_backward(g[f"p{l}"], gout, accumulate=True)
            inp = x if l == 0 else b[f"p{l - 1}"]
            ginp = None if l == 0 else g[f"p{l - 1}"]
            self._conv_back(f"e{l}b", b[f"a{l}"], out, gout, g[f"a{l}"])
            self._conv_back(f"e{l}a", inp, b[f"a{l}"], g[f"a{l}"], ginp)
        return self.loss

    def adam_step(self, lr):
        self.step_count += 1
        for p in self.params.values():
            adam(p["w"], p["wb"], p["gw"], p["mw"], p["vw"], lr, self.step_count)
            adam(p["b"], None, p["gb"], p["mb"], p["vb"], lr, self.step_count)

    def zero_grad(self):
        for p in self.params.values():
            p["gw"].zero_()
            p["gb"].zero_()

    def bf16_weights(self):
        """FP64 copies of the BF16 weights and FP32 biases (for the reference)."""
        torch = self.torch
        out = {}
        for name, p in self.params.items():
            wb = p["wb"].cpu().numpy().astype(np.uint16).astype(np.uint32) << 16
            w = torch.from_numpy(wb.view(np.float32).astype(np.float64))
            out[name] = (w, p["b"].double().cpu())
        return out
