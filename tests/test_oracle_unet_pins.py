"""Pins of the FP64 reference of the warm-start network (no GPU): the layer
operations against brute-force loops and exact identities, and the autograd
gradient against central finite differences of the loss."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import unet_ref as R  # noqa: E402


def test_conv_matches_brute_force():
    g = torch.Generator().manual_seed(1)
    x = torch.rand((2, 4, 5, 3), generator=g, dtype=torch.float64)
    w = torch.rand((3, 2, 27), generator=g, dtype=torch.float64) - 0.5
    b = torch.rand(3, generator=g, dtype=torch.float64)
    y = R.conv(x, w, b)
    C, D, H, W = x.shape
    ref = np.zeros((3, D, H, W))
    for co in range(3):
        for z in range(D):
            for yy in range(H):
                for xx in range(W):
                    s = b[co].item()
                    for ci in range(2):
                        for t in range(27):
                            dz, dy, dx = t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1
                            zz, y2, x2 = z + dz, yy + dy, xx + dx
                            if 0 <= zz < D and 0 <= y2 < H and 0 <= x2 < W:
                                s += w[co, ci, t].item() * x[ci, zz, y2, x2].item()
                    ref[co, z, yy, xx] = s
    assert np.allclose(y.numpy(), ref, atol=1e-13)


def test_pool_and_up_identities():
    g = torch.Generator().manual_seed(2)
    x = torch.rand((3, 5, 4, 7), generator=g, dtype=torch.float64)
    p = R.pool(x)
    assert p.shape == (3, 3, 2, 4)
    # the odd-edge window averages what it has
    assert abs(p[1, 2, 1, 3] - x[1, 4, 2:4, 6].mean()) < 1e-15
    assert abs(p[0, 0, 0, 0] - x[0, 0:2, 0:2, 0:2].mean()) < 1e-15
    assert torch.allclose(R.pool(torch.full((2, 5, 3, 3), 0.7, dtype=torch.float64)), torch.tensor(0.7, dtype=torch.float64))
    # pooling the nearest upsampling of a field returns the field
    c = torch.rand((2, 3, 2, 4), generator=g, dtype=torch.float64)
    assert torch.allclose(R.pool(R.up(c, (5, 4, 7))), c, atol=1e-15)
    assert torch.equal(R.up(c, (5, 4, 7))[:, 4, 3, 6], c[:, 2, 1, 3])


def _params(seed, scale=0.3):
    g = torch.Generator().manual_seed(seed)
    return {n: ((torch.rand((co, ci, 27), generator=g, dtype=torch.float64) * 2 - 1) * scale / np.sqrt(ci * 27) * 4,
                (torch.rand(co, generator=g, dtype=torch.float64) - 0.5) * 0.1)
            for n, ci, co in R.layer_shapes()}


def test_gradient_against_finite_differences():
    g = torch.Generator().manual_seed(3)
    size = (7, 6, 5)
    x = torch.rand((7,) + size, generator=g, dtype=torch.float64) - 0.5
    t = torch.rand((5,) + size, generator=g, dtype=torch.float64) - 0.5
    P = _params(4)
    _, loss, grads = R.loss_and_grads(P, x, t)
    # directional derivative along a random direction of all parameters
    dirs = {k: (torch.rand(w.shape, generator=g, dtype=torch.float64) - 0.5,
                torch.rand(b.shape, generator=g, dtype=torch.float64) - 0.5) for k, (w, b) in P.items()}
    eps = 1e-6

    def L(sign):
        Q = {k: (w + sign * eps * dirs[k][0], b + sign * eps * dirs[k][1]) for k, (w, b) in P.items()}
        return ((R.forward(Q, x) - t) ** 2).mean().item()

    fd = (L(1) - L(-1)) / (2 * eps)
    an = sum((grads[k][0] * dirs[k][0]).sum().item() + (grads[k][1] * dirs[k][1]).sum().item() for k in P)
    assert abs(fd - an) <= 1e-6 * abs(an) + 1e-12
    # single coordinates of the first and last layers
    for name, idx in (("e0a", (3, 5, 13)), ("head", (2, 7, 26)), ("d1a", (5, 60, 4))):
        w, b = P[name]
        e = torch.zeros_like(w)
        e[idx] = 1.0

        def Lw(sign):
            Q = dict(P)
            Q[name] = (w + sign * eps * e, b)
            return ((R.forward(Q, x) - t) ** 2).mean().item()

        fd = (Lw(1) - Lw(-1)) / (2 * eps)
        assert abs(fd - grads[name][0][idx].item()) <= 1e-6 * abs(fd) + 1e-11
