"""Warm-start network kernels on the GPU against the FP64 CPU reference
(oracle/unet_ref.py): each layer operation forward and backward, Adam, and
the whole network's output and parameter gradients.  Tolerance: relative
2e-5 of the output scale for one convolution, 1e-5 for the network's output:
FP32 accumulation on the tensor cores (whose additions need not round to
nearest) over up to 27 x 130 products whose magnitudes add to several times
the output, each with its FP32 operand carried as two BF16 terms (relative
error <= 2^-18); the weights are the same BF16 values on both sides."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import unet_ref as R  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def U():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1903_08882_gb300 import _build

    _build.build()
    from paper_1903_08882_gb300 import unet

    return unet


def _bf16(t):
    """Round FP32/FP64 to BF16 values (nearest even), returned as float64."""
    a = t.detach().cpu().float().numpy().view(np.uint32).astype(np.uint64)
    r = ((a + 0x7FFF + ((a >> 16) & 1)) >> 16) << 16
    return torch.from_numpy(r.astype(np.uint32).view(np.float32).astype(np.float64))


def _rel(a, b):
    return (a.double().cpu() - b).abs().max().item() / max(b.abs().max().item(), 1e-30)


@pytest.mark.parametrize(
    "cin,cout,size",
    [(3, 5, (7, 6, 5)), (19, 13, (9, 4, 11)), (48, 16, (17, 17, 17)), (112, 48, (9, 9, 9)), (7, 37, (1, 3, 21)),
     (130, 5, (3, 4, 5))],
)
def test_conv_forward_backward(U, cin, cout, size):
    g = torch.Generator().manual_seed(cin * 100 + cout)
    x = torch.rand((cin,) + size, generator=g, dtype=torch.float64) - 0.5
    w = (torch.rand((cout, cin, 27), generator=g, dtype=torch.float64) - 0.5) / np.sqrt(cin)
    b = torch.rand(cout, generator=g, dtype=torch.float64) - 0.5
    gy = torch.rand((cout,) + size, generator=g, dtype=torch.float64) - 0.5
    wq = _bf16(w)
    xr = x.clone().requires_grad_(True)
    wr = wq.clone().requires_grad_(True)
    br = b.clone().requires_grad_(True)
    yr = R.conv(xr, wr, br)
    (yr * gy).sum().backward()
    xd, gyd = x.float().cuda(), gy.float().cuda()
    wb = torch.empty((cout, cin, 27), dtype=torch.int16, device="cuda")
    U.to_bf16(w.float().cuda(), wb)
    y = torch.empty((cout,) + size, device="cuda")
    U.conv_forward(xd, wb, b.float().cuda(), cout, y, relu=False)
    assert _rel(y, yr.detach()) < 2e-5
    yrelu = torch.empty_like(y)
    U.conv_forward(xd, wb, b.float().cuda(), cout, yrelu, relu=True)
    assert torch.equal(yrelu, torch.clamp(y, min=0))
    dx = torch.empty_like(xd)
    scratch = torch.empty(cout * cin * 27, dtype=torch.int16, device="cuda")
    U.conv_backward_data(gyd, wb, scratch, cin, dx)
    assert _rel(dx, xr.grad) < 2e-5
    dw = torch.zeros((cout, cin, 27), device="cuda")
    db = torch.zeros(cout, device="cuda")
    if cin > 128:  # the weight gradient takes at most 128 input channels
        with pytest.raises(RuntimeError):
            U.conv_backward_weight(xd, gyd, dw, db)
        return
    U.conv_backward_weight(xd, gyd, dw, db)
    assert _rel(dw, wr.grad) < 2e-5 and _rel(db, br.grad) < 2e-5


def test_pool_up_trilinear(U):
    g = torch.Generator().manual_seed(7)
    x = torch.rand((3, 9, 6, 11), generator=g, dtype=torch.float64)
    p = torch.empty((3, 5, 3, 6), device="cuda")
    U.pool_forward(x.float().cuda(), p)
    assert _rel(p, R.pool(x)) < 1e-6
    gp = torch.rand((3, 5, 3, 6), generator=g, dtype=torch.float64)
    xr = x.clone().requires_grad_(True)
    (R.pool(xr) * gp).sum().backward()
    dx = torch.empty((3, 9, 6, 11), device="cuda")
    U.pool_backward(gp.float().cuda(), dx)
    assert _rel(dx, xr.grad) < 1e-6
    c = torch.rand((4, 5, 3, 6), generator=g, dtype=torch.float64)
    u = torch.empty((4, 9, 6, 11), device="cuda")
    U.up_forward(c.float().cuda(), u)
    assert torch.equal(u.double().cpu(), R.up(c, (9, 6, 11)).float().double())
    gu = torch.rand((4, 9, 6, 11), generator=g, dtype=torch.float64)
    cr = c.clone().requires_grad_(True)
    (R.up(cr, (9, 6, 11)) * gu).sum().backward()
    dc = torch.empty((4, 5, 3, 6), device="cuda")
    U.up_backward(gu.float().cuda(), dc)
    assert _rel(dc, cr.grad) < 1e-6
    s = torch.rand((4, 33, 33, 33), generator=g, dtype=torch.float64)
    f = torch.empty((4, 65, 65, 65), device="cuda")
    U.trilinear(s.float().cuda(), f)
    assert _rel(f, R.trilinear(s, (65, 65, 65))) < 1e-6


def test_adam(U):
    g = torch.Generator().manual_seed(9)
    w = torch.rand(1000, generator=g, dtype=torch.float64) - 0.5
    gr = torch.rand(1000, generator=g, dtype=torch.float64) - 0.5
    wd, gd = w.float().cuda(), gr.float().cuda()
    m, v = torch.zeros_like(wd), torch.zeros_like(wd)
    wb = torch.empty(1000, dtype=torch.int16, device="cuda")
    wn, mn, vn = w.numpy(), np.zeros(1000), np.zeros(1000)
    for t in (1, 2, 3):
        gd.copy_(gr.float().cuda() * t)
        U.adam(wd, wb, gd, m, v, 1e-2, t)
        wn, mn, vn = R.adam(wn, gr.numpy() * t, mn, vn, 1e-2, t)
        assert gd.abs().max().item() == 0.0
    assert np.abs(wd.double().cpu().numpy() - wn).max() < 1e-6


def test_network_output_and_gradients(U):
    size = (17, 17, 17)
    net = U.UNet(size, seed=3)
    g = torch.Generator().manual_seed(5)
    x = torch.rand((7,) + size, generator=g, dtype=torch.float64) - 0.5
    t = torch.rand((5,) + size, generator=g, dtype=torch.float64) - 0.5
    out = net.forward(x.float().cuda())
    net.zero_grad()
    loss = net.backward(x.float().cuda(), t.float().cuda())
    out_ref, loss_ref, grads = R.loss_and_grads(net.bf16_weights(), x, t)
    assert _rel(out, out_ref) < 1e-5
    assert abs(loss.item() - loss_ref) < 1e-5 * loss_ref
    for name, p in net.params.items():
        gw, gb = grads[name]
        assert _rel(p["gw"], gw) < 1e-4, name
        assert _rel(p["gb"], gb) < 1e-4, name


def test_training_reduces_loss(U):
    size = (17, 17, 17)
    net = U.UNet(size, seed=4)
    g = torch.Generator().manual_seed(6)
    x = (torch.rand((7,) + size, generator=g) - 0.5).cuda()
    # a target the network can reach: the residual input shifted per channel
    shift = torch.tensor([0.1, -0.05, 0.08, 0.02, -0.1], device="cuda").view(5, 1, 1, 1)
    t = x[2:7] + shift
    losses = []
    for _ in range(40):
        net.zero_grad()
        net.forward(x)
        losses.append(net.backward(x, t).item())
        net.adam_step(3e-3)
    assert losses[-1] < 0.3 * losses[0], losses[::8]
