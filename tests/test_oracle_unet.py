"""Pins for the CNN oracle: with the BF16 rounding switched off its hand-written
backward passes must equal autograd (torch.autograd.gradcheck in float64), and the
parameter count matches the architecture."""
import pytest
import torch

from oracle import unet as ounet


def test_parameter_count():
    _, _, n = ounet.layout(32)
    assert 1_900_000 < n < 1_950_000  # ~1.92 M parameters at base 32


@pytest.fixture
def no_rounding(monkeypatch):
    monkeypatch.setattr(ounet, "bf16", lambda t: t)


def test_conv_backward_matches_autograd(no_rounding):
    g = torch.Generator().manual_seed(0)
    x = torch.randn((2, 3, 6, 5), dtype=torch.float64, generator=g, requires_grad=True)
    w = torch.randn((4, 3, 3, 3), dtype=torch.float64, generator=g, requires_grad=True)
    b = torch.randn(4, dtype=torch.float64, generator=g, requires_grad=True)
    assert torch.autograd.gradcheck(ounet._Conv3.apply, (x, w, b))


def test_tconv_backward_matches_autograd(no_rounding):
    g = torch.Generator().manual_seed(1)
    x = torch.randn((2, 3, 4, 3), dtype=torch.float64, generator=g, requires_grad=True)
    w = torch.randn((3, 2, 2, 2), dtype=torch.float64, generator=g, requires_grad=True)
    b = torch.randn(2, dtype=torch.float64, generator=g, requires_grad=True)
    assert torch.autograd.gradcheck(ounet._TConv.apply, (x, w, b))


def test_whole_network_gradients(no_rounding):
    base = 8
    _, _, n = ounet.layout(base)
    params = torch.randn(n, dtype=torch.float64, generator=torch.Generator().manual_seed(2)) * 0.2
    tensors, head = ounet.unpack(params, base)
    # seeded (an unseeded draw occasionally put a ReLU / max-pool kink within the
    # finite-difference step of a tested parameter)
    x = torch.randn((1, 64, 64), dtype=torch.float64, generator=torch.Generator().manual_seed(4))
    out = ounet.forward(x, tensors, head)
    gout = torch.randn(out.shape, dtype=torch.float64, generator=torch.Generator().manual_seed(5))
    out.backward(gout)
    g = ounet.pack_grads(tensors, head, base)
    # finite difference on a few parameters of the flat vector
    for i in torch.randint(0, n, (6,), generator=torch.Generator().manual_seed(3)).tolist():
        e = torch.zeros(n, dtype=torch.float64)
        e[i] = 1e-6
        tp, hp = ounet.unpack(params + e, base)
        tm, hm = ounet.unpack(params - e, base)
        fd = float(((ounet.forward(x, tp, hp) - ounet.forward(x, tm, hm)) * gout).sum() / 2e-6)
        assert abs(fd - float(g[i])) < 1e-5 * max(1.0, abs(fd))


def test_linear_conv_backward_matches_autograd(no_rounding):
    g = torch.Generator().manual_seed(6)
    x = torch.randn((2, 3, 5, 6), dtype=torch.float64, generator=g, requires_grad=True)
    w = torch.randn((2, 3, 3, 3), dtype=torch.float64, generator=g, requires_grad=True)
    b = torch.randn(2, dtype=torch.float64, generator=g, requires_grad=True)
    assert torch.autograd.gradcheck(ounet._Conv3Linear.apply, (x, w, b))


def test_layer_grads_by_finite_differences(no_rounding):
    # the per-layer entry of the oracle against central differences of <out, gout>
    g = torch.Generator().manual_seed(7)
    for kind, wshape, relu in (("conv3", (3, 2, 3, 3), False), ("conv3", (3, 2, 3, 3), True),
                               ("tconv2", (2, 3, 2, 2), False)):
        x = torch.randn((2, 2, 4, 5), dtype=torch.float64, generator=g)
        w = torch.randn(wshape, dtype=torch.float64, generator=g)
        b = torch.randn(3, dtype=torch.float64, generator=g)
        o = ounet.layer_grads(kind, x, w, b, torch.zeros(_out_shape(kind, x, w)), relu)[0]
        gout = torch.randn(o.shape, dtype=torch.float64, generator=g)
        _, dx, dw, db = ounet.layer_grads(kind, x, w, b, gout, relu)
        f = lambda xx, ww, bb: float((ounet.layer_grads(kind, xx, ww, bb, torch.zeros(o.shape), relu)[0] * gout).sum())
        for t, grad, name in ((x, dx, "x"), (w, dw, "w"), (b, db, "b")):
            flat = t.reshape(-1)
            for i in (0, flat.numel() // 2, flat.numel() - 1):
                e = torch.zeros_like(flat)
                e[i] = 1e-6
                args = {"x": x, "w": w, "b": b}
                args[name] = (flat + e).reshape(t.shape)
                fp = f(args["x"], args["w"], args["b"])
                args[name] = (flat - e).reshape(t.shape)
                fm = f(args["x"], args["w"], args["b"])
                fd = (fp - fm) / 2e-6
                assert abs(fd - float(grad.reshape(-1)[i])) < 1e-6 * max(1.0, abs(fd)), (kind, name, i)


def _out_shape(kind, x, w):
    n, _, H, W = x.shape
    return (n, w.shape[0], H, W) if kind == "conv3" else (n, w.shape[1], 2 * H, 2 * W)
