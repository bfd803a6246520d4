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
