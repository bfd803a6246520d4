"""The learned CNN's layers one at a time against the FP64 oracle (oracle/unet.py).

Both sides get the same FP32 input, weights, bias and output gradient and round to BF16
at the same points, so what remains is FP32 accumulation (products of BF16 values are
exact in FP32; sums over K <= 8192 terms): relative L2 differences of ~1e-6.  A ReLU mask
can differ where a pre-activation lies within FP32 rounding of zero (a handful of the
~10^5 outputs), which moves the gradients by ~1e-5.  Gate: 1e-4 relative L2 for every
output and gradient - an indexing mistake in any kernel gives O(1).
"""
import pytest

torch = pytest.importorskip("torch")

from oracle import unet as ounet  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = 1e-4


@pytest.fixture(scope="module")
def bsct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_13471_gb300 as m

    m.lib()
    return m


def rel(a, b):
    a, b = a.double().cpu(), b.double().cpu()
    return float((a - b).norm() / b.norm())


def to_dev(t):  # [n, C, H, W] float64 -> [C, n, H, W] float32 on the device
    return t.permute(1, 0, 2, 3).contiguous().float().to(DEV)


def from_dev(t):
    return t.permute(1, 0, 2, 3).double().cpu()


@pytest.mark.parametrize("n,cin,cout,H", [(2, 1, 32, 64), (2, 32, 32, 64), (2, 64, 128, 16), (1, 256, 128, 16),
                                          (2, 128, 256, 8)])
@pytest.mark.parametrize("relu", [True, False])
def test_conv3x3_layer(bsct, n, cin, cout, H, relu):
    g = torch.Generator().manual_seed(n * 1000 + cin + cout + H)
    kpad = ((9 * cin + 7) // 8) * 8
    x = torch.randn((n, cin, H, H), generator=g).float().double()
    w4 = (torch.randn((cout, cin, 3, 3), generator=g) * (2.0 / (9 * cin)) ** 0.5).float().double()
    b = (0.1 * torch.randn(cout, generator=g)).float().double()
    gout = torch.randn((n, cout, H, H), generator=g).float().double()
    wk = torch.zeros((cout, kpad), dtype=torch.float32)
    wk[:, :9 * cin] = w4.reshape(cout, 9 * cin).float()
    out, gin, gw, gb = bsct.conv3x3_layer(to_dev(x), wk.to(DEV), b.float().to(DEV), relu=relu, gout=to_dev(gout))
    ro, rdx, rdw, rdb = ounet.layer_grads("conv3", x, w4, b, gout, relu)
    errs = {"out": rel(from_dev(out), ro), "gin": rel(from_dev(gin), rdx),
            "gw": rel(gw[:, :9 * cin].reshape(cout, cin, 3, 3), rdw), "gb": rel(gb, rdb)}
    print(f"conv3x3 n={n} cin={cin} cout={cout} H={H} relu={relu}:", {k: f"{v:.1e}" for k, v in errs.items()})
    assert max(errs.values()) < TOL, errs
    assert float(gw[:, 9 * cin:].abs().max() if kpad > 9 * cin else 0.0) == 0.0  # padding columns stay zero


@pytest.mark.parametrize("n,cin,cout,H", [(2, 256, 128, 8), (2, 128, 64, 16), (2, 64, 32, 32), (1, 16, 8, 8)])
def test_tconv2x2_layer(bsct, n, cin, cout, H):
    g = torch.Generator().manual_seed(7 * n + cin + cout + H)
    x = torch.randn((n, cin, H, H), generator=g).float().double()
    wt = (torch.randn((cin, cout, 2, 2), generator=g) * cin ** -0.5).float().double()  # torch layout
    b = (0.1 * torch.randn(cout, generator=g)).float().double()
    gout = torch.randn((n, cout, 2 * H, 2 * H), generator=g).float().double()
    wl = wt.permute(1, 2, 3, 0).reshape(cout * 4, cin).float().contiguous()  # [(co*4 + dy*2 + dx)][ci]
    out, gin, gw, gb = bsct.tconv2x2_layer(to_dev(x), wl.to(DEV), b.float().to(DEV), gout=to_dev(gout))
    ro, rdx, rdw, rdb = ounet.layer_grads("tconv2", x, wt, b, gout)
    errs = {"out": rel(from_dev(out), ro), "gin": rel(from_dev(gin), rdx),
            "gw": rel(gw.view(cout, 2, 2, cin).permute(3, 0, 1, 2), rdw), "gb": rel(gb, rdb)}
    print(f"tconv2x2 n={n} cin={cin} cout={cout} H={H}:", {k: f"{v:.1e}" for k, v in errs.items()})
    assert max(errs.values()) < TOL, errs


def test_layer_arguments_checked(bsct):
    x = torch.zeros((3, 1, 4, 4), device=DEV)
    w = torch.zeros((6, 32), device=DEV)  # cout = 6 is not a multiple of 8
    with pytest.raises(RuntimeError, match="invalid argument"):
        bsct.conv3x3_layer(x, w, torch.zeros(6, device=DEV))


def test_layer_gradients_are_bit_reproducible(bsct):
    # the bias gradients are channel sums over ~10^4 outputs, formed as per-block partials
    # added in block order: the same call twice gives the same bits
    g = torch.Generator().manual_seed(21)
    x = torch.randn((16, 2, 64, 64), generator=g).to(DEV)
    w = (torch.randn((32, 144), generator=g) * 0.1).to(DEV)
    b = torch.randn(32, generator=g).to(DEV)
    gout = torch.randn((32, 2, 64, 64), generator=g).to(DEV)
    r1 = bsct.conv3x3_layer(x, w, b, relu=True, gout=gout)
    r2 = bsct.conv3x3_layer(x, w, b, relu=True, gout=gout)
    assert all(torch.equal(a, c) for a, c in zip(r1, r2))
    wt = (torch.randn((64, 16), generator=g) * 0.1).to(DEV)
    bt = torch.randn(16, generator=g).to(DEV)
    gt = torch.randn((16, 2, 128, 128), generator=g).to(DEV)
    t1 = bsct.tconv2x2_layer(x, wt, bt, gout=gt)
    t2 = bsct.tconv2x2_layer(x, wt, bt, gout=gt)
    assert all(torch.equal(a, c) for a, c in zip(t1, t2))
