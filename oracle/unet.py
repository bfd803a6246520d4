"""FP64 CPU reference of the learned warm start's encoder-decoder CNN - oracle side.

Test infrastructure: plain PyTorch CPU float64 operations (conv2d, conv_transpose2d,
max_pool2d) for checking the library's BF16 tensor-core forward and backward kernels.
The CUDA path rounds to BF16 (round to nearest even) at fixed points; this reference
rounds at the same points and computes everything else in float64:
  * 3x3 convolution: input and weights rounded; the ReLU-masked output gradient is
    rounded before both the weight and the input gradient products; bias gradient
    from the unrounded masked gradient;
  * 2x2 stride-2 transposed convolution: input and weights rounded; the output
    gradient rounded before both products; bias gradient unrounded;
  * max-pool, concatenation and the 1x1 head (FP32 weights on the GPU): no rounding.

Flat parameter layout (the library's, reproduced from its description): for each 3x3
convolution W[cout][kpad] with column ci*9 + ky*3 + kx (kpad = 9*cin rounded up to a
multiple of 8, extra columns zero) followed by b[cout]; for each transposed convolution
W[(co*4 + dy*2 + dx)][ci] followed by b[cout]; the head w[base], b[1]; the total
rounded up to a multiple of 8.  Layer order: c0a c0b c1a c1b c2a c2b c3a c3b t3 d2a d2b
t2 d1a d1b t1 d0a d0b head.
"""
import torch
import torch.nn.functional as F


def bf16(t):
    return t.to(torch.bfloat16).to(torch.float64)


def layout(base):
    B = base
    spec = [("c", 1, B), ("c", B, B), ("c", B, 2 * B), ("c", 2 * B, 2 * B), ("c", 2 * B, 4 * B),
            ("c", 4 * B, 4 * B), ("c", 4 * B, 8 * B), ("c", 8 * B, 8 * B), ("t", 8 * B, 4 * B),
            ("c", 8 * B, 4 * B), ("c", 4 * B, 4 * B), ("t", 4 * B, 2 * B), ("c", 4 * B, 2 * B),
            ("c", 2 * B, 2 * B), ("t", 2 * B, B), ("c", 2 * B, B), ("c", B, B)]
    off = 0
    layers = []
    for kind, ci, co in spec:
        if kind == "c":
            kpad = ((9 * ci + 7) // 8) * 8
            layers.append(dict(kind="c", cin=ci, cout=co, kpad=kpad, w=off, b=off + co * kpad))
            off += co * kpad + co
        else:
            layers.append(dict(kind="t", cin=ci, cout=co, w=off, b=off + co * 4 * ci))
            off += co * 4 * ci + co
    head = dict(w=off, b=off + B)
    off += B + 1
    n = ((off + 7) // 8) * 8
    return layers, head, n


class _Conv3(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, w, b):
        xr, wr = bf16(x), bf16(w)
        out = F.relu(F.conv2d(xr, wr, b, padding=1))
        ctx.save_for_backward(xr, wr, out)
        return out

    @staticmethod
    def backward(ctx, g):
        xr, wr, out = ctx.saved_tensors
        d = g * (out > 0)
        db = d.sum(dim=(0, 2, 3))
        dr = bf16(d)
        dx = torch.nn.grad.conv2d_input(xr.shape, wr, dr, padding=1)
        dw = torch.nn.grad.conv2d_weight(xr, wr.shape, dr, padding=1)
        return dx, dw, db


class _Conv3Linear(torch.autograd.Function):
    """The 3x3 convolution without its ReLU (the same rounding points as _Conv3)."""

    @staticmethod
    def forward(ctx, x, w, b):
        xr, wr = bf16(x), bf16(w)
        ctx.save_for_backward(xr, wr)
        return F.conv2d(xr, wr, b, padding=1)

    @staticmethod
    def backward(ctx, g):
        xr, wr = ctx.saved_tensors
        db = g.sum(dim=(0, 2, 3))
        dr = bf16(g)
        dx = torch.nn.grad.conv2d_input(xr.shape, wr, dr, padding=1)
        dw = torch.nn.grad.conv2d_weight(xr, wr.shape, dr, padding=1)
        return dx, dw, db


def layer_grads(kind, x, w, b, gout, relu=True):
    """One layer of the network on its own (kind "conv3" or "tconv2"): returns
    (out, d x, d w, d b) for the output gradient gout, all float64, with the library's
    rounding points.  x [n, cin, H, W]; w in torch layout ([cout, cin, 3, 3] or
    [cin, cout, 2, 2]); b [cout]."""
    xv = x.detach().clone().requires_grad_()
    wv = w.detach().clone().requires_grad_()
    bv = b.detach().clone().requires_grad_()
    if kind == "conv3":
        out = (_Conv3 if relu else _Conv3Linear).apply(xv, wv, bv)
    elif kind == "tconv2":
        out = _TConv.apply(xv, wv, bv)
    else:
        raise ValueError(kind)
    out.backward(gout)
    return out.detach(), xv.grad, wv.grad, bv.grad


class _TConv(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, w, b):
        xr, wr = bf16(x), bf16(w)
        ctx.save_for_backward(xr, wr)
        return F.conv_transpose2d(xr, wr, b, stride=2)

    @staticmethod
    def backward(ctx, g):
        xr, wr = ctx.saved_tensors
        gr = bf16(g)
        with torch.enable_grad():
            xv = xr.detach().requires_grad_()
            wv = wr.detach().requires_grad_()
            y = F.conv_transpose2d(xv, wv, None, stride=2)
            dx, dw = torch.autograd.grad(y, (xv, wv), gr)
        return dx, dw, g.sum(dim=(0, 2, 3))


def unpack(params, base):
    """Flat parameter vector -> list of (weight, bias) tensors in torch layouts (float64, requires grad)."""
    layers, head, n = layout(base)
    p = params.to(torch.float64)
    assert p.numel() == n
    out = []
    for L in layers:
        if L["kind"] == "c":
            W = p[L["w"]:L["w"] + L["cout"] * L["kpad"]].view(L["cout"], L["kpad"])[:, :9 * L["cin"]]
            W = W.reshape(L["cout"], L["cin"], 3, 3)
        else:
            W = p[L["w"]:L["w"] + L["cout"] * 4 * L["cin"]].view(L["cout"], 2, 2, L["cin"]).permute(3, 0, 1, 2)
        bvec = p[L["b"]:L["b"] + L["cout"]]
        out.append([W.clone().requires_grad_(), bvec.clone().requires_grad_()])
    hw = p[head["w"]:head["w"] + base].clone().requires_grad_()
    hb = p[head["b"]:head["b"] + 1].clone().requires_grad_()
    return out, (hw, hb)


def pack_grads(tensors, head, base):
    """Gradients back into the flat layout (padding columns zero)."""
    layers, hd, n = layout(base)
    g = torch.zeros(n, dtype=torch.float64)
    for L, (W, b) in zip(layers, tensors):
        if L["kind"] == "c":
            full = torch.zeros(L["cout"], L["kpad"], dtype=torch.float64)
            full[:, :9 * L["cin"]] = W.grad.reshape(L["cout"], 9 * L["cin"])
            g[L["w"]:L["w"] + L["cout"] * L["kpad"]] = full.reshape(-1)
        else:
            g[L["w"]:L["w"] + L["cout"] * 4 * L["cin"]] = W.grad.permute(1, 2, 3, 0).reshape(-1)
        g[L["b"]:L["b"] + L["cout"]] = b.grad
    g[hd["w"]:hd["w"] + base] = head[0].grad
    g[hd["b"]:hd["b"] + 1] = head[1].grad
    return g


def forward(x, tensors, head):
    """x: [n, H, W] float64 -> [n, H, W]."""
    c = iter(tensors)
    conv = lambda a: _Conv3.apply(a, *next(c))
    h = x[:, None]
    e0 = conv(conv(h))
    e1 = conv(conv(F.max_pool2d(e0, 2)))
    e2 = conv(conv(F.max_pool2d(e1, 2)))
    e3 = conv(conv(F.max_pool2d(e2, 2)))
    W, b = next(c)
    d2 = conv(conv(torch.cat([_TConv.apply(e3, W, b), e2], dim=1)))
    W, b = next(c)
    d1 = conv(conv(torch.cat([_TConv.apply(d2, W, b), e1], dim=1)))
    W, b = next(c)
    d0 = conv(conv(torch.cat([_TConv.apply(d1, W, b), e0], dim=1)))
    out = torch.einsum("c,nchw->nhw", head[0], d0) + head[1]
    return out
