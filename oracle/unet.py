"""FP64 NumPy reference of the warm-start network (TEST INFRASTRUCTURE ONLY).

The same architecture as the library's network, written plainly: convolutions by summing
shifted copies of the zero-padded input times each tap's weight matrix, explicit backward
passes.  Used to check the GPU forward and backward kernels; pinned by finite differences in
tests/test_oracle_unet.py.

Layout: activations [B, H, W, C]; conv weights [Cout, T, Cin] (T = 9 taps of a 3x3 kernel in
row-major (dy, dx) order, or T = 1); flat parameter vector = for each layer its weights then its
bias, then the head's weights [2, 32] and bias [2].
"""
from __future__ import annotations

import numpy as np

SPECS = [(16, 32, 9, 1), (32, 32, 9, 1), (32, 64, 9, 1), (64, 64, 9, 1), (64, 128, 9, 1),
         (128, 128, 9, 1), (128, 256, 9, 1), (256, 256, 9, 1), (256, 128, 1, 0), (128, 128, 9, 1),
         (128, 64, 1, 0), (64, 64, 9, 1), (64, 32, 1, 0), (32, 32, 9, 1)]
HEAD_C = 32


def layout():
    offs = []
    off = 0
    for cin, cout, t, _ in SPECS:
        offs.append((off, off + cout * t * cin))
        off += cout * t * cin + cout
    head = off
    return offs, head, head + 2 * HEAD_C + 2


def unpack(params):
    offs, head, total = layout()
    assert params.shape[0] == total
    Ws, bs = [], []
    for (wo, bo), (cin, cout, t, _) in zip(offs, SPECS):
        Ws.append(params[wo:bo].reshape(cout, t, cin))
        bs.append(params[bo:bo + cout])
    hw = params[head:head + 2 * HEAD_C].reshape(2, HEAD_C)
    hb = params[head + 2 * HEAD_C:head + 2 * HEAD_C + 2]
    return Ws, bs, hw, hb


def _shifts(T):
    return [(t // 3 - 1, t % 3 - 1) for t in range(9)] if T == 9 else [(0, 0)]


def conv(x, W, b):
    """out[p] = sum_t x[p + d_t] @ W[:, t, :].T + b (zero outside the image)."""
    B, H, Wd, _ = x.shape
    cout, T, _ = W.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    out = np.zeros((B, H, Wd, cout))
    for t, (dy, dx) in enumerate(_shifts(T)):
        out += xp[:, 1 + dy:1 + dy + H, 1 + dx:1 + dx + Wd, :] @ W[:, t, :].T
    return out + b


def conv_bwd(x, W, g):
    """Gradients of sum(g * conv(x, W, b)) w.r.t. x, W, b."""
    B, H, Wd, _ = x.shape
    cout, T, cin = W.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    dW = np.zeros_like(W)
    dxp = np.zeros_like(xp)
    for t, (dy, dx) in enumerate(_shifts(T)):
        xs = xp[:, 1 + dy:1 + dy + H, 1 + dx:1 + dx + Wd, :]
        dW[:, t, :] = np.einsum("bhwo,bhwi->oi", g, xs)
        dxp[:, 1 + dy:1 + dy + H, 1 + dx:1 + dx + Wd, :] += g @ W[:, t, :]
    return dxp[:, 1:1 + H, 1:1 + Wd, :], dW, g.sum(axis=(0, 1, 2))


def pool(x):
    return 0.25 * (x[:, 0::2, 0::2] + x[:, 1::2, 0::2] + x[:, 0::2, 1::2] + x[:, 1::2, 1::2])


def pool_bwd(g):
    return 0.25 * np.repeat(np.repeat(g, 2, axis=1), 2, axis=2)


def up(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up_bwd(g):
    return g[:, 0::2, 0::2] + g[:, 1::2, 0::2] + g[:, 0::2, 1::2] + g[:, 1::2, 1::2]


def relu(x):
    return np.maximum(x, 0.0)


def forward(params, x):
    Ws, bs, hw, hb = unpack(params)
    c = {"x": x}

    def L(i, inp):
        o = conv(inp, Ws[i], bs[i])
        return relu(o) if SPECS[i][3] else o

    c["a0"] = L(0, x)
    c["s0"] = L(1, c["a0"])
    c["p0"] = pool(c["s0"])
    c["a1"] = L(2, c["p0"])
    c["s1"] = L(3, c["a1"])
    c["p1"] = pool(c["s1"])
    c["a2"] = L(4, c["p1"])
    c["s2"] = L(5, c["a2"])
    c["p2"] = pool(c["s2"])
    c["a3"] = L(6, c["p2"])
    c["b3"] = L(7, c["a3"])
    c["r2"] = L(8, c["b3"])
    c["u2"] = up(c["r2"]) + c["s2"]
    c["d2"] = L(9, c["u2"])
    c["r1"] = L(10, c["d2"])
    c["u1"] = up(c["r1"]) + c["s1"]
    c["d1"] = L(11, c["u1"])
    c["r0"] = L(12, c["d1"])
    c["u0"] = up(c["r0"]) + c["s0"]
    c["d0"] = L(13, c["u0"])
    out = c["d0"] @ hw.T + hb
    return out, c


def loss(out, target):
    """Mean over pixels of the summed squared errors of both outputs, and d loss / d out."""
    P = out.shape[0] * out.shape[1] * out.shape[2]
    e = out - target
    return float((e * e).sum() / P), 2.0 * e / P


def backward(params, c, dout):
    Ws, bs, hw, hb = unpack(params)
    offs, head, total = layout()
    grad = np.zeros(total)

    def put(i, dW, db):
        wo, bo = offs[i]
        grad[wo:bo] = dW.reshape(-1)
        grad[bo:bo + SPECS[i][1]] = db

    grad[head:head + 2 * HEAD_C] = np.einsum("bhwj,bhwc->jc", dout, c["d0"]).reshape(-1)
    grad[head + 2 * HEAD_C:] = dout.sum(axis=(0, 1, 2))
    g = dout @ hw

    def back(i, inp, outv, g):
        if SPECS[i][3]:
            g = g * (outv > 0)
        dx, dW, db = conv_bwd(inp, Ws[i], g)
        put(i, dW, db)
        return dx

    du0 = back(13, c["u0"], c["d0"], g)
    ds0 = du0.copy()
    dd1 = back(12, c["d1"], c["r0"], up_bwd(du0))
    du1 = back(11, c["u1"], c["d1"], dd1)
    ds1 = du1.copy()
    dd2 = back(10, c["d2"], c["r1"], up_bwd(du1))
    du2 = back(9, c["u2"], c["d2"], dd2)
    ds2 = du2.copy()
    db3 = back(8, c["b3"], c["r2"], up_bwd(du2))
    da3 = back(7, c["a3"], c["b3"], db3)
    dp2 = back(6, c["p2"], c["a3"], da3)
    ds2 += pool_bwd(dp2)
    da2 = back(5, c["a2"], c["s2"], ds2)
    dp1 = back(4, c["p1"], c["a2"], da2)
    ds1 += pool_bwd(dp1)
    da1 = back(3, c["a1"], c["s1"], ds1)
    dp0 = back(2, c["p0"], c["a1"], da1)
    ds0 += pool_bwd(dp0)
    da0 = back(1, c["a0"], c["s0"], ds0)
    back(0, c["x"], c["a0"], da0)
    return grad


def loss_and_grad(params, x, target):
    out, cache = forward(params, x)
    lval, dout = loss(out, target)
    return lval, backward(params, cache, dout)
