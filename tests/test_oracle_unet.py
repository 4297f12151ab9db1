"""Pins of the FP64 reference network (oracle/unet.py) to finite differences."""
import numpy as np
import pytest

from oracle import unet


def _small_case(seed=0):
    rng = np.random.default_rng(seed)
    _, _, total = unet.layout()
    params = np.zeros(total)
    offs, head, _ = unet.layout()
    for (wo, bo), (cin, cout, t, _) in zip(offs, unet.SPECS):
        params[wo:bo] = rng.normal(size=bo - wo) * np.sqrt(2.0 / (t * cin))
        params[bo:bo + cout] = rng.normal(size=cout) * 0.1
    params[head:] = rng.normal(size=total - head) * 0.2
    x = rng.normal(size=(1, 8, 8, 16))
    target = rng.normal(size=(1, 8, 8, 2))
    return params, x, target


def test_conv_matches_direct_definition():
    # out[y, x, o] = sum over the 3x3 window of in * w, zero padding: checked element by element
    rng = np.random.default_rng(1)
    x = rng.normal(size=(1, 5, 6, 3))
    W = rng.normal(size=(4, 9, 3))
    b = rng.normal(size=4)
    out = unet.conv(x, W, b)
    for (yy, xx, o) in [(0, 0, 0), (2, 3, 1), (4, 5, 3), (1, 0, 2)]:
        s = b[o]
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                t = (dy + 1) * 3 + (dx + 1)
                if 0 <= yy + dy < 5 and 0 <= xx + dx < 6:
                    s += x[0, yy + dy, xx + dx] @ W[o, t]
        assert out[0, yy, xx, o] == pytest.approx(s, rel=1e-12, abs=1e-12)


def test_gradients_match_finite_differences():
    params, x, target = _small_case()
    lval, grad = unet.loss_and_grad(params, x, target)
    rng = np.random.default_rng(2)
    offs, head, total = unet.layout()
    # a few entries of every layer's weights and biases, and of the head
    idx = []
    for (wo, bo), (_, cout, _, _) in zip(offs, unet.SPECS):
        idx += list(rng.integers(wo, bo, 2)) + [int(rng.integers(bo, bo + cout))]
    idx += list(range(head, total, 13))
    h = 1e-6
    for i in idx:
        p1 = params.copy()
        p1[i] += h
        p2 = params.copy()
        p2[i] -= h
        fd = (unet.loss_and_grad(p1, x, target)[0] - unet.loss_and_grad(p2, x, target)[0]) / (2 * h)
        assert grad[i] == pytest.approx(fd, rel=1e-5, abs=1e-8), i


def test_pool_and_upsample_are_adjoint_pairs():
    rng = np.random.default_rng(3)
    a = rng.normal(size=(2, 8, 6, 3))
    b = rng.normal(size=(2, 4, 3, 3))
    assert np.sum(unet.pool(a) * b) == pytest.approx(np.sum(a * unet.pool_bwd(b)))
    assert np.sum(unet.up(b) * a) == pytest.approx(np.sum(b * unet.up_bwd(a)))
