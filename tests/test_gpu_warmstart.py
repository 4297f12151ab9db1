"""The learned warm start: network kernels against the FP64 reference network, training, and
the gain over the cold start."""
import numpy as np
import pytest

import gabp_synth
from gpu_common import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _bf16_round(a):
    """Round float32 values to BF16 (round to nearest even), returned as float64."""
    a = np.ascontiguousarray(a, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _to_bf16_bits(a):
    a = np.ascontiguousarray(a, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    return (((u + 0x7FFF + ((u >> 16) & 1)) >> 16) & 0xFFFF).astype(np.uint16)


def _case(torch, H=16, W=24, B=2, seed=0, learnable=False):
    rng = np.random.default_rng(seed)
    x = np.zeros((B, H, W, 16), np.float32)
    x[..., 0] = rng.normal(size=(B, H, W)) * (rng.random((B, H, W)) < 0.2)
    x[..., 1] = (x[..., 0] != 0)
    x[..., 2] = rng.normal(size=(B, 1, 1))
    if learnable:   # a function of the inputs the network can represent
        t = np.stack([3.0 * x[..., 0] + 1.0, x[..., 2] + x[..., 1]], axis=-1).astype(np.float32)
    else:
        t = rng.normal(size=(B, H, W, 2)).astype(np.float32)
    dev = torch.device("cuda", 0)
    xs = [torch.tensor(_to_bf16_bits(x[b]).view(np.int16), device=dev) for b in range(B)]
    ts = [torch.tensor(t[b], device=dev) for b in range(B)]
    return x, t, xs, ts


def test_network_forward_and_gradients_match_reference():
    torch = pytest.importorskip("torch")
    from oracle import unet
    from paper_2404_12968_gb300 import WarmStartNet, gabp_wsnet_forward, gabp_wsnet_gradients

    net = WarmStartNet(seed=3, device=0)
    rng = np.random.default_rng(4)
    params = net.params().astype(np.float64)
    # random biases and head too, so every path carries signal
    _, head, total = unet.layout()
    params += rng.normal(size=total) * 0.02
    net.set_params(params.astype(np.float32))
    H, W, B = 16, 24, 2
    x, t, xs, ts = _case(torch, H, W, B)
    # the network computes with BF16 weights and inputs: give the reference the same values
    p_ref = params.copy()
    offs, head, _ = unet.layout()
    for (wo, bo) in offs:
        p_ref[wo:bo] = _bf16_round(params[wo:bo])
    x_ref = _bf16_round(x).reshape(B, H, W, 16)
    out_ref, _ = unet.forward(p_ref, x_ref)
    out = np.empty((B, H, W, 2), np.float32)
    xb = torch.stack(xs).contiguous()
    gabp_wsnet_forward(net.handle, xb, B, H, W, out)
    rel = np.linalg.norm(out - out_ref) / np.linalg.norm(out_ref)
    assert rel < 3e-2, rel     # BF16 activations between layers
    loss_ref, g_ref = unet.loss_and_grad(p_ref, x_ref, t.astype(np.float64))
    g = np.empty(total, np.float32)
    loss = gabp_wsnet_gradients(net.handle, xs, ts, H, W, g)
    assert loss == pytest.approx(loss_ref, rel=3e-2)
    # per layer: weight and bias gradients within BF16 accuracy of the reference
    for i, (wo, bo) in enumerate(offs):
        cout = unet.SPECS[i][1]
        for a, b in [(wo, bo), (bo, bo + cout)]:
            gr, gg = g_ref[a:b], g[a:b]
            if i == 0 and b == bo:
                # layer 0 reads input channels 0..2 only; the zero channels carry no signal
                mask = (np.arange(b - a) % 16) < 3
                gr, gg = gr[mask], gg[mask]
            e = np.linalg.norm(gg - gr) / (np.linalg.norm(gr) + 1e-12)
            assert e < 6e-2, (i, a, e)
    e = np.linalg.norm(g[head:] - g_ref[head:]) / np.linalg.norm(g_ref[head:])
    assert e < 3e-2
    net.close()


@pytest.mark.parametrize("B,H,W", [(2, 40, 72), (1, 64, 64)])
def test_tensor_core_gradients_match_mma_sync_gradients(B, H, W):
    """Training gradients with the tcgen05 kernels (forward, backward-data and weight-gradient
    convolutions) against the mma.sync kernels of the same network: the same BF16 arithmetic
    up to the accumulation order, per layer within the BF16 bar of the reference comparison;
    the bias gradients are the same kernel on both."""
    torch = pytest.importorskip("torch")
    from oracle import unet
    from paper_2404_12968_gb300 import (GABP_WSNET_MMA_SYNC, GABP_WSNET_TCGEN05, WarmStartNet,
                                        gabp_wsnet_gradients, gabp_wsnet_set_kernels)
    net = WarmStartNet(seed=7, device=0)
    rng = np.random.default_rng(8)
    offs, head, total = unet.layout()
    net.set_params((net.params() + rng.normal(size=total) * 0.02).astype(np.float32))
    _, _, xs, ts = _case(torch, H, W, B, seed=10)
    grads, losses = {}, {}
    for k in (GABP_WSNET_TCGEN05, GABP_WSNET_MMA_SYNC):
        gabp_wsnet_set_kernels(net.handle, k)
        g = np.empty(total, np.float32)
        losses[k] = gabp_wsnet_gradients(net.handle, xs, ts, H, W, g)
        grads[k] = g
    net.close()
    a, b = grads[GABP_WSNET_TCGEN05], grads[GABP_WSNET_MMA_SYNC]
    assert np.all(np.isfinite(a))
    assert losses[GABP_WSNET_TCGEN05] == pytest.approx(losses[GABP_WSNET_MMA_SYNC], rel=1e-2)
    for i, (wo, bo) in enumerate(offs):
        e = np.linalg.norm(a[wo:bo] - b[wo:bo]) / (np.linalg.norm(b[wo:bo]) + 1e-12)
        assert e < 6e-2, (i, e)


@pytest.mark.parametrize("B,H,W", [(2, 40, 72), (1, 64, 64), (3, 16, 24)])
def test_tensor_core_forward_matches_mma_sync_forward(B, H, W):
    """The tcgen05 forward (fused pooling, upsampling additions and head) against the mma.sync
    forward of the same network: the same BF16 arithmetic up to the accumulation order.  The
    shapes give partial 16 x 8 tiles at every level, several output-channel blocks (Cout 256),
    and batches."""
    torch = pytest.importorskip("torch")
    from oracle import unet
    from paper_2404_12968_gb300 import (GABP_WSNET_MMA_SYNC, GABP_WSNET_TCGEN05, WarmStartNet, gabp_wsnet_forward,
                                        gabp_wsnet_set_kernels)
    net = WarmStartNet(seed=5, device=0)
    rng = np.random.default_rng(6)
    _, _, total = unet.layout()
    net.set_params((net.params() + rng.normal(size=total) * 0.02).astype(np.float32))
    _, _, xs, _ = _case(torch, H, W, B, seed=9)
    xb = torch.stack(xs).contiguous()
    outs = {}
    for k in (GABP_WSNET_TCGEN05, GABP_WSNET_MMA_SYNC):
        gabp_wsnet_set_kernels(net.handle, k)
        o = np.empty((B, H, W, 2), np.float32)
        gabp_wsnet_forward(net.handle, xb, B, H, W, o)
        outs[k] = o
    a, b = outs[GABP_WSNET_TCGEN05], outs[GABP_WSNET_MMA_SYNC]
    assert np.all(np.isfinite(a))
    rel = np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel < 1e-2, rel
    net.close()


def test_training_reduces_loss():
    torch = pytest.importorskip("torch")
    from paper_2404_12968_gb300 import WarmStartNet, gabp_wsnet_train_step
    net = WarmStartNet(seed=1, device=0)
    _, _, xs, ts = _case(torch, 32, 32, 4, seed=7, learnable=True)
    first = gabp_wsnet_train_step(net.handle, xs, ts, 32, 32, 1e-3)
    for _ in range(80):
        last = gabp_wsnet_train_step(net.handle, xs, ts, 32, 32, 1e-3)
    assert last < 0.3 * first, (first, last)
    net.close()


def test_learned_warm_start_sets_beliefs_from_the_network():
    torch = pytest.importorskip("torch")
    from paper_2404_12968_gb300 import Solver, WarmStartNet, gabp_wsnet_forward, gabp_wsnet_input_shape, gabp_wsnet_sample
    p = gabp_synth.scaled_config(100, 0.05, 3, 6)
    net = WarmStartNet(seed=2, device=0)
    with Solver(p, precision="fp32") as s:
        H, W, scale = gabp_wsnet_input_shape(s.ctx)
        assert (H, W) == (104, 104)
        dev = torch.device("cuda", 0)
        x = torch.zeros((H, W, 16), dtype=torch.int16, device=dev)
        gabp_wsnet_sample(s.ctx, x, None)
        xh = x.cpu().numpy().astype(np.uint16).astype(np.uint32) << 16
        xf = xh.view(np.float32)
        assert set(np.unique(xf[..., 1])) <= {0.0, 1.0} and xf[..., 1].sum() > 0
        assert np.allclose(xf[:100, :100, 2], np.log(0.05) + 3, atol=1e-2)
        assert np.all(xf[..., 3:] == 0)
        out = np.empty((1, H, W, 2), np.float32)
        gabp_wsnet_forward(net.handle, x, 1, H, W, out)
        s.learned_warm_start(net)
        mu, var = s.marginals()
        exp_mu = scale * out[0, :100, :100, 0].reshape(-1)
        exp_lam = np.exp(np.clip(out[0, :100, :100, 1].astype(np.float64), -10, 15)).reshape(-1)
        np.testing.assert_allclose(mu, exp_mu, rtol=1e-5, atol=1e-6 * scale)
        np.testing.assert_allclose(1.0 / var, exp_lam, rtol=1e-5)
        s.iterate(50, 0.3)
        assert np.isfinite(s.residual())
    net.close()
