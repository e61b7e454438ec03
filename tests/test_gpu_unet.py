"""Parity of the BF16 U-Net kernels (through the C ABI) with the FP64 oracle.

Two comparisons per case:

* tight, against the oracle with BF16 storage rounding (``quantize=bf16``: input, weights,
  stored activations and the gradients fed to products rounded as the kernels store them,
  so ReLU masks and max-pool choices are taken on the same values).  What remains is FP32
  accumulation against FP64 sums, which only rarely moves a stored value to the neighbouring
  BF16 number: rel-L2 <= 1e-2 for outputs, loss and every parameter block, 3e-2 for the first
  layer's weights (their sum over every cell cancels to a few per cent of its terms; 1.4%
  measured at 128 x 256);
* loose, against the plain FP64 oracle.  The BF16 roundings themselves (relative 2^-9 each)
  move outputs by < 1e-2 and gradient blocks by up to 6% (18% for the first layer's weights,
  whose sum over all cells cancels heavily), as the rounded oracle shows on these cases:
  rel-L2 <= 3e-2 for outputs and loss, 0.1 per block, 0.25 for the first layer's weights.
"""
import numpy as np
import pytest
import torch

from oracle import unet_oracle as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def make(dev, levels, base, cin, cout, H, W, n, seed, gemm=0):
    from paper_2506_20513_gb300.unet import UNet
    net = UNet(levels, base, cin, cout, H, W, max_batch=n, device=dev)
    net.set_gemm(gemm)
    p = net.init_params(seed).cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(seed + 1)
    x = rng.standard_normal((n, H, W, cin)).astype(np.float32)
    t = rng.standard_normal((n, H, W, cout)).astype(np.float32)
    mask = (rng.random((n, H, W)) > 0.25).astype(np.float32)
    return net, p, x, t, mask


def check_blocks(g_gpu, g_ref, levels, base, cin, cout, tol, tol_first=None):
    off = 0
    worst = 0.0
    for name, k, ci, co in U.layer_shapes(levels, base, cin, cout):
        nw = k * k * ci * co
        for part, sl in (("W", slice(off, off + nw)), ("b", slice(off + nw, off + nw + co))):
            r = rel(g_gpu[sl], g_ref[sl])
            worst = max(worst, r)
            lim = tol_first if (tol_first and name == "enc0a" and part == "W") else tol
            assert r <= lim, (name, part, r)
        off += nw + co
    return worst


def compare(net, p, x, t, mask, dev, levels, base, cin, cout):
    xd, td, md = (torch.from_numpy(a).to(dev) for a in (x, t, mask))
    y = net.forward(xd).cpu().numpy()
    loss, g = net.loss_and_grad(xd, td, md, grads=True)
    L, g = float(loss.item()), g.cpu().numpy()
    # tight: same storage rounding
    yq = U.forward(p, x, levels, base, cin, cout, quantize=U.bf16)
    Lq, gq, _ = U.loss_and_gradient(p, x, t, mask, levels, base, cin, cout, quantize=U.bf16)
    assert rel(y, yq) <= 1e-2
    assert L == pytest.approx(Lq, rel=1e-2)
    check_blocks(g, gq, levels, base, cin, cout, 1e-2, tol_first=3e-2)
    # loose: plain FP64
    y0 = U.forward(p, x, levels, base, cin, cout)
    L0, g0, _ = U.loss_and_gradient(p, x, t, mask, levels, base, cin, cout)
    assert rel(y, y0) <= 3e-2
    assert L == pytest.approx(L0, rel=3e-2)
    check_blocks(g, g0, levels, base, cin, cout, 0.1, tol_first=0.25)
    net.status()
    return y


@pytest.mark.parametrize("gemm", [0, 1, 2], ids=["mma_sync", "tcgen05_tma", "tcgen05"])
@pytest.mark.parametrize("levels,base,cin,cout,H,W,n", [
    (3, 8, 4, 2, 24, 44, 2),    # ragged GEMM tiles (2112 rows), narrow channels
    (2, 16, 3, 5, 10, 14, 3),   # odd cin / cout: scalar staging paths
    (1, 8, 4, 2, 9, 7, 1),      # one level: no pooling, no decoder
])
def test_unet_forward_loss_and_gradient_match_oracle(dev, levels, base, cin, cout, H, W, n, gemm):
    net, p, x, t, mask = make(dev, levels, base, cin, cout, H, W, n, seed=100 + levels, gemm=gemm)
    compare(net, p, x, t, mask, dev, levels, base, cin, cout)


@pytest.mark.parametrize("gemm", [0, 1, 2], ids=["mma_sync", "tcgen05_tma", "tcgen05"])
def test_unet_full_size_matches_oracle(dev, gemm):
    """The preconditioner's network: 4 levels, 32 base channels, 4 in / 2 out, 128 x 256."""
    levels, base, cin, cout, H, W, n = 4, 32, 4, 2, 128, 256, 2
    net, p, x, t, mask = make(dev, levels, base, cin, cout, H, W, n, seed=7, gemm=gemm)
    y = compare(net, p, x, t, mask, dev, levels, base, cin, cout)
    # a batch of one gives the first image's own result
    xd = torch.from_numpy(x).to(dev)
    y1 = net.forward(xd[:1].contiguous()).cpu().numpy()
    np.testing.assert_array_equal(y1, y[:1])


def test_unet_gemm_engines_agree(dev):
    """tcgen05 and mma.sync products of the full network: same result up to FP32 summation
    order (which can move a stored BF16 activation by one unit in the last place)."""
    levels, base, cin, cout, H, W, n = 4, 32, 4, 2, 128, 256, 4
    net, p, x, t, mask = make(dev, levels, base, cin, cout, H, W, n, seed=9, gemm=0)
    xd, td = torch.from_numpy(x).to(dev), torch.from_numpy(t).to(dev)
    y0 = net.forward(xd).clone()
    _, g0 = net.loss_and_grad(xd, td, grads=True)
    for mode in (1, 2):
        net.set_gemm(mode)
        y1 = net.forward(xd).clone()
        _, g1 = net.loss_and_grad(xd, td, grads=True)
        net.status()
        assert rel(y1.cpu().numpy(), y0.cpu().numpy()) <= 2e-3
        assert rel(g1.cpu().numpy(), g0.cpu().numpy()) <= 1e-2


def test_unet_gradient_is_deterministic_and_adam_matches_oracle(dev):
    levels, base, cin, cout, H, W, n = 3, 8, 4, 2, 16, 24, 2
    net, p, x, t, mask = make(dev, levels, base, cin, cout, H, W, n, seed=11)
    xd, td, md = (torch.from_numpy(a).to(dev) for a in (x, t, mask))
    _, g1 = net.loss_and_grad(xd, td, md, grads=True)
    _, g2 = net.loss_and_grad(xd, td, md, grads=True)
    assert torch.equal(g1, g2)
    w0 = net.get_params().cpu().numpy().astype(np.float64)
    g = g1.cpu().numpy().astype(np.float64)
    m = np.zeros_like(w0)
    v = np.zeros_like(w0)
    for step in (1, 2):
        net.adam_step(1e-2)
        w0, m, v = U.adam_step(w0, g, m, v, step, 1e-2)
        np.testing.assert_allclose(net.get_params().cpu().numpy(), w0, rtol=1e-5, atol=1e-6)


def test_unet_mask_and_errors(dev):
    from paper_2506_20513_gb300 import _lib
    net, p, x, t, mask = make(dev, 2, 8, 4, 2, 8, 8, 2, seed=3)
    xd, td = torch.from_numpy(x).to(dev), torch.from_numpy(t).to(dev)
    loss, g = net.loss_and_grad(xd, td, torch.zeros(2, 8, 8, device=dev), grads=True)
    assert float(loss.item()) == 0.0 and not g.any()
    with pytest.raises(ValueError):
        net.forward(torch.zeros(3, 8, 8, 4, device=dev))
    rc = net.lib.gf_unet_forward(net._net, 3, xd.data_ptr(), xd.data_ptr(), None)
    assert rc == _lib.GF_EINVAL
    fresh = type(net)(2, 8, 4, 2, 8, 8, max_batch=1, device=dev)
    with pytest.raises(_lib.GfError) as e:
        fresh.adam_step(1e-3)
    assert e.value.code == _lib.GF_ESTATE


def test_unet_training_reduces_loss(dev):
    """Adam on a fixed smooth target: the loss falls well below its start."""
    from paper_2506_20513_gb300.unet import UNet
    net = UNet(3, 8, 4, 2, 32, 32, max_batch=4, device=dev)
    net.init_params(5)
    g = torch.Generator().manual_seed(5)
    x = torch.randn(4, 32, 32, 4, generator=g).to(dev)
    t = (0.5 * x[..., :2] - 0.25 * x[..., 2:]).contiguous()
    first = None
    for _ in range(150):
        loss = net.train_step(x, t, lr=3e-3)
        first = float(loss.item()) if first is None else first
    assert float(loss.item()) < 0.3 * first


def test_unet_expired_wait_reports_timeout_and_recovers(dev):
    """Make every tensor-core GEMM wait give up after one poll (a host-side budget, no fault):
    the call completes, gf_unet_status reports GF_ETIMEOUT once, and with the normal budget
    the next call is correct again."""
    from paper_2506_20513_gb300 import _lib
    levels, base, cin, cout, H, W, n = 3, 16, 4, 2, 32, 64, 2
    net, p, x, t, mask = make(dev, levels, base, cin, cout, H, W, n, seed=12, gemm=1)
    xd = torch.from_numpy(x).to(dev)
    y_ref = net.forward(xd).clone()
    net.status()
    net.set_wait_budget(64)
    net.forward(xd)
    with pytest.raises(_lib.GfError) as e:
        net.status()
    assert e.value.code == _lib.GF_ETIMEOUT
    net.set_wait_budget(0)
    y = net.forward(xd)
    net.status()
    assert torch.equal(y, y_ref)
