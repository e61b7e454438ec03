"""Learned preconditioner pipeline on the GPU: training pairs from the FDTD/adjoint kernels,
a few U-Net training steps, and the misfit-guarded learned step inside FWI."""
import numpy as np
import pytest
import torch

from paper_2506_20513_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NT = 400


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def setup(dev):
    from paper_2506_20513_gb300 import FDTD
    from paper_2506_20513_gb300.fdtd import ricker
    from paper_2506_20513_gb300.precond import PreconditionerScales, generate_pairs, seeded_models
    wl = W.preconditioner_model(7000, nt=NT)
    g = wl.grid
    fd = FDTD(g, wl.src, wl.rec, device=dev)
    wav = torch.tensor(ricker(wl.f0, g.dt, g.nt), device=dev)
    seeds = list(range(7000, 7006))
    X, T, _ = generate_pairs(fd, seeded_models(seeds, NT), len(seeds), wav,
                             PreconditionerScales(), g.npml)
    return fd, wl, wav, seeds, X, T


def test_training_pairs(setup):
    fd, wl, wav, seeds, X, T = setup
    p = wl.grid.npml
    assert X.shape == (6, 128, 256, 4) and T.shape == (6, 128, 256, 2)
    assert torch.isfinite(X).all() and torch.isfinite(T).all()
    for i, s in enumerate(seeds):
        w = W.preconditioner_model(s, nt=NT)
        de = (w.eps_true - w.eps_init)[p:-p, p:-p]
        ds = (w.sig_true - w.sig_init)[p:-p, p:-p] / 1e-2
        np.testing.assert_allclose(T[i, ..., 0].cpu().numpy(), de, rtol=1e-5, atol=1e-5)
        np.testing.assert_allclose(T[i, ..., 1].cpu().numpy(), ds, rtol=1e-4, atol=1e-5)
        np.testing.assert_allclose(X[i, ..., 2].cpu().numpy(), w.eps_init[p:-p, p:-p] / 10.0,
                                   rtol=1e-6)
        for c in (0, 1):
            assert float(X[i, ..., c].abs().max()) == pytest.approx(1.0, rel=1e-6)
        assert float(X[i, ..., 3].max()) == pytest.approx(1.0, rel=1e-6)
        assert float(X[i, ..., 3].min()) >= 0.0


def test_training_and_guarded_fwi_step(setup, dev):
    from paper_2506_20513_gb300.fwi import FWI, FWIConfig, interior_mask
    from paper_2506_20513_gb300.precond import LearnedPreconditioner, train
    from paper_2506_20513_gb300.unet import UNet
    fd, wl, wav, seeds, X, T = setup
    net = UNet(4, 32, 4, 2, 128, 256, max_batch=2, device=dev)
    net.init_params(3)
    losses = train(net, X, T, epochs=3, batch=2, lr=1e-3, seed=1)
    assert all(np.isfinite(losses))
    assert net.kernel_launches > 0
    pre = LearnedPreconditioner(net, wl.grid.npml)
    de, ds = pre.update(*(torch.zeros(fd.shape, device=dev) for _ in range(2)),
                        torch.tensor(wl.eps_init, dtype=torch.float32, device=dev),
                        torch.ones(fd.shape, device=dev))
    p = wl.grid.npml
    assert de.shape == fd.shape and not de[:p].any() and not ds[:, :p].any()
    obs = fd.forward_model(torch.tensor(wl.eps_true, dtype=torch.float32, device=dev),
                           torch.tensor(wl.sig_true, dtype=torch.float32, device=dev), wav)
    inv = FWI(fd, lambda f: obs, interior_mask(wl.grid, 4), FWIConfig(bands=((wl.f0, 3),)),
              preconditioner=pre)
    e0 = torch.tensor(wl.eps_init, dtype=torch.float32, device=dev)
    s0 = torch.tensor(wl.sig_init, dtype=torch.float32, device=dev)
    _, _, hist = inv.run(e0, s0)
    assert len(hist.misfit) >= 1 and len(hist.learned) == len(hist.misfit)
    seq = hist.misfit + [hist.final_misfit]
    assert all(b <= a for a, b in zip(seq, seq[1:]))   # every kept step lowers J
