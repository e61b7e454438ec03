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


def test_stage_pairs_at_the_updated_model(setup, dev):
    """Pairs for a second network: features and target at the model the first network's
    update reaches (masked below the top rows, eps_r >= 1), with the start model's
    illumination."""
    from paper_2506_20513_gb300.fwi import interior_mask
    from paper_2506_20513_gb300.precond import (LearnedPreconditioner, PreconditionerScales,
                                                generate_stage_pairs, seeded_models)
    from paper_2506_20513_gb300.unet import UNet
    fd, wl, wav, seeds, X, T = setup
    g = wl.grid
    p = g.npml
    net = UNet(4, 32, 4, 2, 128, 256, max_batch=2, device=dev)
    net.init_params(11)
    pre = LearnedPreconditioner(net, p)
    n = 3
    X2, T2, _ = generate_stage_pairs(fd, seeded_models(seeds[:n], NT), n, wav,
                                     PreconditionerScales(), p, pre, interior_mask(g, 4))
    assert X2.shape == (n, 128, 256, 4) and T2.shape == (n, 128, 256, 2)
    assert torch.isfinite(X2).all() and torch.isfinite(T2).all()
    for i, s in enumerate(seeds[:n]):
        w = W.preconditioner_model(s, nt=NT)
        e1 = X2[i, ..., 2].double().cpu().numpy() * 10.0
        e0 = w.eps_init[p:-p, p:-p]
        # the update leaves the masked top rows alone and keeps eps_r >= 1
        np.testing.assert_allclose(e1[:4], e0[:4], rtol=1e-6)
        assert e1.min() >= 1.0 - 1e-6
        assert np.abs(e1[4:] - e0[4:]).max() > 1e-3
        # target: the truth minus the updated model
        np.testing.assert_allclose(T2[i, ..., 0].cpu().numpy(), w.eps_true[p:-p, p:-p] - e1,
                                   rtol=1e-5, atol=2e-5)
        # the gradient is taken at the updated model, the illumination at the start model
        assert not torch.equal(X2[i, ..., 0], X[i, ..., 0])
        torch.testing.assert_close(X2[i, ..., 3], X[i, ..., 3], rtol=1e-5, atol=1e-6)


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


def test_trained_network_gains_on_held_out_models(dev):
    """What the trained network gains over plain L-BFGS, on the preconditioner workload
    (256 x 128 cells + 20-cell CPML, 16 shots, 64 receivers, nt 1500): the U-Net is trained
    here on 1500 seeded models (pairs from the FDTD/adjoint kernels, 30 epochs of the
    library's BF16 training kernels), then on 12 held-out models plain L-BFGS runs 50
    iterations and sets the target misfit, and the learned run (network update tried first,
    plain step as fallback) runs until it reaches that misfit.  At the median over the
    held-out models the learned run needs at most 3/4 of the plain run's forward-equivalent
    FDTD time loops (a misfit-only evaluation 1, a gradient 2; measured 56.5 against 108.5)
    and fewer iterations and less time, and at least 8 of the 12 models reach the target
    (measured 10)."""
    import time

    from paper_2506_20513_gb300 import FDTD
    from paper_2506_20513_gb300.fdtd import ricker
    from paper_2506_20513_gb300.fwi import FWI, FWIConfig, interior_mask
    from paper_2506_20513_gb300.precond import (LearnedPreconditioner, PreconditionerScales,
                                                generate_pairs, pair_fractions, seeded_models,
                                                train)
    from paper_2506_20513_gb300.unet import UNet
    nt = 1500
    first = W.preconditioner_model(100000, nt=nt)
    g = first.grid
    fd = FDTD(g, first.src, first.rec, device=dev)
    wav = torch.tensor(ricker(first.f0, g.dt, g.nt), device=dev)
    seeds = np.arange(100000, 101500)
    # the host-side model generation runs in 4 spawned processes, overlapping the GPU work
    X, T, _ = generate_pairs(fd, seeded_models(seeds, nt, workers=4), len(seeds), wav,
                             PreconditionerScales(), g.npml, fractions=pair_fractions(seeds))
    net = UNet(4, 32, 4, 2, g.ny - 2 * g.npml, g.nx - 2 * g.npml, max_batch=16, device=dev)
    net.init_params(5)
    losses = train(net, X, T, epochs=30, batch=16, lr=1e-3, seed=5, decay_every=10)
    del X, T
    assert losses[-1] < 0.5 * losses[0]
    pre = LearnedPreconditioner(net, g.npml)
    mask = interior_mask(g, rows_below_top=4)
    t32 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    rows = []
    for s in range(1100000, 1100012):
        w = W.preconditioner_model(s, nt=nt)
        obs = fd.forward_model(t32(w.eps_true), t32(w.sig_true), wav)
        runs = []
        for p in (None, pre):
            inv = FWI(fd, lambda f: obs, mask, FWIConfig(bands=((w.f0, 50),)), preconditioner=p)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            _, _, h = inv.run(t32(w.eps_init), t32(w.sig_init),
                              stop_misfit=runs[0][0] if p is not None else None)
            torch.cuda.synchronize(dev)
            runs.append((h.final_misfit, sum(h.passes), len(h.misfit), sum(h.evaluations),
                         time.perf_counter() - t0))
        rows.append(runs)
    fd.status()
    reached = sum(r[1][0] <= r[0][0] for r in rows)
    med = lambda k, i: float(np.median([r[k][i] for r in rows]))
    print(f"\ntrain loss {losses[0]:.3f} -> {losses[-1]:.3f}; reached {reached}/12; median "
          f"passes {med(0, 1)} -> {med(1, 1)}, iterations {med(0, 2)} -> {med(1, 2)}, "
          f"evaluations {med(0, 3)} -> {med(1, 3)}, seconds {med(0, 4):.3f} -> {med(1, 4):.3f}")
    assert reached >= 8
    assert med(1, 1) <= 0.75 * med(0, 1)
    assert med(1, 2) < med(0, 2)
    assert med(1, 4) < med(0, 4)
    net.close()
    fd.close()
