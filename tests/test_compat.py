"""The paper-shaped compute(...) entry point: geometry on the CPU (Table values of the
cross-hole example, Sec. 4), traces and autograd gradients on the GPU against the direct
FDTD calls."""
import numpy as np
import pytest
import torch

from paper_2506_20513_gb300.compat import paper_geometry

TABLE = dict(dx=0.05, dy=0.05, nx=220, ny=120, source_location=[0.5, 0.5, 0],
             source_step=[0.25, 0, 0], receiver_location=[0.5, 5.5, 0],
             receiver_step=[0.05, 0, 0], step=40, nsrc=1, nrx=200)


def test_geometry_of_the_cross_hole_table():
    src, rec = paper_geometry(**TABLE)
    assert src.shape == (40, 1, 2) and rec.shape == (40, 200, 2)
    np.testing.assert_array_equal(src[:, 0, 0], 10 + 5 * np.arange(40))   # 0.5 m + s 0.25 m
    assert (src[:, 0, 1] == 10).all()
    np.testing.assert_array_equal(rec[0, :, 0], 10 + np.arange(200))      # 0.5 m + r 0.05 m
    assert (rec[..., 1] == 110).all()                                       # 5.5 m
    assert (rec == rec[0]).all()                                            # same line every shot


def test_geometry_rejects_points_outside_the_grid():
    bad = dict(TABLE, source_step=[0.3, 0, 0])   # shot 39 at 12.2 m > 10.9 m
    with pytest.raises(ValueError):
        paper_geometry(**bad)
    with pytest.raises(ValueError):
        paper_geometry(**dict(TABLE, nsrc=2))


@pytest.mark.gpu
def test_compute_matches_the_library_and_differentiates():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_20513_gb300 import FDTD
    from paper_2506_20513_gb300.compat import compute
    from paper_2506_20513_gb300.fdtd import ricker
    from paper_2506_20513_gb300.workloads import GridSpec, default_pml
    dev = torch.device("cuda:0")
    nx, ny, pml, dx, dt, f0 = 60, 40, 8, 0.02, 4e-11, 4e8
    rng = np.random.default_rng(3)
    eps = torch.tensor(4 + 3 * rng.random((nx, ny, 1)), dtype=torch.float32, device=dev)
    sig = torch.tensor(1e-3 + 1e-2 * rng.random((nx, ny, 1)), dtype=torch.float32, device=dev)
    eps.requires_grad_()
    sig.requires_grad_()
    args = dict(device="cuda", dx=dx, ny=ny, nx=nx, nz=1, time_windows=200 * dt,
                source=["hertzian", "z"], source_location=[0.2, 0.2, 0],
                source_step=[0.2, 0, 0], receiver_location=[0.2, 0.6, 0],
                receiver_step=[0.04, 0, 0], pmlthick=pml, source_amplitudes=["ricker", 2.0, f0],
                step=3, epsilon=eps, sigma=sig, miu=1, nsrc=1, nrx=20, freq=None, dt=dt)
    tr, t = compute(**args)
    assert tr.shape == (3, 200, 20) and t.shape == (200,)
    (0.5 * (tr ** 2).sum()).backward()
    # the same run through the FDTD object, in its own layout
    src, rec = paper_geometry(dx, dx, nx, ny, [0.2, 0.2, 0], [0.2, 0, 0], [0.2, 0.6, 0],
                              [0.04, 0, 0], 3, 1, 20)
    g = default_pml(GridSpec(nx=nx, ny=ny, npml=pml, nt=200, dx=dx, dy=dx, dt=dt), f0)
    fd = FDTD(g, src, rec, device=dev)
    wav = torch.tensor(2.0 * ricker(f0, dt, 200), device=dev)
    e2 = eps.detach()[:, :, 0].T.contiguous()
    s2 = sig.detach()[:, :, 0].T.contiguous()
    tr2 = fd.forward_model(e2, s2, wav)
    torch.testing.assert_close(tr.detach(), tr2, rtol=1e-6, atol=1e-6 * float(tr2.abs().max()))
    zero = torch.zeros_like(tr2)
    _, ge, gs = fd.misfit_and_gradient(e2, s2, wav, zero)
    torch.testing.assert_close(eps.grad[:, :, 0].T, ge, rtol=1e-5, atol=1e-6 * float(ge.abs().max()))
    torch.testing.assert_close(sig.grad[:, :, 0].T, gs, rtol=1e-5, atol=1e-6 * float(gs.abs().max()))


@pytest.mark.gpu
def test_paper_demo_loop_with_adam_reduces_the_loss():
    """The paper's demo loop (Sec. 3.1): compute(...) inside torch.optim.Adam with separate
    learning rates for eps_r and sigma, MSE loss, gradients zeroed near the sources, values
    clamped to physical ranges; a few epochs lower the loss."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_20513_gb300.compat import compute
    from paper_2506_20513_gb300 import workloads as W
    dev = torch.device("cuda:0")
    nx, ny, pml, dx, dt, f0 = 80, 50, 10, 0.02, 4e-11, 4e8
    eps_true, sig_true = W.layered_blob_model(5, nx - 2 * pml, ny - 2 * pml, dx)
    eps_true, sig_true = W.pad_edges(eps_true, pml), W.pad_edges(sig_true, pml)
    eps_init = W.pad_edges(W.smooth(eps_true[pml:-pml, pml:-pml], 0.1, dx), pml)
    to_paper = lambda a: torch.tensor(a.T[:, :, None].copy(), dtype=torch.float32, device=dev)
    args = dict(device="cuda", dx=dx, ny=ny, nx=nx, nz=1, time_windows=300 * dt,
                source=["hertzian", "z"], source_location=[0.25, 0.24, 0],
                source_step=[0.2, 0, 0], receiver_location=[0.22, 0.24, 0],
                receiver_step=[0.04, 0, 0], pmlthick=pml, source_amplitudes=["ricker", 1.0, f0],
                step=6, miu=1, nsrc=1, nrx=30, freq=None, dt=dt)
    with torch.no_grad():
        observed, _ = compute(epsilon=to_paper(eps_true), sigma=to_paper(sig_true), **args)
    epsilon = to_paper(eps_init).requires_grad_()
    sigma = to_paper(sig_true).requires_grad_()
    opt = torch.optim.Adam([{"params": epsilon, "lr": 0.05}, {"params": sigma, "lr": 1e-4}])
    mse = torch.nn.MSELoss()
    losses = []
    for _ in range(6):
        opt.zero_grad()
        result, _ = compute(epsilon=epsilon, sigma=sigma, **args)
        loss = mse(result, observed)
        loss.backward()
        epsilon.grad[:, :pml + 1, :] = 0
        sigma.grad[:, :pml + 1, :] = 0
        opt.step()
        with torch.no_grad():
            epsilon.clamp_(min=1.0)
            sigma.clamp_(min=0.0)
        losses.append(float(loss.detach()))
    assert losses[-1] < 0.8 * losses[0]


@pytest.mark.gpu
def test_compute_with_x_and_y_polarised_sources():
    """['hertzian', 'x' | 'y'] runs the TE model: the traces are the source component of
    forward_model_te; asking autograd for gradients is refused (the TE gradient call takes
    observed traces, not a trace cotangent)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_20513_gb300 import FDTD
    from paper_2506_20513_gb300.compat import compute
    from paper_2506_20513_gb300.fdtd import ricker
    from paper_2506_20513_gb300.workloads import GridSpec, default_pml
    dev = torch.device("cuda:0")
    nx, ny, pml, dx, dt, f0 = 60, 40, 8, 0.02, 4e-11, 4e8
    rng = np.random.default_rng(4)
    eps = torch.tensor(4 + 3 * rng.random((nx, ny, 1)), dtype=torch.float32, device=dev)
    sig = torch.tensor(1e-3 + 1e-2 * rng.random((nx, ny, 1)), dtype=torch.float32, device=dev)
    args = dict(device="cuda", dx=dx, ny=ny, nx=nx, nz=1, time_windows=200 * dt,
                source_location=[0.2, 0.2, 0], source_step=[0.2, 0, 0],
                receiver_location=[0.2, 0.6, 0], receiver_step=[0.04, 0, 0], pmlthick=pml,
                source_amplitudes=["ricker", 2.0, f0], step=3, epsilon=eps, sigma=sig, miu=1,
                nsrc=1, nrx=20, freq=None, dt=dt)
    src, rec = paper_geometry(dx, dx, nx, ny, [0.2, 0.2, 0], [0.2, 0, 0], [0.2, 0.6, 0],
                              [0.04, 0, 0], 3, 1, 20)
    g = default_pml(GridSpec(nx=nx, ny=ny, npml=pml, nt=200, dx=dx, dy=dx, dt=dt), f0)
    fd = FDTD(g, src, rec, device=dev)
    wav = torch.tensor(2.0 * ricker(f0, dt, 200), dtype=torch.float32, device=dev)
    e2 = eps[:, :, 0].transpose(0, 1).contiguous()
    s2 = sig[:, :, 0].transpose(0, 1).contiguous()
    for pol, name in ((0, "x"), (1, "y")):
        tr, t = compute(source=["hertzian", name], **args)
        assert tr.shape == (3, 200, 20) and t.shape == (200,)
        ref = fd.forward_model_te(e2, s2, wav, pol)[..., pol]
        assert torch.equal(tr, ref)
        assert float(tr.abs().max()) > 0
    fd.close()
    with pytest.raises(ValueError):
        compute(source=["hertzian", "x"], **dict(args, epsilon=eps.clone().requires_grad_()))
    with pytest.raises(ValueError):
        compute(source=["hertzian", "w"], **args)
