"""FWI driver pieces on the GPU vs the FP64 oracle: the TV term (Algorithm 3), the misfit-only
entry point, the first L-BFGS step, and misfit decrease over a short multiscale run."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fwi_oracle as F  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2506_20513_gb300 import _lib, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_20513_gb300 import build as B
    B.build_library()
    return torch.device("cuda", 0)


def t32(a, dev):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("nx,ny,lam,iters", [(64, 48, 0.05, 30), (37, 29, 0.2, 60), (540, 290, 0.02, 20)])
def test_tv_kernel_matches_oracle(dev, nx, ny, lam, iters):
    rng = np.random.default_rng(nx)
    X = 3 + 9 * rng.random((ny, nx))
    X[ny // 3:, :] += 2.0
    G = rng.standard_normal((ny, nx))
    lib = _lib.load()
    Xd, Gd = t32(X, dev), t32(G, dev)
    scratch = torch.empty(lib.gf_tv_scratch_bytes(nx, ny), dtype=torch.uint8, device=dev)
    rc = lib.gf_tv_gradient(nx, ny, Xd.data_ptr(), Gd.data_ptr(), scratch.data_ptr(), lam, 0.2,
                            iters, 0.3, None)
    assert rc == 0, lib.gf_last_error(None)
    torch.cuda.synchronize()
    ref = F.tv_gradient(X, G, lam, 0.2, iters, 0.3)
    assert rel(Gd.cpu().numpy() - G, ref - G) <= 1e-4


def test_misfit_entry_point(dev):
    from paper_2506_20513_gb300 import FDTD
    wl = W.small_random(50, nxp=50, nyp=30, npml=6, nt=160, nshots=3, nrec=7)
    wav = np.broadcast_to(O.ricker(wl.f0, wl.grid.dt, wl.grid.nt), (3, 1, wl.grid.nt))
    obs = O.forward(wl.grid, wl.eps_true, wl.sig_true, wl.src, wav, wl.rec)
    J64, _, _ = O.misfit_and_gradient(wl.grid, wl.eps_init, wl.sig_init, wl.src, wav, wl.rec, obs)
    fd = FDTD(wl.grid, wl.src, wl.rec, device=dev)
    e, s, w, o = (t32(a, dev) for a in (wl.eps_init, wl.sig_init, wav, obs))
    J = fd.misfit(e, s, w, o)
    fd.status()
    assert abs(J.item() - J64) <= 1e-5 * J64


def _small_fwi_case():
    wl = W.small_random(51, nxp=60, nyp=40, npml=8, nt=260, nshots=4, nrec=12)
    wl.src[:, 0, 1] = wl.grid.npml + 2
    wl.rec[:, :, 1] = wl.grid.npml + 2
    wl.rec[:, :, 0] = wl.grid.npml + np.linspace(2, 57, 12).astype(np.int32)
    return wl


def test_first_lbfgs_step_matches_oracle(dev):
    """The first iteration is a scaled steepest-descent step with Armijo backtracking; replay
    it with oracle gradients and misfits."""
    from paper_2506_20513_gb300 import FDTD
    from paper_2506_20513_gb300.fwi import FWI, FWIConfig, interior_mask
    wl = _small_fwi_case()
    g = wl.grid
    f0 = wl.f0
    wav64 = np.broadcast_to(O.ricker(f0, g.dt, g.nt), (wl.nshots, 1, g.nt))
    obs64 = O.forward(g, wl.eps_true, wl.sig_true, wl.src, wav64, wl.rec)
    fd = FDTD(g, wl.src, wl.rec, device=dev)
    mask = interior_mask(g, rows_below_top=4)
    cfg = FWIConfig(bands=((f0, 1),), sigma_ref=1e-2, first_step=0.03)
    drv = FWI(fd, lambda f: t32(obs64, dev), mask, cfg)
    eps1, sig1, hist = drv.run(t32(wl.eps_init, dev), t32(wl.sig_init, dev))
    # oracle replay
    m = mask.numpy().astype(np.float64)
    J0, ge, gs = O.misfit_and_gradient(g, wl.eps_init, wl.sig_init, wl.src, wav64, wl.rec, obs64)
    gx = np.concatenate([(ge * m).ravel(), (gs * m * 1e-2).ravel()])
    x0 = np.concatenate([wl.eps_init.ravel(), wl.sig_init.ravel() / 1e-2])
    d = -gx
    n = x0.size // 2
    alpha = 0.03 * x0[:n].max() / np.abs(d[:n]).max()
    evals = 0
    for _ in range(cfg.backtracks):
        x1 = x0 + alpha * d
        e1 = np.maximum(x1[:n], 1.0).reshape(g.ny, g.nx)
        s1 = np.maximum(x1[n:] * 1e-2, 0.0).reshape(g.ny, g.nx)
        d1 = O.forward(g, e1, s1, wl.src, wav64, wl.rec)
        J1 = 0.5 * np.sum((d1 - obs64) ** 2)
        evals += 1
        if J1 <= J0 + cfg.armijo * alpha * np.dot(gx, d):
            break
        alpha *= 0.5
    assert hist.evaluations[0] == evals + 1
    assert abs(hist.misfit[0] - J0) <= 1e-5 * J0
    assert rel(eps1.cpu().numpy(), e1) <= 1e-5
    assert rel(sig1.cpu().numpy(), s1) <= 1e-4
    fd.close()


def test_multiscale_tv_run_decreases_misfit(dev):
    from paper_2506_20513_gb300 import FDTD
    from paper_2506_20513_gb300.fwi import FWI, FWIConfig, interior_mask
    wl = _small_fwi_case()
    g = wl.grid
    fd = FDTD(g, wl.src, wl.rec, device=dev)
    from paper_2506_20513_gb300.fdtd import ricker
    e_t, s_t = t32(wl.eps_true, dev), t32(wl.sig_true, dev)

    def observed(f0):
        w = torch.tensor(ricker(f0, g.dt, g.nt), device=dev)
        return fd.forward_model(e_t, s_t, w)

    cfg = FWIConfig(bands=((150e6, 4), (300e6, 5)), tv=True, tv_lambda=0.02, tv_weight=0.05)
    drv = FWI(fd, observed, interior_mask(g, rows_below_top=4), cfg)
    eps, sig, hist = drv.run(t32(wl.eps_init, dev), t32(wl.sig_init, dev))
    fd.status()
    for band in (150e6, 300e6):
        Js = [J for J, b in zip(hist.misfit, hist.band) if b == band]
        assert len(Js) >= 3
        assert all(b < a for a, b in zip(Js, Js[1:]))
        assert Js[-1] < 0.9 * Js[0]
    m = np.linalg.norm
    e0 = m(wl.eps_init - wl.eps_true)
    assert m(eps.cpu().numpy() - wl.eps_true) < e0
    assert float(eps.min()) >= 1.0 and float(sig.min()) >= 0.0
    fd.close()


def test_checkpoint_resume_is_exact_and_logs(dev, tmp_path):
    """Stop a two-band run after iteration 2 of the second band (state saved every 2
    iterations), resume it from the file in a fresh driver: the final model and the misfit
    history equal those of the uninterrupted run; the JSON log has one line per iteration."""
    import json
    from paper_2506_20513_gb300 import FDTD
    from paper_2506_20513_gb300.fdtd import ricker
    from paper_2506_20513_gb300.fwi import FWI, FWIConfig, interior_mask
    wl = _small_fwi_case()
    g = wl.grid
    fd = FDTD(g, wl.src, wl.rec, device=dev)
    e_t, s_t = t32(wl.eps_true, dev), t32(wl.sig_true, dev)

    def observed(f0):
        return fd.forward_model(e_t, s_t, torch.tensor(ricker(f0, g.dt, g.nt), device=dev))

    cfg = FWIConfig(bands=((150e6, 3), (300e6, 4)), tv=True, tv_lambda=0.02, tv_weight=0.05)
    mask = interior_mask(g, rows_below_top=4)
    e0, s0 = t32(wl.eps_init, dev), t32(wl.sig_init, dev)
    log = tmp_path / "fwi.jsonl"
    eps_a, sig_a, hist_a = FWI(fd, observed, mask, cfg).run(e0, s0, log=str(log))
    lines = [json.loads(l) for l in open(log)]
    assert len(lines) == len(hist_a.misfit) and lines[-1]["band_f0"] == 300e6

    class Stop(Exception):
        pass

    def stop(it, J, x):
        if hist_b_band[0] == 1 and it == 1:
            raise Stop

    ck = tmp_path / "state.pt"
    hist_b_band = [0]

    def observed_b(f0):
        hist_b_band[0] = 0 if f0 == 150e6 else 1
        return observed(f0)

    with pytest.raises(Stop):
        FWI(fd, observed_b, mask, cfg).run(e0, s0, callback=stop, checkpoint=str(ck),
                                          checkpoint_every=2)
    eps_c, sig_c, hist_c = FWI(fd, observed, mask, cfg).run(e0, s0, resume=str(ck))
    assert torch.equal(eps_c, eps_a) and torch.equal(sig_c, sig_a)
    assert hist_c.misfit == hist_a.misfit
    fd.close()
