"""The staged Adam inversion loop (Sec. 2.3 update, Sec. 3.1 loop, Sec. 3.4 staged rates) on
the GPU, replayed against the FP64 oracle: two epochs, the first updating eps_r alone, the
second both parameters, must move the model as Adam's equations applied to the oracle's
gradients do (moments, bias corrections, the per-parameter rates, the mask and the clamps)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2506_20513_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_20513_gb300 import build as B
    B.build_library()
    return torch.device("cuda", 0)


def adam_expected(x, g_list, lr_list, xmin, mask, b1=0.9, b2=0.999, eps=1e-8):
    """Adam's update (Sec. 2.3) written out in FP64 for a sequence of gradients and rates."""
    m = np.zeros_like(x)
    v = np.zeros_like(x)
    for t, (g, lr) in enumerate(zip(g_list, lr_list), start=1):
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        x = np.where(mask != 0, np.maximum(xmin, x - lr * mh / (np.sqrt(vh) + eps)), x)
    return x


def test_two_staged_epochs_replay_the_oracle(dev):
    from paper_2506_20513_gb300 import FDTD
    from paper_2506_20513_gb300.adam import AdamConfig, Stage, StagedAdam
    from paper_2506_20513_gb300.fwi import interior_mask
    wl = W.small_random(41, nxp=64, nyp=44, npml=8, nt=220, nshots=3, nrec=10)
    g = wl.grid
    wav1 = O.ricker(wl.f0, g.dt, g.nt)
    wav = np.broadcast_to(wav1, (wl.nshots, 1, g.nt)).copy()
    obs = O.forward(g, wl.eps_true, wl.sig_true, wl.src, wav, wl.rec)
    energy = 0.5 * float((obs.astype(np.float32).astype(np.float64) ** 2).sum())
    fd = FDTD(g, wl.src, wl.rec, device=dev)
    obs_d = torch.tensor(obs, dtype=torch.float32, device=dev)
    mask = interior_mask(g, rows_below_top=4)   # the sources sit 1-3 rows below the top
    lr = ((0.2, 0.0), (0.1, 1e-4))
    cfg = AdamConfig(stages=(Stage(1, *lr[0]), Stage(1, *lr[1])))
    models = []
    drv = StagedAdam(fd, lambda f0: obs_d, mask, wl.f0, cfg)
    e0 = torch.tensor(wl.eps_init, dtype=torch.float32)
    s0 = torch.tensor(wl.sig_init, dtype=torch.float32)
    eps2, sig2, hist = drv.run(e0, s0, callback=lambda ep, J, e, s: models.append(
        (e.cpu().numpy().astype(np.float64), s.cpu().numpy().astype(np.float64))))
    fd.status()
    x0e, x0s = e0.numpy().astype(np.float64), s0.numpy().astype(np.float64)
    (x1e, x1s), (x2e, x2s) = models
    # the oracle's gradients at the models the loop visited
    J0, ge0, gs0 = O.misfit_and_gradient(g, x0e, x0s, wl.src, wav, wl.rec, obs)
    J1, ge1, gs1 = O.misfit_and_gradient(g, x1e, x1s, wl.src, wav, wl.rec, obs)
    assert hist.misfit[0] == pytest.approx(J0 / energy, rel=1e-4)
    assert hist.misfit[1] == pytest.approx(J1 / energy, rel=1e-4)
    m = mask.numpy()
    # epoch 1: eps_r only; sigma untouched everywhere
    assert np.array_equal(x1s, x0s)
    want1 = adam_expected(x0e, [ge0 / energy], [lr[0][0]], 1.0, m)
    # epoch 2: eps_r's second Adam step, sigma's first
    want2e = adam_expected(x0e, [ge0 / energy, ge1 / energy], [lr[0][0], lr[1][0]], 1.0, m)
    want2s = adam_expected(x0s, [gs1 / energy], [lr[1][1]], 0.0, m)
    # masked cells never move
    for a, b in ((x1e, x0e), (x2e, x0e), (x2s, x0s)):
        assert np.array_equal(a[m == 0], b[m == 0])
    # where the gradients are well above FP32 rounding, the steps agree with the replay
    free = m != 0
    big = lambda a: np.abs(a) > 1e-2 * np.abs(a[free]).max()
    robust_e = free & big(ge0) & big(ge1)
    robust_s = free & big(gs1)
    assert robust_e.sum() > 0.05 * free.sum() and robust_s.sum() > 0.05 * free.sum()
    assert np.abs(x1e - want1)[robust_e].max() <= 5e-3 * lr[0][0]
    assert np.abs(x2e - want2e)[robust_e].max() <= 1e-2 * lr[1][0]
    assert np.abs(x2s - want2s)[robust_s].max() <= 1e-2 * lr[1][1]
    # the clamps hold everywhere
    assert x2e.min() >= 1.0 and x2s.min() >= 0.0
    assert np.allclose(eps2.cpu().numpy(), x2e) and np.allclose(sig2.cpu().numpy(), x2s)
    fd.close()


def test_staged_adam_lowers_the_misfit(dev):
    from paper_2506_20513_gb300 import FDTD
    from paper_2506_20513_gb300.adam import AdamConfig, Stage, StagedAdam
    from paper_2506_20513_gb300.fdtd import ricker
    from paper_2506_20513_gb300.fwi import interior_mask
    wl = W.small_random(42, nxp=80, nyp=50, npml=8, nt=260, nshots=4, nrec=16)
    g = wl.grid
    fd = FDTD(g, wl.src, wl.rec, device=dev)
    t32 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    obs = {}

    def observed(f0):
        if f0 not in obs:
            obs[f0] = fd.forward_model(t32(wl.eps_true), t32(wl.sig_true),
                                       torch.tensor(ricker(f0, g.dt, g.nt), device=dev))
        return obs[f0]

    cfg = AdamConfig(stages=(Stage(10, 0.05, 0.0, wl.f0 / 2), Stage(15, 0.03, 2e-4, wl.f0)),
                     tv=True)
    drv = StagedAdam(fd, observed, interior_mask(g, rows_below_top=2), wl.f0, cfg)
    eps, sig, hist = drv.run(t32(wl.eps_init), t32(wl.sig_init))
    fd.status()
    assert hist.stage == [0] * 10 + [1] * 15
    # each stage lowers its own misfit (the data of the two stages differ)
    assert min(hist.misfit[1:10]) < hist.misfit[0]
    assert min(hist.misfit[11:]) < hist.misfit[10]
    e_err = lambda e: np.linalg.norm(np.asarray(e) - wl.eps_true)
    assert e_err(eps.cpu().numpy()) < e_err(wl.eps_init)
    fd.close()
