"""FP32 CUDA path vs the FP64 oracle, element by element on the same seeded inputs.

Tolerances (relative L2): traces <= 1e-4, g_eps_r and g_sigma <= 1e-3, misfit <= 1e-3.
Cases span several tiles with ragged edge tiles, several time-block depths, several shots
and sources, a CPML with kappa_max > 1, perfect-conductor cells, and the full-size
32-shot 540x290 workload in the launch configuration the benchmark times (sampled).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2506_20513_gb300 import _lib, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

TRACE_TOL = 1e-4
GRAD_TOL = 1e-3


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_20513_gb300 import build as B
    B.build_library()
    return torch.device("cuda", 0)


def t32(a, dev):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)


def wavelets(wl, nsrc=1):
    w = O.ricker(wl.f0, wl.grid.dt, wl.grid.nt)
    return np.ascontiguousarray(np.broadcast_to(w, (wl.nshots, nsrc, wl.grid.nt)))


def gpu_gradient(wl, dev, obs, tiling=None, wav=None, checkpoint_every=0):
    from paper_2506_20513_gb300 import FDTD, Tiling
    fd = FDTD(wl.grid, wl.src, wl.rec, device=dev, tiling=Tiling(*tiling) if tiling else None)
    if checkpoint_every:
        fd.set_storage(checkpoint_every)
    wav = wavelets(wl, wl.src.shape[1]) if wav is None else wav
    J, ge, gs, tr = fd.misfit_and_gradient(t32(wl.eps_init, dev), t32(wl.sig_init, dev),
                                           t32(wav, dev), t32(obs, dev), return_traces=True)
    fd.status()
    out = float(J.item()), ge.cpu().numpy(), gs.cpu().numpy(), tr.cpu().numpy()
    fd.close()
    return out


def fit_variant(tiling):
    """Tile widths are multiples of 4 (windows start on 16-byte boundaries).  Variant 1 stages
    a 64 x 32 window: shrink the tile height to fit (tile + 2K <= 32).  Variant 3 (persistent)
    wants tiles at least K wide and high."""
    if not tiling:
        return tiling
    tw, th, k = tiling[:3]
    v = tiling[3] if len(tiling) == 4 else None
    if tw > 0:
        tw = max(tw - tw % 4, 4)
        if v == 3:
            tw = max(tw, 4 * ((k + 3) // 4))
    if v == 1 and th > 0:
        th = max(1, min(th, 32 - 2 * k))
    if v == 3 and th > 0:
        th = max(th, k)
    return (tw, th, k) + ((v,) if v is not None else ())


def check_case(wl, dev, tiling=None, nsrc=1, checkpoint_every=0):
    tiling = fit_variant(tiling)
    wav = wavelets(wl, nsrc)
    obs = O.forward(wl.grid, wl.eps_true, wl.sig_true, wl.src, wav, wl.rec)
    J, ge, gs, tr = gpu_gradient(wl, dev, obs, tiling, wav, checkpoint_every)
    J64, ge64, gs64, tr64 = O.misfit_and_gradient(wl.grid, wl.eps_init, wl.sig_init, wl.src, wav,
                                                  wl.rec, obs, nthreads=4, return_traces=True)
    assert rel(tr, tr64) <= TRACE_TOL
    assert abs(J - J64) <= GRAD_TOL * J64
    assert rel(ge, ge64) <= GRAD_TOL
    assert rel(gs, gs64) <= GRAD_TOL
    return J64


def test_single_shot_disc(dev):
    """100x100 (+10 CPML) disc model, one 200 MHz shot, 20 receivers, nt 600."""
    wl = W.single_shot_disc()
    check_case(wl, dev)


def test_preconditioner_workload_subset(dev):
    """The learned preconditioner's grid (256x128 + 20-cell CPML, dx 0.01 m, 400 MHz, 64
    receivers, nt 1500), two of its 16 shots, in the default launch configuration: traces
    and both gradients against the FP64 oracle."""
    import dataclasses
    wl = W.preconditioner_model(100123, nshots=16, nt=1500)
    wl = dataclasses.replace(wl, src=wl.src[[3, 11]], rec=wl.rec[[3, 11]])
    check_case(wl, dev)


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("seed,tiling,kappa,pec", [
    (1, None, 1.0, False),
    (2, (8, 6, 3), 2.0, True),
    (3, (12, 7, 4), 1.0, True),
    (4, (10, 10, 1), 2.0, False),
    (5, (56, 39, 3), 1.0, False),   # one tile covers the whole grid
    (6, (30, 9, 6), 1.0, False),
])
def test_small_random(dev, seed, tiling, kappa, pec, variant):
    wl = W.small_random(seed, nxp=46, nyp=27, npml=6, nt=150, nshots=3, nrec=9,
                        kappa_max=kappa, with_pec=pec)
    check_case(wl, dev, (tiling or (0, 0, 0)) + (variant,))


@pytest.mark.parametrize("variant", [0, 3])
@pytest.mark.parametrize("nrec,tiling", [(200, (0, 0, 4)), (400, (0, 0, 4)), (400, (12, 7, 4)),
                                         (900, (0, 0, 4)), (900, (0, 0, 10))])
def test_dense_receivers(dev, nrec, tiling, variant):
    """Hundreds of receivers scattered over the grid, duplicates included: launches whose
    window lists fit the shared-memory staging of positions, indices and (adjoint) residual
    samples (up to 682 entries at K = 4, 341 at K = 10) and launches that exceed it (900
    entries) and decode them from global memory."""
    wl = W.small_random(51, nxp=46, nyp=27, npml=6, nt=150, nshots=2, nrec=nrec)
    check_case(wl, dev, tiling + (variant,))


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("npml,tiling", [(0, (16, 16, 4)), (3, (20, 18, 5)), (8, (40, 40, 12))])
def test_tiles_off_the_absorbing_strips(dev, npml, tiling, variant):
    """Large grids with thin (or no) CPML: most tiles take the body without CPML memories."""
    wl = W.small_random(30 + npml, nxp=110, nyp=84, npml=npml, nt=280, nshots=2, nrec=8,
                        with_pec=True)
    check_case(wl, dev, tiling + (variant,))


@pytest.mark.parametrize("k,tiling", [(1, (20, 14, 3, 0)), (7, (20, 14, 4, 1)), (16, None),
                                      (150, None), (64, (44, 30, 5, 0)), (33, (0, 0, 5, 2)),
                                      (33, (20, 14, 5, 3)), (1, (0, 0, 3, 3))])
def test_checkpointed_gradient(dev, k, tiling):
    """Checkpoints every k steps and segment recomputation in the adjoint (k = 1, k not a
    multiple of the time block, k = nt)."""
    wl = W.small_random(8, nxp=46, nyp=27, npml=6, nt=150, nshots=2, nrec=7, kappa_max=2.0,
                        with_pec=True)
    check_case(wl, dev, tiling, checkpoint_every=k)


def test_checkpointed_matches_full_store_at_scale(dev):
    """540x290, 32 shots, nt 400: checkpoints every 50 steps vs the full wavefield store."""
    wl = W.multishot_layered(nt=400)
    wav = wavelets(wl)
    from paper_2506_20513_gb300 import FDTD
    fd = FDTD(wl.grid, wl.src, wl.rec, device=dev)
    obs = fd.forward_model(t32(wl.eps_true, dev), t32(wl.sig_true, dev), t32(wav, dev))
    full = fd.misfit_and_gradient(t32(wl.eps_init, dev), t32(wl.sig_init, dev), t32(wav, dev), obs)
    fd.set_storage(50)
    ck = fd.misfit_and_gradient(t32(wl.eps_init, dev), t32(wl.sig_init, dev), t32(wav, dev), obs)
    fd.status()
    # launches split at segment boundaries round differently (FP32), nothing more
    assert abs(full[0].item() - ck[0].item()) <= 1e-6 * full[0].item()
    for a, b in zip(full[1:], ck[1:]):
        assert rel(b.cpu().numpy(), a.cpu().numpy()) <= 1e-5
    fd.close()


def test_multiple_sources_per_shot(dev):
    wl = W.small_random(9, nxp=40, nyp=30, npml=5, nt=120, nshots=2, nrec=6)
    rng = np.random.default_rng(0)
    src = np.zeros((2, 3, 2), dtype=np.int32)
    src[:, :, 0] = wl.grid.npml + rng.integers(1, 39, size=(2, 3))
    src[:, :, 1] = wl.grid.npml + rng.integers(1, 29, size=(2, 3))
    src[1, 2] = src[1, 1]  # two sources in one cell add up
    wl.src = src
    check_case(wl, dev, nsrc=3)


def test_adjoint_of_arbitrary_cotangent(dev):
    """gf_adjoint driven by a random trace cotangent equals the oracle's transpose."""
    from paper_2506_20513_gb300 import FDTD
    wl = W.small_random(12, nxp=50, nyp=33, npml=7, nt=140, nshots=2, nrec=8, kappa_max=2.0)
    g = wl.grid
    wav = wavelets(wl)
    r = np.random.default_rng(5).standard_normal((wl.nshots, g.nt, wl.nrec))
    fd = FDTD(g, wl.src, wl.rec, device=dev)
    tr = fd.forward(t32(wl.eps_true, dev), t32(wl.sig_true, dev), t32(wav, dev))
    ge, gs = fd.adjoint(t32(wl.eps_true, dev), t32(wl.sig_true, dev), t32(r, dev))
    fd.status()
    ge64 = np.zeros((g.ny, g.nx))
    gs64 = np.zeros((g.ny, g.nx))
    for s in range(wl.nshots):
        fw = O.forward_shot(g, wl.eps_true, wl.sig_true, wl.src[s], wav[s], wl.rec[s], history=True)
        assert rel(tr[s].cpu().numpy(), fw["traces"]) <= TRACE_TOL
        a = O.adjoint_shot(g, wl.eps_true, wl.sig_true, wl.src[s], wl.rec[s], r[s], fw["ez_hist"])
        ge64 += a["g_eps_r"]
        gs64 += a["g_sigma"]
    assert rel(ge.cpu().numpy(), ge64) <= GRAD_TOL
    assert rel(gs.cpu().numpy(), gs64) <= GRAD_TOL


def test_dot_product_of_gpu_adjoint_with_oracle_tangent(dev):
    """<J dm, r> = <dm, J^T r>: the oracle's FP64 tangent-linear traces along a smooth random
    model perturbation dm, against the GPU adjoint's gradient for a random trace cotangent r
    (CPML with kappa_max = 2, PEC cells, two shots).  FP32 bound 1e-5 relative."""
    from paper_2506_20513_gb300 import FDTD
    wl = W.small_random(13, nxp=52, nyp=36, npml=7, nt=150, nshots=2, nrec=9, kappa_max=2.0,
                        with_pec=True)
    g = wl.grid
    wav = wavelets(wl)
    rng = np.random.default_rng(17)
    r = rng.standard_normal((wl.nshots, g.nt, wl.nrec))
    from scipy.ndimage import gaussian_filter
    de = gaussian_filter(rng.standard_normal((g.ny, g.nx)), 2.0)
    ds = 1e-3 * gaussian_filter(rng.standard_normal((g.ny, g.nx)), 2.0)
    fd = FDTD(g, wl.src, wl.rec, device=dev)
    fd.forward(t32(wl.eps_init, dev), t32(wl.sig_init, dev), t32(wav, dev))
    ge, gs = fd.adjoint(t32(wl.eps_init, dev), t32(wl.sig_init, dev), t32(r, dev))
    fd.status()
    lhs = sum(float((O.tangent(g, wl.eps_init, wl.sig_init, de, ds, wl.src[k], wav[k],
                                wl.rec[k]) * r[k]).sum()) for k in range(wl.nshots))
    rhs = float((de * ge.cpu().numpy().astype(np.float64)).sum()
                + (ds * gs.cpu().numpy().astype(np.float64)).sum())
    assert abs(lhs) > 0
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    fd.close()


def test_autograd_function_matches_misfit_and_gradient(dev):
    from paper_2506_20513_gb300 import FDTD, FDTDFunction
    wl = W.small_random(14, nxp=36, nyp=24, npml=5, nt=100, nshots=2, nrec=5)
    wav = t32(wavelets(wl), dev)
    fd = FDTD(wl.grid, wl.src, wl.rec, device=dev)
    obs = fd.forward_model(t32(wl.eps_true, dev), t32(wl.sig_true, dev), wav)
    e = t32(wl.eps_init, dev).requires_grad_()
    s = t32(wl.sig_init, dev).requires_grad_()
    d = FDTDFunction.apply(e, s, fd, wav)
    loss = 0.5 * ((d - obs) ** 2).sum()
    loss.backward()
    J, ge, gs = fd.misfit_and_gradient(e.detach(), s.detach(), wav, obs)
    fd.status()
    assert abs(loss.item() - J.item()) <= 1e-5 * J.item()
    assert rel(e.grad.cpu().numpy(), ge.cpu().numpy()) <= 1e-5
    assert rel(s.grad.cpu().numpy(), gs.cpu().numpy()) <= 1e-5


def test_illumination(dev):
    """illum = sum over shots and n = 1..nt of Ez^n squared."""
    from paper_2506_20513_gb300 import FDTD
    wl = W.small_random(15, nxp=30, nyp=22, npml=4, nt=90, nshots=2, nrec=4)
    g = wl.grid
    wav = wavelets(wl)
    fd = FDTD(g, wl.src, wl.rec, device=dev)
    _, ill = fd.forward_model(t32(wl.eps_true, dev), t32(wl.sig_true, dev), t32(wav, dev),
                              illumination=True)
    ref = np.zeros((g.ny, g.nx))
    for s in range(wl.nshots):
        h = O.forward_shot(g, wl.eps_true, wl.sig_true, wl.src[s], wav[s], wl.rec[s],
                           history=True)["ez_hist"]
        ref += (h[1:] ** 2).sum(axis=0)
    assert rel(ill.cpu().numpy(), ref) <= 1e-4


def test_single_step_and_short_runs(dev):
    """nt = 1: the only trace sample is Ez^0 = 0 and the gradient vanishes; nt = 2 is
    ragged against every time-block depth."""
    from paper_2506_20513_gb300 import FDTD
    for nt in (1, 2, 5):
        wl = W.small_random(16, nxp=20, nyp=12, npml=3, nt=nt, nshots=1, nrec=3)
        wav = np.ones((1, 1, nt))
        fd = FDTD(wl.grid, wl.src, wl.rec, device=dev)
        obs = np.random.default_rng(nt).standard_normal((1, nt, 3))
        J, ge, gs, tr = fd.misfit_and_gradient(t32(wl.eps_init, dev), t32(wl.sig_init, dev),
                                               t32(wav, dev), t32(obs, dev), return_traces=True)
        fd.status()
        J64, ge64, gs64, tr64 = O.misfit_and_gradient(wl.grid, wl.eps_init, wl.sig_init, wl.src,
                                                      wav, wl.rec, obs, return_traces=True)
        assert np.all(tr[:, 0].cpu().numpy() == 0)
        np.testing.assert_allclose(tr.cpu().numpy(), tr64, rtol=1e-4, atol=1e-6 * np.abs(tr64).max() + 1e-30)
        assert abs(J.item() - J64) <= 1e-5 * J64
        if nt == 1:
            assert not ge.abs().max().item() and not gs.abs().max().item()
        # for nt = 2 the exact gradient vanishes (Ez^1 is nonzero only at the source)
        for a, b in ((ge, ge64), (gs, gs64)):
            a = a.cpu().numpy()
            np.testing.assert_allclose(a, b, rtol=GRAD_TOL, atol=GRAD_TOL * np.abs(b).max() + 1e-30)


def test_invalid_model_is_reported(dev):
    from paper_2506_20513_gb300 import FDTD
    wl = W.small_random(18, nxp=20, nyp=12, npml=3, nt=10, nshots=1, nrec=2)
    fd = FDTD(wl.grid, wl.src, wl.rec, device=dev)
    e = t32(wl.eps_true, dev)
    e[5, 5] = 0.5
    fd.forward_model(e, t32(wl.sig_true, dev), t32(np.ones(10), dev))
    with pytest.raises(_lib.GfError) as ex:
        fd.status()
    assert ex.value.code == _lib.GF_EINVAL
    fd.status()  # cleared after reading


def test_oversized_tiling_is_rejected(dev):
    """A tile whose shared-memory footprint cannot fit is refused, not run."""
    from paper_2506_20513_gb300 import FDTD, Tiling
    wl = W.small_random(22, nxp=20, nyp=12, npml=3, nt=10, nshots=1, nrec=2)
    fd = FDTD(wl.grid, wl.src, wl.rec, device=dev)
    with pytest.raises(_lib.GfError) as ex:
        fd.set_tiling(Tiling(4096, 4096, 8))
    assert ex.value.code == _lib.GF_EINVAL


def test_adjoint_without_forward_is_rejected(dev):
    from paper_2506_20513_gb300 import FDTD
    wl = W.small_random(19, nxp=20, nyp=12, npml=3, nt=10, nshots=1, nrec=2)
    fd = FDTD(wl.grid, wl.src, wl.rec, device=dev)
    with pytest.raises(_lib.GfError) as ex:
        fd.adjoint(t32(wl.eps_true, dev), t32(wl.sig_true, dev), t32(np.zeros((1, 10, 2)), dev))
    assert ex.value.code == _lib.GF_ESTATE


def test_host_tensors_end_to_end(dev):
    """CPU tensors in, CPU results out (the end-to-end path the benchmark times)."""
    from paper_2506_20513_gb300 import FDTD
    wl = W.small_random(20, nxp=30, nyp=20, npml=4, nt=80, nshots=2, nrec=4)
    wav = wavelets(wl)
    obs = O.forward(wl.grid, wl.eps_true, wl.sig_true, wl.src, wav, wl.rec)
    fd = FDTD(wl.grid, wl.src, wl.rec, device=dev)
    c = lambda a: torch.tensor(a, dtype=torch.float32).pin_memory()
    J, ge, gs = fd.misfit_and_gradient(c(wl.eps_init), c(wl.sig_init), c(wav), c(obs))
    assert not ge.is_cuda
    J64, ge64, gs64 = O.misfit_and_gradient(wl.grid, wl.eps_init, wl.sig_init, wl.src, wav,
                                            wl.rec, obs)
    assert rel(ge.numpy(), ge64) <= GRAD_TOL and rel(gs.numpy(), gs64) <= GRAD_TOL


@pytest.mark.parametrize("variant,K", [(3, 7), (1, 4), (2, 7), (0, 10)])
def test_variants_at_scale(dev, variant, K):
    """540x290, 32 shots, nt 300: other kernel variants and time-block depths against the
    default launch configuration (variant 0, K = 7): traces, misfit, gradients, over many
    tiles and shots."""
    from paper_2506_20513_gb300 import FDTD, Tiling
    wl = W.multishot_layered(nt=300)
    wav = t32(wavelets(wl), dev)
    e0, s0 = t32(wl.eps_init, dev), t32(wl.sig_init, dev)
    fd = FDTD(wl.grid, wl.src, wl.rec, device=dev)
    obs = fd.forward_model(t32(wl.eps_true, dev), t32(wl.sig_true, dev), wav)
    ref = fd.misfit_and_gradient(e0, s0, wav, obs, return_traces=True)
    fd.set_tiling(Tiling(0, 0, K, variant))
    got = fd.misfit_and_gradient(e0, s0, wav, obs, return_traces=True)
    fd.status()
    assert abs(got[0].item() - ref[0].item()) <= 1e-5 * ref[0].item()
    for a, b in zip(got[1:], ref[1:]):
        assert rel(a.cpu().numpy(), b.cpu().numpy()) <= 1e-4
    fd.close()


def test_full_size_multishot_sampled(dev):
    """540x290 grid, 32 shots, nt 2000, 100 receivers, in the benchmark's launch
    configuration: all 32 shots run on the GPU; the oracle recomputes the traces of two
    sampled shots and the exact gradient of a two-shot subset at the same full size."""
    from paper_2506_20513_gb300 import FDTD
    wl = W.multishot_layered()
    g = wl.grid
    wav = wavelets(wl)
    fd = FDTD(g, wl.src, wl.rec, device=dev)
    tr = fd.forward_model(t32(wl.eps_true, dev), t32(wl.sig_true, dev), t32(wav, dev)).cpu().numpy()
    fd.status()
    fd.close()
    picks = [0, 17]
    tr64 = O.forward(g, wl.eps_true, wl.sig_true, wl.src[picks], wav[picks], wl.rec[picks],
                     nthreads=2)
    for k, s in enumerate(picks):
        assert rel(tr[s], tr64[k]) <= TRACE_TOL
    sub = [0, 31]
    wl2 = W.Workload(wl.name, g, wl.f0, wl.src[sub], wl.rec[sub], wl.eps_true, wl.sig_true,
                     wl.eps_init, wl.sig_init)
    obs = np.stack([tr64[0], O.forward(g, wl.eps_true, wl.sig_true, wl.src[[31]], wav[[31]],
                                       wl.rec[[31]])[0]])
    J, ge, gs, _ = gpu_gradient(wl2, dev, obs)
    J64, ge64, gs64 = O.misfit_and_gradient(g, wl.eps_init, wl.sig_init, wl2.src, wav[sub],
                                            wl2.rec, obs, nthreads=2)
    assert abs(J - J64) <= GRAD_TOL * J64
    assert rel(ge, ge64) <= GRAD_TOL
    assert rel(gs, gs64) <= GRAD_TOL



def test_directional_derivative_matches_gradient(dev):
    """<g, dm> against central differences of J along a smooth random direction dm of both
    parameters at once (the linearised model -> misfit map against its adjoint, FP32)."""
    from paper_2506_20513_gb300 import FDTD
    from scipy.ndimage import gaussian_filter
    wl = W.small_random(31, nxp=70, nyp=50, npml=8, nt=300, nshots=3, nrec=9)
    g = wl.grid
    wav = t32(wavelets(wl), dev)
    fd = FDTD(g, wl.src, wl.rec, device=dev)
    obs = fd.forward_model(t32(wl.eps_true, dev), t32(wl.sig_true, dev), wav)
    e0, s0 = t32(wl.eps_init, dev), t32(wl.sig_init, dev)
    J, ge, gs = fd.misfit_and_gradient(e0, s0, wav, obs)
    rng = np.random.default_rng(31)
    de = gaussian_filter(rng.standard_normal((g.ny, g.nx)), 3.0)
    ds = gaussian_filter(rng.standard_normal((g.ny, g.nx)), 3.0)
    de *= 0.01 * float(e0.mean()) / np.abs(de).max()
    ds *= 0.01 * float(s0.mean()) / np.abs(ds).max()
    pred = float((ge.double() * t32(de, dev).double()).sum() + (gs.double() * t32(ds, dev).double()).sum())
    J1 = []
    for h in (1.0, -1.0):
        J1.append(float(fd.misfit(e0 + h * t32(de, dev), s0 + h * t32(ds, dev), wav, obs).item()))
    fdv = (J1[0] - J1[1]) / 2.0
    assert fdv == pytest.approx(pred, rel=2e-3)

def test_large_grid_gradient_vs_central_differences(dev):
    """2108x1084 grid (30-cell CPML), dx 5 mm, 1 GHz, 16 shots, 400 receivers, nt 4000, the
    gradient checkpointed every 200 steps: central differences of the misfit at 20 cells
    drawn uniformly among the interior cells whose |g| exceeds 1% of the interior maximum,
    for eps_r (step h = 0.5% of the cell's value) and for sigma (h = 5%).

    Tolerance, per cell: |fd - g| <= 0.01 |g| + 10 n / (2 h).
    * 0.01 |g| bounds the central difference's truncation error, h^2 J'''(m) / 6: J depends
      on one cell's eps_r or sigma smoothly, over a scale of the value itself, so that error
      is about (h / value)^2 of |g|: 2.5e-5 (eps_r) and 2.5e-3 (sigma).  It also covers the
      FP32 gradient's own error, below 1e-3 of |g| where |g| is at least 1% of the maximum.
    * n is the rounding noise of one FP32 misfit evaluation; the two evaluations of a
      central difference differ by up to about 2 n.  It is measured here as the larger of
      |J_A - J_B| for the same model run with two tilings (different rounding order, same
      arithmetic), and eta ||r|| ||d|| / sqrt(N): the residual-weighted sum over N trace
      samples whose FP32 rounding is eta ||d|| in norm (eta = ||d_A - d_B|| / ||d_A||), taken
      as uncorrelated with the residual r.  The factor 10 is the margin for the noise of the
      perturbed runs, which is not that of the unperturbed one.
    On top, the picks' finite differences and gradients must correlate at >= 0.999."""
    from paper_2506_20513_gb300 import FDTD, Tiling
    wl = W.large_checkpointed(nt=4000)
    g = wl.grid
    wav = t32(wavelets(wl), dev)
    fd = FDTD(g, wl.src, wl.rec, device=dev)
    fd.set_storage(200)
    obs = fd.forward_model(t32(wl.eps_true, dev), t32(wl.sig_true, dev), wav)
    e0, s0 = t32(wl.eps_init, dev), t32(wl.sig_init, dev)
    J, ge, gs = fd.misfit_and_gradient(e0, s0, wav, obs)
    fd.status()
    J = float(J.item())
    # rounding noise of one misfit: the same model under another tiling
    dA = fd.forward_model(e0, s0, wav)
    fdB = FDTD(g, wl.src, wl.rec, device=dev, tiling=Tiling(40, 40, 4, 0))
    dB = fdB.forward_model(e0, s0, wav)
    JB = float(fdB.misfit(e0, s0, wav, obs).item())
    fdB.close()
    JA = float(fd.misfit(e0, s0, wav, obs).item())
    # the gradient's forward runs in checkpoint segments (launches split at their ends):
    # the same misfit to FP32 rounding
    assert JA == pytest.approx(J, rel=1e-5)
    eta = float((dA - dB).double().norm() / dA.double().norm())
    r_norm = float((dA - obs).double().norm())
    noise = max(abs(JA - JB), eta * r_norm * float(dA.double().norm()) / math.sqrt(dA.numel()))
    rng = np.random.default_rng(4000)
    p = g.npml
    for name, grad, model, rel_h in (("eps", ge, e0, 5e-3), ("sig", gs, s0, 5e-2)):
        a = grad.abs().cpu().numpy()
        a[:p + 4, :] = 0   # the absorbing layer and the rows of the sources
        a[-p:, :] = 0
        a[:, :p] = 0
        a[:, -p:] = 0
        cand = np.argwhere(a > 1e-2 * a.max())
        picks = cand[rng.choice(len(cand), 20, replace=False)]
        fdv, adv, tol = [], [], []
        for j, i in picks:
            v = float(model[j, i])
            h = rel_h * v
            Jpm = []
            for sgn in (1, -1):
                m = model.clone()
                m[j, i] = v + sgn * h
                args = (m, s0) if name == "eps" else (e0, m)
                Jpm.append(fd.misfit(*args, wav, obs).item())
            fdv.append((Jpm[0] - Jpm[1]) / (2 * h))
            adv.append(float(grad[j, i]))
            tol.append(0.01 * abs(adv[-1]) + 10 * noise / (2 * h))
        fdv, adv, tol = np.array(fdv), np.array(adv), np.array(tol)
        err = np.abs(fdv - adv)
        print(f"{name}: noise {noise:.3e} J {J:.6e} eta {eta:.2e} max rel err "
              f"{(err / np.abs(adv)).max():.3e} max err/tol {(err / tol).max():.3f}")
        assert np.all(err <= tol), (name, (err / np.abs(adv)).max(), (err / tol).max())
        assert np.corrcoef(fdv, adv)[0, 1] >= 0.999, name
    fd.close()


def test_dependency_wait_timeout_is_reported_and_recovered(dev):
    """The persistent kernels' dependency waits are bounded: with a budget of zero polls a
    wait that is not already satisfied gives up, the CTA ends and gf_status reports
    GF_ETIMEOUT (nothing hangs, the context stays usable); with the default budget restored the
    next call is exact again."""
    from paper_2506_20513_gb300 import FDTD
    # 3 x 3 tiles and 2 shots: 18 items per time block, fewer than the resident CTAs, so the
    # items of block b + 1 are taken while their neighbours' block b is still running
    from paper_2506_20513_gb300 import Tiling
    wl = W.small_random(60, nxp=140, nyp=110, npml=8, nt=200, nshots=2, nrec=8)
    g = wl.grid
    wav = t32(wavelets(wl), dev)
    fd = FDTD(g, wl.src, wl.rec, device=dev, tiling=Tiling(0, 0, 7, 3))
    obs = fd.forward_model(t32(wl.eps_true, dev), t32(wl.sig_true, dev), wav)
    e0, s0 = t32(wl.eps_init, dev), t32(wl.sig_init, dev)
    ref = fd.misfit_and_gradient(e0, s0, wav, obs)
    fd.status()
    _lib.check(fd.lib, fd.ctx, fd.lib.gf_set_wait_budget(fd.ctx, 0))
    fd.misfit_and_gradient(e0, s0, wav, obs)
    with pytest.raises(_lib.GfError) as ex:
        fd.status()
    assert ex.value.code == _lib.GF_ETIMEOUT
    _lib.check(fd.lib, fd.ctx, fd.lib.gf_set_wait_budget(fd.ctx, 1 << 22))
    got = fd.misfit_and_gradient(e0, s0, wav, obs)
    fd.status()
    assert got[0].item() == ref[0].item()
    for a, b in zip(got[1:], ref[1:]):
        assert torch.equal(a, b)
    fd.close()


@pytest.mark.parametrize("k", [0, 40])
def test_shot_lanes_give_identical_results(dev, k):
    """Shots split into 1, 2, 3 or 4 lanes running concurrently (full store and checkpoints
    every k steps): bit-identical misfit and gradients, since every shot's arithmetic and
    every sum's order are the same; and the oracle's gradient within tolerance."""
    from paper_2506_20513_gb300 import FDTD
    wl = W.small_random(77, nxp=120, nyp=70, npml=8, nt=260, nshots=5, nrec=11, with_pec=True)
    g = wl.grid
    wav = wavelets(wl)
    obs = O.forward(g, wl.eps_true, wl.sig_true, wl.src, wav, wl.rec)
    out = []
    for lanes in (1, 2, 3, 4):
        fd = FDTD(g, wl.src, wl.rec, device=dev)
        assert fd.lib.gf_set_lanes(fd.ctx, lanes) == 0
        if k:
            fd.set_storage(k)
        J, ge, gs = fd.misfit_and_gradient(t32(wl.eps_init, dev), t32(wl.sig_init, dev),
                                           t32(wav, dev), t32(obs, dev))
        tr = fd.forward_model(t32(wl.eps_init, dev), t32(wl.sig_init, dev), t32(wav, dev))
        Jm = fd.misfit(t32(wl.eps_init, dev), t32(wl.sig_init, dev), t32(wav, dev), t32(obs, dev))
        fd.status()
        out.append((J.item(), ge.cpu(), gs.cpu(), tr.cpu(), Jm.item()))
        fd.close()
    for J, ge, gs, tr, Jm in out[1:]:
        assert J == out[0][0] and Jm == out[0][4]
        assert torch.equal(ge, out[0][1]) and torch.equal(gs, out[0][2])
        assert torch.equal(tr, out[0][3])
    J64, ge64, gs64 = O.misfit_and_gradient(g, wl.eps_init, wl.sig_init, wl.src, wav, wl.rec, obs)
    assert rel(out[0][1].numpy(), ge64) <= GRAD_TOL and rel(out[0][2].numpy(), gs64) <= GRAD_TOL


@pytest.mark.parametrize("tiling", [None, (20, 14, 5, 3), (0, 0, 4, 1)])
def test_magnetic_receiver_components(dev, tiling):
    """gf_forward_model_fields: the receivers' Hx^{n-1/2}, Hy^{n-1/2} against the oracle's
    (traces tolerance), the Ez traces bit-identical to gf_forward_model's; dense receivers,
    a kappa_max = 2 CPML, two lanes, the persistent and the two-CTA variants."""
    from paper_2506_20513_gb300 import FDTD, Tiling
    wl = W.small_random(81, nxp=64, nyp=40, npml=7, nt=170, nshots=3, nrec=40, kappa_max=2.0)
    g = wl.grid
    wav = wavelets(wl)
    fd = FDTD(g, wl.src, wl.rec, device=dev, tiling=Tiling(*fit_variant(tiling)) if tiling else None)
    args = (t32(wl.eps_true, dev), t32(wl.sig_true, dev), t32(wav, dev))
    tr, h = fd.forward_model(*args, fields=True)
    tr0 = fd.forward_model(*args)
    fd.status()
    assert torch.equal(tr, tr0)
    hx = np.zeros((wl.nshots, g.nt, wl.nrec))
    hy = np.zeros_like(hx)
    for s in range(wl.nshots):
        o = O.forward_shot(g, wl.eps_true, wl.sig_true, wl.src[s], wav[s], wl.rec[s], fields=True)
        hx[s], hy[s] = o["h_traces"][..., 0], o["h_traces"][..., 1]
    h = h.cpu().numpy()
    assert rel(h[..., 0], hx) <= TRACE_TOL and rel(h[..., 1], hy) <= TRACE_TOL
    assert np.all(h[:, 0] == 0.0)   # H^{-1/2} = 0
    fd.close()
