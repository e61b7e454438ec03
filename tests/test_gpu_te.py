"""TE-mode forward model and gradient (x- and y-directed sources: Ex, Ey, Hz) on the GPU vs
the FP64 oracle, element by element on the same seeded inputs.  Gradients: misfit, g_eps_r
and g_sigma to rel-L2 <= 1e-3.

Tolerance: relative L2 <= 1e-4 per shot and component (a component far weaker than its
unit's strongest one, e.g. a cross-polar trace near a symmetry line, is held to 1e-4 of a
hundredth of that scale).  Cases: heterogeneous lossy models with a CPML (kappa_max 1 and
2), perfect-conductor cells, a PEC box without CPML, several sources per shot (two in one
cell), dense and duplicate receivers, one- and two-step runs, and the full-size 32-shot
540 x 290, nt 2000 workload (sampled shots); plus the error paths and the reuse of the
forward workspace.
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2506_20513_gb300 import _lib, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

TRACE_TOL = 1e-4


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_20513_gb300 import build as B
    B.build_library()
    return torch.device("cuda", 0)


def t32(a, dev):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)


def wavelets(wl, nsrc):
    w = O.ricker(wl.f0, wl.grid.dt, wl.grid.nt)
    # a different amplitude per source, so that a source mixed up with another shows
    return np.ascontiguousarray(np.stack([np.stack([w * (1.0 + 0.5 * k) for k in range(nsrc)])
                                          for _ in range(wl.nshots)]))


def compare(gpu, ref):
    """gpu, ref: [nt, nrec, 3] of one shot."""
    ref = np.asarray(ref, dtype=np.float64)
    gpu = np.asarray(gpu, dtype=np.float64)
    scale_e = max(np.linalg.norm(ref[..., 0]), np.linalg.norm(ref[..., 1]))
    scale = (scale_e, scale_e, np.linalg.norm(ref[..., 2]))
    for c in range(3):
        bound = max(np.linalg.norm(ref[..., c]), 1e-2 * scale[c])
        if bound == 0.0:
            # no field has reached the receivers yet (short runs): exactly zero on both sides
            assert not gpu[..., c].any(), c
            continue
        err = np.linalg.norm(gpu[..., c] - ref[..., c])
        assert err <= TRACE_TOL * bound, (c, err / max(np.linalg.norm(ref[..., c]), 1e-30))


def run_case(wl, dev, pol, shots=None, wav=None):
    from paper_2506_20513_gb300 import FDTD
    nsrc = wl.src.shape[1]
    wav = wavelets(wl, nsrc) if wav is None else wav
    fd = FDTD(wl.grid, wl.src, wl.rec, device=dev)
    tr = fd.forward_model_te(t32(wl.eps_true, dev), t32(wl.sig_true, dev), t32(wav, dev),
                             pol).cpu().numpy()
    fd.status()
    fd.close()
    assert tr.shape == (wl.nshots, wl.grid.nt, wl.rec.shape[1], 3)
    for s in (range(wl.nshots) if shots is None else shots):
        ref = O.forward_te_shot(wl.grid, wl.eps_true, wl.sig_true, pol, wl.src[s], wav[s],
                                wl.rec[s])["traces"]
        compare(tr[s], ref)
    return tr


@pytest.mark.parametrize("pol", [0, 1])
@pytest.mark.parametrize("seed,kappa,pec", [(31, 1.0, False), (32, 2.0, True)])
def test_small_random(dev, seed, kappa, pec, pol):
    wl = W.small_random(seed, nxp=46, nyp=27, npml=6, nt=150, nshots=3, nrec=9,
                        kappa_max=kappa, with_pec=pec)
    run_case(wl, dev, pol)


@pytest.mark.parametrize("pol", [0, 1])
def test_pec_box_without_cpml(dev, pol):
    wl = W.small_random(33, nxp=37, nyp=22, npml=0, nt=120, nshots=2, nrec=6)
    rec = wl.rec.copy()   # receivers off the walls (the acquisition must lie inside them)
    rec[..., 0] = np.clip(rec[..., 0], 1, wl.grid.nx - 2)
    rec[..., 1] = np.clip(rec[..., 1], 1, wl.grid.ny - 2)
    run_case(dataclasses.replace(wl, rec=rec), dev, pol)


@pytest.mark.parametrize("pol", [0, 1])
def test_several_sources_and_dense_receivers(dev, pol):
    """Three sources per shot, two of them in one cell; 300 receivers with duplicates."""
    wl = W.small_random(34, nxp=50, nyp=30, npml=5, nt=140, nshots=2, nrec=300)
    src = np.concatenate([wl.src, wl.src, wl.src], axis=1).copy()
    src[:, 2] = [5 + 31, 5 + 17]   # inside the 50 x 30 physical part
    rec = wl.rec.copy()
    rec[:, 1] = rec[:, 0]
    run_case(dataclasses.replace(wl, src=src, rec=rec), dev, pol)


@pytest.mark.parametrize("nt", [1, 2, 5])
def test_short_runs(dev, nt):
    """The receivers record before each step's updates: zero at n = 0."""
    wl = W.small_random(35, nxp=20, nyp=14, npml=3, nt=nt, nshots=2, nrec=4)
    rec = wl.rec.copy()
    rec[:, 0] = wl.src[:, 0]   # one receiver on the source cell: non-zero from n = 1
    tr = run_case(dataclasses.replace(wl, rec=rec), dev, 0)
    assert not tr[:, 0].any()
    if nt > 1:
        assert tr[:, 1, 0, 0].all()


def test_full_size_multishot_sampled(dev):
    """540x290 grid, 32 shots, nt 2000, 100 receivers: all shots on the GPU, two sampled
    shots recomputed by the oracle, for each polarisation."""
    wl = W.multishot_layered()
    wav = wavelets(wl, 1)
    for pol in (0, 1):
        run_case(wl, dev, pol, shots=[0, 31] if pol == 0 else [13], wav=wav)


def test_errors_and_workspace_reuse(dev):
    """Another polarisation is refused; a bad model is reported; a TE call between two TM
    calls leaves the TM traces unchanged, and drops a stored TM forward (adjoint refused)."""
    from paper_2506_20513_gb300 import FDTD
    wl = W.small_random(36, nxp=30, nyp=20, npml=4, nt=80, nshots=2, nrec=5)
    fd = FDTD(wl.grid, wl.src, wl.rec, device=dev)
    e, s = t32(wl.eps_true, dev), t32(wl.sig_true, dev)
    w = t32(wavelets(wl, 1), dev)
    with pytest.raises(_lib.GfError) as ex:
        fd.forward_model_te(e, s, w, 2)
    assert ex.value.code == _lib.GF_EINVAL
    bad = e.clone()
    bad[5, 5] = 0.5
    fd.forward_model_te(bad, s, w, 0)
    with pytest.raises(_lib.GfError) as ex:
        fd.status()
    assert ex.value.code == _lib.GF_EINVAL
    tm0 = fd.forward_model(e, s, w).cpu().numpy()
    te = fd.forward_model_te(e, s, w, 1).cpu().numpy()
    tm1 = fd.forward_model(e, s, w).cpu().numpy()
    assert np.array_equal(tm0, tm1)
    assert np.array_equal(te, fd.forward_model_te(e, s, w, 1).cpu().numpy())
    fd.forward(e, s, w)
    fd.forward_model_te(e, s, w, 0)
    with pytest.raises(_lib.GfError) as ex:
        fd.adjoint(e, s, t32(np.zeros((2, 80, 5)), dev))
    assert ex.value.code == _lib.GF_ESTATE
    fd.status()
    fd.close()


GRAD_TOL = 1e-3


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gradient_case(wl, dev, pol):
    from paper_2506_20513_gb300 import FDTD
    g = wl.grid
    wav = wavelets(wl, wl.src.shape[1])
    obs = np.stack([O.forward_te_shot(g, wl.eps_true, wl.sig_true, pol, wl.src[k], wav[k],
                                      wl.rec[k])["traces"][:, :, pol]
                    for k in range(wl.nshots)])
    fd = FDTD(g, wl.src, wl.rec, device=dev)
    e0, s0, w = t32(wl.eps_init, dev), t32(wl.sig_init, dev), t32(wav, dev)
    J, ge, gs, tr = fd.misfit_and_gradient_te(e0, s0, w, t32(obs, dev), pol,
                                              return_traces=True)
    fd.status()
    # the gradient call's traces are the forward model's
    assert torch.equal(tr, fd.forward_model_te(e0, s0, w, pol))
    # observed = its own traces: J = 0 and no gradient
    J0, ge0, gs0 = fd.misfit_and_gradient_te(e0, s0, w, tr[..., pol].contiguous(), pol)
    assert float(J0.item()) == 0.0 and not ge0.any() and not gs0.any()
    fd.status()
    fd.close()
    J64, ge64, gs64 = O.misfit_and_gradient_te(g, wl.eps_init, wl.sig_init, pol, wl.src, wav,
                                               wl.rec, obs)
    assert abs(float(J.item()) - J64) <= GRAD_TOL * J64
    assert rel(ge.cpu().numpy(), ge64) <= GRAD_TOL
    assert rel(gs.cpu().numpy(), gs64) <= GRAD_TOL


@pytest.mark.parametrize("pol", [0, 1])
@pytest.mark.parametrize("seed,kappa,pec", [(41, 1.0, False), (42, 2.0, True)])
def test_gradient_small_random(dev, seed, kappa, pec, pol):
    wl = W.small_random(seed, nxp=46, nyp=27, npml=6, nt=150, nshots=3, nrec=9,
                        kappa_max=kappa, with_pec=pec)
    gradient_case(wl, dev, pol)


def test_gradient_pec_box_and_several_sources(dev):
    """No CPML; three sources per shot (two in one cell), duplicate receivers."""
    wl = W.small_random(43, nxp=37, nyp=22, npml=0, nt=120, nshots=2, nrec=6)
    rec = wl.rec.copy()
    rec[..., 0] = np.clip(rec[..., 0], 1, wl.grid.nx - 2)
    rec[..., 1] = np.clip(rec[..., 1], 1, wl.grid.ny - 2)
    rec[:, 1] = rec[:, 0]
    src = np.concatenate([wl.src, wl.src, wl.src], axis=1).copy()
    src[:, 2] = [20, 12]
    gradient_case(dataclasses.replace(wl, src=src, rec=rec), dev, 1)


@pytest.mark.parametrize("pol", [0, 1])
def test_gradient_larger_grid(dev, pol):
    """110 x 84 physical cells with an 8-cell CPML, nt 400, two shots, a perfect conductor."""
    wl = W.small_random(44, nxp=110, nyp=84, npml=8, nt=400, nshots=2, nrec=12,
                        with_pec=True)
    gradient_case(wl, dev, pol)


def test_gradient_errors(dev):
    from paper_2506_20513_gb300 import FDTD
    wl = W.small_random(45, nxp=20, nyp=14, npml=3, nt=20, nshots=1, nrec=3)
    fd = FDTD(wl.grid, wl.src, wl.rec, device=dev)
    e, s = t32(wl.eps_init, dev), t32(wl.sig_init, dev)
    w = t32(wavelets(wl, 1), dev)
    obs = t32(np.zeros((1, 20, 3)), dev)
    with pytest.raises(_lib.GfError) as ex:
        fd.misfit_and_gradient_te(e, s, w, obs, 2)
    assert ex.value.code == _lib.GF_EINVAL
    fd.close()


def test_misfit_alone_and_fwi_on_the_te_mode(dev):
    """gf_misfit_te gives the gradient call's J bit for bit; the L-BFGS driver inverts the
    x-polarised traces through TEMode: its first misfit is the oracle's, and every accepted
    step lowers it."""
    from paper_2506_20513_gb300 import FDTD, TEMode
    from paper_2506_20513_gb300.fwi import FWI, FWIConfig, interior_mask
    wl = W.small_random(46, nxp=46, nyp=27, npml=6, nt=150, nshots=3, nrec=9)
    g = wl.grid
    wav = wavelets(wl, 1)
    obs = np.stack([O.forward_te_shot(g, wl.eps_true, wl.sig_true, 0, wl.src[k], wav[k],
                                      wl.rec[k])["traces"][:, :, 0]
                    for k in range(wl.nshots)])
    fd = FDTD(g, wl.src, wl.rec, device=dev)
    e0, s0, w, o = (t32(a, dev) for a in (wl.eps_init, wl.sig_init, wav, obs))
    J1 = fd.misfit_te(e0, s0, w, o, 0)
    J2, _, _ = fd.misfit_and_gradient_te(e0, s0, w, o, 0)
    assert float(J1.item()) == float(J2.item())
    J64, _, _ = O.misfit_and_gradient_te(g, wl.eps_init, wl.sig_init, 0, wl.src, wav, wl.rec,
                                         obs)
    inv = FWI(TEMode(fd, 0), lambda f0: o, interior_mask(g, rows_below_top=2),
              FWIConfig(bands=((wl.f0, 6),)))
    eps, sig, hist = inv.run(e0, s0)
    fd.status()
    fd.close()
    assert abs(hist.misfit[0] - J64) <= GRAD_TOL * J64
    seq = hist.misfit + [hist.final_misfit]
    assert all(b <= a for a, b in zip(seq, seq[1:]))
    assert hist.final_misfit < 0.9 * hist.misfit[0]
