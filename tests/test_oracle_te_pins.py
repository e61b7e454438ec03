"""Pins of the oracle's TE-mode forward model (x- and y-polarised sources, Sec. 3.2 source
listing; fields Ex, Ey, Hz) against what the mathematics fixes:

* the analytic field of an x-directed line current in a homogeneous medium (Hankel
  functions, lossless and lossy), on the line through the source across the current and on
  the line along it -- for the y-polarised source with the axes exchanged -- and its Hz
  through Faraday's law;
* exact discrete energy conservation of the lossless scheme in a PEC box, and decay with
  Ohmic loss;
* source-receiver reciprocity, co-polar and cross-polar, in a heterogeneous lossy medium;
* CPML absorption against a domain large enough that no reflection arrives.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2506_20513_gb300 import workloads as W


def _pec_box(nx=48, ny=40, nt=400, dx=0.01, seed=0, lossy=False):
    g = W.GridSpec(nx=nx, ny=ny, npml=0, nt=nt, dx=dx, dy=dx, dt=0.95 * W.cfl_dt_max(dx, dx))
    rng = np.random.default_rng(seed)
    eps = 1.0 + 8.0 * rng.random((ny, nx))
    sig = (5e-3 * rng.random((ny, nx))) if lossy else np.zeros((ny, nx))
    return g, eps, sig


@pytest.mark.parametrize("pol", [0, 1])
def test_te_energy_conserved_lossless_pec_box(pol):
    """W^n = sum(eps (Ex^n^2 + Ey^n^2) + mu0 Hz^{n-1/2} Hz^{n+1/2}) is exactly constant once
    the source has stopped (heterogeneous eps_r, sigma = 0, no CPML)."""
    g, eps, sig = _pec_box()
    wav = O.ricker(1.5e9, g.dt, g.nt)
    wav[120:] = 0.0
    out = O.forward_te_shot(g, eps, sig, pol, [[20, 17]], wav[None], [[30, 30]], energy=True)
    E = out["energy"][121:]
    assert E[0] > 0
    assert np.max(np.abs(E - E[0])) / E[0] < 1e-12


def test_te_energy_decays_lossy():
    g, eps, sig = _pec_box(lossy=True)
    wav = O.ricker(1.5e9, g.dt, g.nt)
    wav[120:] = 0.0
    E = O.forward_te_shot(g, eps, sig, 0, [[20, 17]], wav[None], [[30, 30]],
                          energy=True)["energy"][121:]
    assert np.all(np.diff(E) <= 1e-12 * E[0])
    assert E[-1] < 0.999 * E[0]


def test_te_reciprocity_pec_box():
    """Swapping source and receiver gives the same trace, for the same component
    (Ex -> Ex) and across components (an x-source seen in Ey equals a y-source seen in Ex),
    in a heterogeneous lossy PEC box."""
    g, eps, sig = _pec_box(seed=3, lossy=True)
    wav = O.ricker(1.5e9, g.dt, g.nt)
    a, b = [11, 9], [35, 29]
    ab_x = O.forward_te_shot(g, eps, sig, 0, [a], wav[None], [b])["traces"][:, 0]
    ba_x = O.forward_te_shot(g, eps, sig, 0, [b], wav[None], [a])["traces"][:, 0]
    ba_y = O.forward_te_shot(g, eps, sig, 1, [b], wav[None], [a])["traces"][:, 0]
    s = np.abs(ab_x[:, 0]).max()
    assert s > 0 and np.abs(ab_x[:, 1]).max() > 1e-3 * s
    assert np.max(np.abs(ab_x[:, 0] - ba_x[:, 0])) <= 1e-10 * s
    assert np.max(np.abs(ab_x[:, 1] - ba_y[:, 0])) <= 1e-10 * s


@pytest.mark.parametrize("eps_r,sigma", [(1.0, 0.0), (4.0, 5e-3)])
def test_te_analytic_dipole_line_source(eps_r, sigma):
    """Ex at 0.6 m from a 100 MHz Ricker x-directed line current, across and along the
    current, vs the Hankel-function solution (>= 50 cells per wavelength at 3 f0).  The Ex
    node of cell (i, j) sits at (i + 1/2, j), so the receivers (c, c + m) and (c + m, c) lie
    exactly on the two lines through the source node (c, c).  As in the TM mode, the current
    of step n acts at (n + 1/2) dt.  The y-polarised source gives the same traces in Ey with
    the axes exchanged."""
    dx, f0, npml = 0.01, 100e6, 20
    g = W.default_pml(W.GridSpec(nx=2 * npml + 260, ny=2 * npml + 260, npml=npml, nt=0, dx=dx,
                                 dy=dx, dt=0.0), f0)
    dt = 0.5 * W.cfl_dt_max(dx, dx)
    rho = 0.6
    t_end = math.sqrt(2.0) / f0 * 2.0 + rho / (W.C0 / math.sqrt(eps_r)) + 1.5 / f0
    nt = int(t_end / dt)
    g.dt, g.nt = dt, nt
    c = g.nx // 2
    m = int(round(rho / dx))
    eps = np.full((g.ny, g.nx), eps_r)
    sig = np.full((g.ny, g.nx), sigma)
    wav = O.ricker(f0, dt, nt)
    cur = O.ricker(f0, dt, nt, t0=math.sqrt(2.0) / f0 + 0.5 * dt)
    across = O.dipole_line_source_trace(cur, dt, m * dx, eps_r, sigma, along=False)
    along = O.dipole_line_source_trace(cur, dt, m * dx, eps_r, sigma, along=True)
    tx = O.forward_te_shot(g, eps, sig, 0, [[c, c]], wav[None], [[c, c + m], [c + m, c]])
    ty = O.forward_te_shot(g, eps, sig, 1, [[c, c]], wav[None], [[c + m, c], [c, c + m]])
    for tr, comp in ((tx["traces"], 0), (ty["traces"], 1)):
        for k, ana in enumerate((across, along)):
            num = tr[:, k, comp]
            corr = np.dot(num, ana) / (np.linalg.norm(num) * np.linalg.norm(ana))
            rel = np.linalg.norm(num - ana) / np.linalg.norm(ana)
            # measured: rel 2e-4 (lossless), 2e-4 to 4e-4 (lossy); a half step of delay
            # dropped or a dropped H1 / (k rho) term gives far more, a wrong sign O(1)
            assert corr >= 0.99999, (comp, k, corr)
            assert rel <= 2e-3, (comp, k, rel)
    # the two polarisations are mirror images of one another on a square grid
    np.testing.assert_allclose(ty["traces"][:, :, 1], tx["traces"][:, :, 0], rtol=0,
                               atol=1e-9 * np.abs(tx["traces"][:, :, 0]).max())


@pytest.mark.parametrize("eps_r,sigma", [(1.0, 0.0), (4.0, 5e-3)])
def test_te_analytic_magnetic_component(eps_r, sigma):
    """The receivers' Hz against Faraday's law applied to the vector potential of the
    x-directed line current: Hz = -dG/dy I = -(j k / 4) I H1^(2)(k y) on the line across the
    current (y > 0).  The Hz node of cell (c, c + m) sits at y = (m + 1/2) dy on that line and
    is sampled half a step before E^n (Hz^{n-1/2}), so the analytic current is the wavelet
    delayed by a whole step; the node of cell (c, c - m - 1), at -(m + 1/2) dy, is its mirror
    image with the opposite sign."""
    dx, f0, npml = 0.01, 100e6, 20
    g = W.default_pml(W.GridSpec(nx=2 * npml + 260, ny=2 * npml + 260, npml=npml, nt=0, dx=dx,
                                 dy=dx, dt=0.0), f0)
    dt = 0.5 * W.cfl_dt_max(dx, dx)
    rho = 0.6
    t_end = math.sqrt(2.0) / f0 * 2.0 + rho / (W.C0 / math.sqrt(eps_r)) + 1.5 / f0
    g.dt, g.nt = dt, int(t_end / dt)
    c = g.nx // 2
    m = int(round(rho / dx))
    eps = np.full((g.ny, g.nx), eps_r)
    sig = np.full((g.ny, g.nx), sigma)
    tr = O.forward_te_shot(g, eps, sig, 0, [[c, c]], O.ricker(f0, dt, g.nt)[None],
                           [[c, c + m], [c, c - m - 1]])["traces"]
    cur = O.ricker(f0, dt, g.nt, t0=math.sqrt(2.0) / f0 + dt)
    ana = O.line_source_hy_trace(cur, dt, (m + 0.5) * dx, eps_r, sigma)
    hz = tr[:, 0, 2]
    corr = np.dot(hz, ana) / (np.linalg.norm(hz) * np.linalg.norm(ana))
    rel = np.linalg.norm(hz - ana) / np.linalg.norm(ana)
    # measured: rel 1e-4 (lossless), 4e-4 (lossy); half a step of timing off gives 4.5e-3
    assert corr >= 0.99999, corr
    assert rel <= 2e-3, rel
    assert np.abs(hz + tr[:, 1, 2]).max() <= 1e-5 * np.abs(hz).max()


def test_te_cpml_reflection_below_minus_40db():
    """Traces with a 20-cell CPML vs the same traces in a domain so large that no echo
    arrives inside the window, for every component."""
    dx, f0 = 0.01, 400e6
    dt = 0.9 * W.cfl_dt_max(dx, dx)
    nt = 700
    npml, n = 20, 100

    def run(nphys):
        g = W.default_pml(W.GridSpec(nx=nphys + 2 * npml, ny=nphys + 2 * npml, npml=npml,
                                     nt=nt, dx=dx, dy=dx, dt=dt), f0)
        c = g.nx // 2
        eps = np.full((g.ny, g.nx), 4.0)
        sig = np.full((g.ny, g.nx), 1e-3)
        return O.forward_te_shot(g, eps, sig, 0, [[c, c]], O.ricker(f0, dt, nt)[None],
                                 [[c + 35, c + 10]])["traces"][:, 0]

    small = run(n)
    big = run(n + 2 * 400)
    for comp in range(3):
        err = np.max(np.abs(small[:, comp] - big[:, comp])) / np.max(np.abs(big[:, comp]))
        assert 20 * math.log10(err) < -40.0, comp


def test_te_rejects_other_polarisations():
    g, eps, sig = _pec_box(nt=4)
    with pytest.raises(ValueError):
        O.forward_te_shot(g, eps, sig, 2, [[20, 17]], np.zeros((1, 4)), [[30, 30]])


@pytest.mark.parametrize("pol,kappa,pec", [(0, 2.0, True), (1, 1.0, False)])
def test_te_misfit_gradient_fd_every_cell(pol, kappa, pec):
    """The adjoint gradient of J = 1/2 sum (d - o)^2 over the source component's traces
    against central differences at every cell of a tiny grid (CPML, two shots, lossy
    heterogeneous model; kappa_max 2 and a perfect conductor in one case).  Every cell
    carries a gradient: the cells of the outer rows and columns hold one updated E
    component each."""
    wl = W.small_random(13, nxp=12, nyp=10, npml=3, nt=90, nshots=2, nrec=4,
                        kappa_max=kappa, with_pec=pec)
    g = wl.grid
    wav = np.stack([O.ricker(wl.f0, g.dt, g.nt)[None]] * wl.nshots)

    def traces(e, s):
        return np.stack([O.forward_te_shot(g, e, s, pol, wl.src[k], wav[k], wl.rec[k])
                         ["traces"][:, :, pol] for k in range(wl.nshots)])

    obs = traces(wl.eps_true, wl.sig_true)
    e0, s0 = wl.eps_init.copy(), wl.sig_init.copy()
    J, ge, gs = O.misfit_and_gradient_te(g, e0, s0, pol, wl.src, wav, wl.rec, obs)
    assert J > 0
    assert J == pytest.approx(0.5 * np.sum((traces(e0, s0) - obs) ** 2), rel=1e-12)

    def Jof(e, s):
        return 0.5 * np.sum((traces(e, s) - obs) ** 2)

    fde = np.zeros_like(ge)
    fds = np.zeros_like(gs)
    for j in range(g.ny):
        for i in range(g.nx):
            he = 1e-6 * e0[j, i]
            hs = 1e-6 * s0[j, i]
            ep, em = e0.copy(), e0.copy()
            ep[j, i] += he
            em[j, i] -= he
            fde[j, i] = (Jof(ep, s0) - Jof(em, s0)) / (2 * he)
            sp, sm = s0.copy(), s0.copy()
            sp[j, i] += hs
            sm[j, i] -= hs
            fds[j, i] = (Jof(e0, sp) - Jof(e0, sm)) / (2 * hs)
    for a, b in ((ge, fde), (gs, fds)):
        assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(a)
    # the corner cell (nx-1, ny-1) holds no updated component
    assert ge[-1, -1] == 0 and gs[-1, -1] == 0
