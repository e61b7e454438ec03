"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself:
* the analytic 2-D line-source solution of Maxwell's equations (Eqs. faraday, ampere),
* exact discrete energy conservation of the lossless Yee scheme (Eqs. 3-5), and energy
  decay with Ohmic loss,
* source-receiver reciprocity,
* the adjoint dot-product test against an independently written tangent-linear model,
  which in turn is pinned by central finite differences,
* central finite differences of the misfit (Eq. objective) at every cell of a tiny grid,
* the identity between the zero-lag gradient form (Eqs. grad_sigma, grad_eps) and the
  coefficient-chain-rule form of the coefficient listing (Sec. 3.2),
* the CFL bound (Eq. cfl) on the paper's own stable configurations (tests/golden),
* CPML absorption against a domain large enough that no reflection arrives.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2506_20513_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _pec_box(nx=48, ny=40, nt=400, dx=0.01, seed=0, lossy=False):
    g = W.GridSpec(nx=nx, ny=ny, npml=0, nt=nt, dx=dx, dy=dx, dt=0.95 * W.cfl_dt_max(dx, dx))
    rng = np.random.default_rng(seed)
    eps = 1.0 + 8.0 * rng.random((ny, nx))
    sig = (5e-3 * rng.random((ny, nx))) if lossy else np.zeros((ny, nx))
    return g, eps, sig


def test_ricker_closed_form():
    """Peak A at t0, zero crossings at t0 +- 1/(sqrt(2) pi f0), zero mean."""
    f0, dt = 200e6, 1e-12
    nt = 40000
    w = O.ricker(f0, dt, nt, amp=2.5)
    t0 = math.sqrt(2.0) / f0
    n0 = int(round(t0 / dt))
    assert w[n0] == pytest.approx(2.5, rel=1e-6)
    tz = t0 + 1.0 / (math.sqrt(2.0) * math.pi * f0)
    nz = int(tz / dt)
    assert w[nz] > 0 > w[nz + 1]
    assert abs(w.sum() * dt) < 1e-6 * np.abs(w).max() * t0


def test_energy_conserved_lossless_pec_box():
    """W^n = sum(eps Ez^n^2 + mu0 H^{n-1/2} H^{n+1/2}) is exactly constant once the source
    has stopped (PEC box, sigma = 0, no CPML)."""
    g, eps, sig = _pec_box()
    wav = O.ricker(1.5e9, g.dt, g.nt)
    wav[120:] = 0.0  # switch the source off
    out = O.forward_shot(g, eps, sig, [[20, 17]], wav[None], [[30, 30]], energy=True)
    E = out["energy"][121:]
    assert E[0] > 0
    assert np.max(np.abs(E - E[0])) / E[0] < 1e-12


def test_energy_decays_lossy():
    g, eps, sig = _pec_box(lossy=True)
    wav = O.ricker(1.5e9, g.dt, g.nt)
    wav[120:] = 0.0
    E = O.forward_shot(g, eps, sig, [[20, 17]], wav[None], [[30, 30]], energy=True)["energy"][121:]
    assert np.all(np.diff(E) <= 1e-12 * E[0])
    assert E[-1] < 0.999 * E[0]


def test_reciprocity_pec_box():
    """Swapping source and receiver gives the same trace (heterogeneous, lossy, PEC box)."""
    g, eps, sig = _pec_box(seed=3, lossy=True)
    wav = O.ricker(1.5e9, g.dt, g.nt)
    a, b = [11, 9], [35, 29]
    tab = O.forward_shot(g, eps, sig, [a], wav[None], [b])["traces"][:, 0]
    tba = O.forward_shot(g, eps, sig, [b], wav[None], [a])["traces"][:, 0]
    assert np.abs(tab).max() > 0
    assert np.max(np.abs(tab - tba)) <= 1e-10 * np.abs(tab).max()


@pytest.mark.parametrize("kappa_max,pec", [(1.0, False), (2.0, True)])
def test_tangent_linear_vs_central_difference(kappa_max, pec):
    """The tangent-linear model is the derivative of the forward traces."""
    wl = W.small_random(5, kappa_max=kappa_max, with_pec=pec)
    g = wl.grid
    wav = O.ricker(wl.f0, g.dt, g.nt)[None]
    rng = np.random.default_rng(1)
    de = rng.standard_normal((g.ny, g.nx))
    ds = 1e-3 * rng.standard_normal((g.ny, g.nx))
    tl = O.tangent(g, wl.eps_true, wl.sig_true, de, ds, wl.src[0], wav, wl.rec[0])
    h = 1e-6
    fp = O.forward_shot(g, wl.eps_true + h * de, wl.sig_true + h * ds, wl.src[0], wav, wl.rec[0])
    fm = O.forward_shot(g, wl.eps_true - h * de, wl.sig_true - h * ds, wl.src[0], wav, wl.rec[0])
    fd = (fp["traces"] - fm["traces"]) / (2 * h)
    assert np.linalg.norm(fd - tl) / np.linalg.norm(tl) < 1e-6


@pytest.mark.parametrize("kappa_max,pec", [(1.0, False), (2.0, True)])
def test_adjoint_dot_product(kappa_max, pec):
    """<T dm, r> = <dm, A r> with T the tangent-linear model and A the adjoint."""
    wl = W.small_random(7, kappa_max=kappa_max, with_pec=pec)
    g = wl.grid
    wav = O.ricker(wl.f0, g.dt, g.nt)[None]
    fw = O.forward_shot(g, wl.eps_true, wl.sig_true, wl.src[0], wav, wl.rec[0], history=True)
    rng = np.random.default_rng(2)
    r = rng.standard_normal(fw["traces"].shape)
    adj = O.adjoint_shot(g, wl.eps_true, wl.sig_true, wl.src[0], wl.rec[0], r, fw["ez_hist"])
    de = rng.standard_normal((g.ny, g.nx))
    ds = 1e-3 * rng.standard_normal((g.ny, g.nx))
    tl = O.tangent(g, wl.eps_true, wl.sig_true, de, ds, wl.src[0], wav, wl.rec[0])
    lhs = float(np.sum(tl * r))
    rhs = float(np.sum(adj["g_eps_r"] * de) + np.sum(adj["g_sigma"] * ds))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_zero_lag_identity():
    """The zero-lag form lam (E^{n+1} -+ E^n) equals the coefficient chain rule."""
    wl = W.small_random(11, kappa_max=2.0, with_pec=True)
    g = wl.grid
    wav = O.ricker(wl.f0, g.dt, g.nt)[None]
    fw = O.forward_shot(g, wl.eps_init, wl.sig_init, wl.src[0], wav, wl.rec[0], history=True,
                        qhistory=True)
    r = np.random.default_rng(3).standard_normal(fw["traces"].shape)
    adj = O.adjoint_shot(g, wl.eps_init, wl.sig_init, wl.src[0], wl.rec[0], r, fw["ez_hist"],
                         fw["q_hist"])
    for a, b in (("g_eps_r", "gc_eps_r"), ("g_sigma", "gc_sigma")):
        scale = np.abs(adj[a]).max()
        assert scale > 0
        assert np.abs(adj[a] - adj[b]).max() <= 1e-12 * scale


def test_misfit_gradient_fd_every_cell():
    """Central differences of J = 1/2 sum (d - o)^2 at every cell of a tiny grid with CPML,
    two shots and a lossy heterogeneous model."""
    wl = W.small_random(13, nxp=12, nyp=10, npml=3, nt=90, nshots=2, nrec=4)
    g = wl.grid
    wav = np.stack([O.ricker(wl.f0, g.dt, g.nt)[None]] * wl.nshots)
    obs = O.forward(g, wl.eps_true, wl.sig_true, wl.src, wav, wl.rec)
    e0, s0 = wl.eps_init.copy(), wl.sig_init.copy()
    J, ge, gs = O.misfit_and_gradient(g, e0, s0, wl.src, wav, wl.rec, obs)
    assert J > 0

    def Jof(e, s):
        d = O.forward(g, e, s, wl.src, wav, wl.rec)
        return 0.5 * np.sum((d - obs) ** 2)

    fde = np.zeros_like(ge)
    fds = np.zeros_like(gs)
    for j in range(1, g.ny - 1):
        for i in range(1, g.nx - 1):
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
    # the PEC ring carries no gradient
    assert np.all(ge[0, :] == 0) and np.all(gs[:, -1] == 0)


def test_wavelet_gradient_is_exact():
    """J is quadratic in the source samples: a central difference is exact up to rounding."""
    wl = W.small_random(17, nt=80)
    g = wl.grid
    wav = O.ricker(wl.f0, g.dt, g.nt)[None]
    obs = np.random.default_rng(4).standard_normal((g.nt, wl.nrec))
    fw = O.forward_shot(g, wl.eps_true, wl.sig_true, wl.src[0], wav, wl.rec[0], history=True)
    adj = O.adjoint_shot(g, wl.eps_true, wl.sig_true, wl.src[0], wl.rec[0],
                         fw["traces"] - obs, fw["ez_hist"])
    for n in (5, 20, 41):
        h = 1e-3
        wp, wm = wav.copy(), wav.copy()
        wp[0, n] += h
        wm[0, n] -= h
        Jp = 0.5 * np.sum((O.forward_shot(g, wl.eps_true, wl.sig_true, wl.src[0], wp,
                                          wl.rec[0])["traces"] - obs) ** 2)
        Jm = 0.5 * np.sum((O.forward_shot(g, wl.eps_true, wl.sig_true, wl.src[0], wm,
                                          wl.rec[0])["traces"] - obs) ** 2)
        fd = (Jp - Jm) / (2 * h)
        assert adj["g_wav"][0, n] == pytest.approx(fd, rel=1e-7, abs=1e-9 * abs(fd) + 1e-12)


@pytest.mark.parametrize("eps_r,sigma", [(1.0, 0.0), (4.0, 5e-3)])
def test_analytic_line_source(eps_r, sigma):
    """Homogeneous medium, trace at rho = 0.6 m from a 100 MHz Ricker line current vs the
    Hankel-function solution; >= 50 cells per wavelength at 3 f0 (negligible dispersion).
    The source current of step n acts at t = (n + 1/2) dt (Ampere's law is centred on the
    half step), so the analytic current is the wavelet delayed by dt/2."""
    dx, f0, npml = 0.01, 100e6, 20
    g = W.default_pml(W.GridSpec(nx=2 * npml + 260, ny=2 * npml + 260, npml=npml, nt=0, dx=dx,
                                 dy=dx, dt=0.0), f0)
    dt = 0.5 * W.cfl_dt_max(dx, dx)
    v = W.C0 / math.sqrt(eps_r)
    rho = 0.6
    # window: the whole Ricker pulse plus the arrival, ending before a boundary echo
    t_end = math.sqrt(2.0) / f0 * 2.0 + rho / v + 1.5 / f0
    nt = int(t_end / dt)
    g.dt, g.nt = dt, nt
    c = g.nx // 2
    src = [[c, c]]
    rec = [[c + int(round(rho / dx)), c]]
    eps = np.full((g.ny, g.nx), eps_r)
    sig = np.full((g.ny, g.nx), sigma)
    wav = O.ricker(f0, dt, nt)
    num = O.forward_shot(g, eps, sig, src, wav[None], rec)["traces"][:, 0]
    cur = O.ricker(f0, dt, nt, t0=math.sqrt(2.0) / f0 + 0.5 * dt)
    ana = O.line_source_trace(cur, dt, rho, eps_r, sigma)
    corr = np.dot(num, ana) / (np.linalg.norm(num) * np.linalg.norm(ana))
    rel = np.linalg.norm(num - ana) / np.linalg.norm(ana)
    # measured: rel 6e-5 (lossless), 5e-4 (lossy); dropping the half-step source delay
    # gives 5e-3 and a wrong source sign or scale gives O(1), so 2e-3 pins both
    assert corr >= 0.99999, corr
    assert rel <= 2e-3, rel


@pytest.mark.parametrize("eps_r,sigma", [(1.0, 0.0), (4.0, 5e-3)])
def test_analytic_line_source_magnetic_components(eps_r, sigma):
    """The receivers' magnetic components against Faraday's law applied to the Hankel
    solution: on the +x axis Hy = -(j k / 4) I H1^(2)(k x) and Hx = 0.  Hy of receiver cell
    i sits half a cell further out (x = rho + dx / 2) and is sampled half a step before Ez^n
    (H^{n-1/2}), so the analytic current is the wavelet delayed by a whole step."""
    dx, f0, npml = 0.01, 100e6, 20
    g = W.default_pml(W.GridSpec(nx=2 * npml + 260, ny=2 * npml + 260, npml=npml, nt=0, dx=dx,
                                 dy=dx, dt=0.0), f0)
    dt = 0.5 * W.cfl_dt_max(dx, dx)
    v = W.C0 / math.sqrt(eps_r)
    rho = 0.6
    t_end = math.sqrt(2.0) / f0 * 2.0 + rho / v + 1.5 / f0
    nt = int(t_end / dt)
    g.dt, g.nt = dt, nt
    c = g.nx // 2
    i_r = c + int(round(rho / dx))
    eps = np.full((g.ny, g.nx), eps_r)
    sig = np.full((g.ny, g.nx), sigma)
    wav = O.ricker(f0, dt, nt)
    # the receiver on the axis and its mirror one row below it
    out = O.forward_shot(g, eps, sig, [[c, c]], wav[None], [[i_r, c], [i_r, c - 1]],
                         fields=True)
    hx, hy = out["h_traces"][:, 0, 0], out["h_traces"][:, 0, 1]
    hx_below = out["h_traces"][:, 1, 0]
    cur = O.ricker(f0, dt, nt, t0=math.sqrt(2.0) / f0 + dt)
    ana = O.line_source_hy_trace(cur, dt, (i_r - c + 0.5) * dx, eps_r, sigma)
    corr = np.dot(hy, ana) / (np.linalg.norm(hy) * np.linalg.norm(ana))
    rel = np.linalg.norm(hy - ana) / np.linalg.norm(ana)
    # measured: rel 1e-4 (lossless); the half-cell offset or the half-step delay dropped gives
    # 4e-3 to 1e-2, a wrong sign O(1)
    assert corr >= 0.99999, corr
    assert rel <= 2e-3, rel
    # Hx of the receiver cell sits half a cell above the axis (y = +dx/2), that of the cell
    # below half a cell under it: mirror images, so they are opposite (up to the absorbing
    # layer's small reflections, which the grid does not place symmetrically: 1e-5)
    assert np.abs(hx).max() > 1e-3 * np.abs(hy).max()
    assert np.abs(hx + hx_below).max() <= 1e-4 * np.abs(hx).max()
    # and the Ez receivers are unchanged by asking for the magnetic components
    ez = O.forward_shot(g, eps, sig, [[c, c]], wav[None], [[i_r, c], [i_r, c - 1]])["traces"]
    assert np.array_equal(ez, out["traces"])


def test_cpml_reflection_below_minus_40db():
    """Trace with a 20-cell CPML vs the same trace in a domain so large that no echo
    arrives inside the window."""
    dx, f0 = 0.01, 400e6
    dt = 0.9 * W.cfl_dt_max(dx, dx)
    nt = 700
    npml, n = 20, 100

    def run(nphys, npml_):
        g = W.default_pml(W.GridSpec(nx=nphys + 2 * npml_, ny=nphys + 2 * npml_, npml=npml_,
                                     nt=nt, dx=dx, dy=dx, dt=dt), f0)
        c = g.nx // 2
        eps = np.full((g.ny, g.nx), 4.0)
        sig = np.full((g.ny, g.nx), 1e-3)
        src = [[c, c]]
        rec = [[c + 35, c + 10]]  # 15 cells from the absorbing layer in the small domain
        return O.forward_shot(g, eps, sig, src, O.ricker(f0, dt, nt)[None], rec)["traces"][:, 0]

    small = run(n, npml)
    big = run(n + 2 * 400, npml)
    err = np.max(np.abs(small - big)) / np.max(np.abs(big))
    assert 20 * math.log10(err) < -40.0


def test_cfl_on_paper_configurations():
    """Every configuration the paper ran satisfies Eq. cfl (vacuum speed of light)."""
    with open(os.path.join(GOLDEN, "paper_tables.json")) as f:
        tables = json.load(f)
    for name, t in tables["configurations"].items():
        dtmax = W.cfl_dt_max(t["dx"], t["dy"])
        assert 0.8 * dtmax < t["dt"] <= dtmax, name


@pytest.mark.parametrize("factor,stable", [(0.99, True), (1.02, False)])
def test_cfl_bound_is_the_stability_limit(factor, stable):
    """In vacuum the scheme is stable just below the Eq. cfl step and blows up just above
    it (energy of a PEC box, random initial excitation through the source)."""
    dx = 0.01
    g = W.GridSpec(nx=48, ny=48, npml=0, nt=1500, dx=dx, dy=dx,
                   dt=factor * W.cfl_dt_max(dx, dx))
    eps = np.ones((g.ny, g.nx))
    sig = np.zeros((g.ny, g.nx))
    wav = np.zeros(g.nt)
    wav[:5] = np.random.default_rng(0).standard_normal(5)
    tr = O.forward_shot(g, eps, sig, [[24, 24]], wav[None], [[10, 30]])["traces"][:, 0]
    growth = np.abs(tr[-200:]).max() / np.abs(tr[:200]).max()
    assert (growth < 10.0) == stable, growth
