"""Seeded synthetic workloads: grids, acquisition geometry and layered/anomaly models.

This module only generates inputs.  It holds none of the method's arithmetic (no field
update, coefficient, CPML or gradient formula); the CUDA path and the CPU oracle both take
its arrays as plain inputs, so parity never depends on how an input was drawn.

Grids follow the paper's convention that model arrays include the absorbing layer
(Sec. 3.1 demo script, which strips ``pmlthick`` cells from each side before saving):
an array is [ny][nx] = [ny_phys + 2 npml][nx_phys + 2 npml], x (horizontal) fastest, y
(depth) second.  Positions in metres are measured from the top-left corner of the physical
domain and map to cells by rounding half up, offset by npml.

The workload shapes follow the paper's experiments (Sec. 4: 10^4-10^5 cells, nt 350-1000,
1-200 receivers, 100-500 MHz Ricker sources, relative permittivity 3-12).  The paper's own
models (landfill, Overthrust, sand-pit field data) are not available; the layered + Gaussian
blob generator below stands in for them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

EPS0 = 8.8541878128e-12
C0 = 299792458.0


@dataclass
class GridSpec:
    """Padded FDTD grid and CPML parameters (the fields of ``gf_grid_desc``)."""
    nx: int
    ny: int
    npml: int
    nt: int
    dx: float
    dy: float
    dt: float
    pml_order: int = 3
    pml_sigma_max: float = 0.0  # <= 0: default grading 0.8 (m+1) / (eta0 d sqrt(eps_ref))
    pml_kappa_max: float = 1.0
    pml_alpha_max: float = 0.0
    pml_eps_ref: float = 1.0

    @property
    def ncells(self) -> int:
        return self.nx * self.ny


@dataclass
class Workload:
    name: str
    grid: GridSpec
    f0: float
    src: np.ndarray  # [nshots, nsrc, 2] int32 cell indices (i, j)
    rec: np.ndarray  # [nshots, nrec, 2]
    eps_true: np.ndarray  # [ny, nx] float64
    sig_true: np.ndarray
    eps_init: np.ndarray
    sig_init: np.ndarray
    seed: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def nshots(self) -> int:
        return int(self.src.shape[0])

    @property
    def nrec(self) -> int:
        return int(self.rec.shape[1])

    def cell_updates(self) -> int:
        """Forward + adjoint cell-updates of one gradient: 2 * N * nt * nshots."""
        return 2 * self.grid.ncells * self.grid.nt * self.nshots


def cell_of(pos_m: float, d: float, npml: int) -> int:
    """Metres from the physical origin -> padded cell index (round half up)."""
    return npml + int(math.floor(pos_m / d + 0.5))


def pad_edges(a: np.ndarray, npml: int) -> np.ndarray:
    """Extend a physical model into the absorbing layer by edge replication."""
    return np.pad(a, npml, mode="edge")


def default_pml(grid: GridSpec, f0: float) -> GridSpec:
    """CPML grading used by every workload: cubic, kappa_max 1, alpha_max = 2 pi eps0 f0."""
    return replace(grid, pml_order=3, pml_sigma_max=0.0, pml_kappa_max=1.0,
                   pml_alpha_max=2.0 * math.pi * EPS0 * f0, pml_eps_ref=1.0)


def cfl_dt_max(dx: float, dy: float) -> float:
    """Largest stable time step in vacuum (Eq. cfl)."""
    return 1.0 / (C0 * math.sqrt(1.0 / dx ** 2 + 1.0 / dy ** 2))


# ------------------------------------------------------------------------------------------
# Random layered + blob models
# ------------------------------------------------------------------------------------------
def _layer_blob_field(rng, nxp, nyp, dx, lo, hi, nlayers, nblobs, blob_amp, rmin=0.05,
                      rmax=0.3):
    ys = np.sort(rng.uniform(0.0, nyp * dx, size=nlayers - 1))
    vals = rng.uniform(lo, hi, size=nlayers)
    y = (np.arange(nyp) * dx)[:, None]
    x = (np.arange(nxp) * dx)[None, :]
    layer = np.searchsorted(ys, y[:, 0])
    f = np.repeat(vals[layer][:, None], nxp, axis=1).astype(np.float64)
    for _ in range(nblobs):
        cx, cy = rng.uniform(0, nxp * dx), rng.uniform(0, nyp * dx)
        R = rng.uniform(rmin, rmax)
        A = rng.uniform(-blob_amp, blob_amp)
        f += A * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * R * R))
    return np.clip(f, lo, hi)


def layered_blob_model(seed: int, nxp: int, nyp: int, dx: float, eps_range=(3.0, 12.0),
                       sig_range_mS=(0.1, 20.0), rho: float = 0.6):
    """Physical-domain (eps_r, sigma [S/m]) of a seeded layered + Gaussian-blob model.

    eps_r: 3-6 horizontal layers uniform in ``eps_range`` plus 5-10 Gaussian blobs of
    radius 0.05-0.3 m and amplitude U(-3, 3), clipped to the range.  sigma: log-uniform in
    ``sig_range_mS`` mS/m, correlated with eps_r through a Gaussian copula,
    z_sigma = rho z_eps + sqrt(1 - rho^2) xi, xi an independent layered/blob field."""
    from scipy.special import ndtr

    rng = np.random.default_rng(seed)
    lo, hi = eps_range
    nl = int(rng.integers(3, 7))
    nb = int(rng.integers(5, 11))
    eps = _layer_blob_field(rng, nxp, nyp, dx, lo, hi, nl, nb, 3.0)
    xi = _layer_blob_field(rng, nxp, nyp, dx, 0.0, 1.0, int(rng.integers(3, 7)),
                           int(rng.integers(5, 11)), 0.3)
    z_eps = (eps - 0.5 * (lo + hi)) / ((hi - lo) / math.sqrt(12.0))
    z_xi = (xi - 0.5) / (1.0 / math.sqrt(12.0))
    z = rho * z_eps + math.sqrt(1.0 - rho * rho) * z_xi
    u = ndtr(z)
    slo, shi = math.log(sig_range_mS[0] * 1e-3), math.log(sig_range_mS[1] * 1e-3)
    sig = np.exp(slo + u * (shi - slo))
    return eps, sig


def smooth(a: np.ndarray, sigma_m: float, dx: float) -> np.ndarray:
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(a, sigma=sigma_m / dx, mode="nearest")


def surface_acquisition(nshots: int, nrec: int, nxp: int, dx: float, npml: int,
                        depth_cells: int = 2):
    """Shots at x = (s + 1/2) Lx / nshots and receivers at x = (r + 1/2) Lx / nrec, both
    ``depth_cells`` below the top of the physical domain."""
    Lx = nxp * dx
    j = npml + depth_cells
    src = np.array([[[cell_of((s + 0.5) * Lx / nshots, dx, npml), j]] for s in range(nshots)],
                   dtype=np.int32)
    rx = [cell_of((r + 0.5) * Lx / nrec, dx, npml) for r in range(nrec)]
    rec = np.array([[[i, j] for i in rx] for _ in range(nshots)], dtype=np.int32)
    return src, rec


# ------------------------------------------------------------------------------------------
# The workloads
# ------------------------------------------------------------------------------------------
def single_shot_disc() -> Workload:
    """100x100 cells (+10-cell CPML), dx 0.02 m, dt 40 ps, nt 600, one 200 MHz Ricker
    source at (1.0, 0.1) m, 20 receivers at depth 0.1 m spaced 0.08 m; background
    eps_r 4 / 1 mS/m with a disc of radius 0.3 m at (1.0, 1.0) m, eps_r 9 / 10 mS/m.
    Starting model: the background."""
    npml, nxp, dx, f0 = 10, 100, 0.02, 200e6
    g = default_pml(GridSpec(nx=nxp + 2 * npml, ny=nxp + 2 * npml, npml=npml, nt=600, dx=dx,
                             dy=dx, dt=40e-12), f0)
    ii = (np.arange(g.nx) - npml) * dx
    jj = (np.arange(g.ny) - npml) * dx
    X, Y = np.meshgrid(ii, jj)
    disc = (X - 1.0) ** 2 + (Y - 1.0) ** 2 <= 0.3 ** 2
    eps_bg = np.full((g.ny, g.nx), 4.0)
    sig_bg = np.full((g.ny, g.nx), 1e-3)
    eps_t = np.where(disc, 9.0, eps_bg)
    sig_t = np.where(disc, 10e-3, sig_bg)
    src = np.array([[[cell_of(1.0, dx, npml), cell_of(0.1, dx, npml)]]], dtype=np.int32)
    rec = np.array([[[cell_of(1.0 + (r - 9.5) * 0.08, dx, npml), cell_of(0.1, dx, npml)]
                     for r in range(20)]], dtype=np.int32)
    return Workload("single_shot_disc_120x120", g, f0, src, rec, eps_t, sig_t, eps_bg, sig_bg)


def multishot_layered(seed: int = 1000, nshots: int = 32, nt: int = 2000) -> Workload:
    """500x250 cells (+20-cell CPML), dx 0.01 m, dt 15 ps, nt 2000, 400 MHz Ricker,
    32 surface shots and 100 surface receivers; seeded layered + blob model with eps_r
    3-12 and sigma 0.1-20 mS/m (copula rho 0.6); start = true model smoothed (0.2 m)."""
    npml, nxp, nyp, dx, f0 = 20, 500, 250, 0.01, 400e6
    g = default_pml(GridSpec(nx=nxp + 2 * npml, ny=nyp + 2 * npml, npml=npml, nt=nt, dx=dx,
                             dy=dx, dt=15e-12), f0)
    eps, sig = layered_blob_model(seed, nxp, nyp, dx)
    eps_i, sig_i = smooth(eps, 0.2, dx), np.exp(smooth(np.log(sig), 0.2, dx))
    src, rec = surface_acquisition(nshots, 100, nxp, dx, npml)
    return Workload(f"multishot_layered_{g.nx}x{g.ny}_{nshots}shots_nt{nt}", g, f0, src, rec,
                    pad_edges(eps, npml), pad_edges(sig, npml), pad_edges(eps_i, npml),
                    pad_edges(sig_i, npml), seed=seed)


def uneven_instances(seed: int = 2000, count: int = 64):
    """64 independent instances: sizes uniform in [128, 768] x [128, 384] (multiples of 8),
    nt uniform in 800..3000, 1-8 shots, dx 0.01 m, 20-cell CPML, dt 15 ps, 400 MHz."""
    out = []
    for k in range(count):
        rng = np.random.default_rng(seed + k)
        nxp = int(rng.integers(16, 97)) * 8
        nyp = int(rng.integers(16, 49)) * 8
        nt = int(rng.integers(800, 3001))
        ns = int(rng.integers(1, 9))
        npml, dx, f0 = 20, 0.01, 400e6
        g = default_pml(GridSpec(nx=nxp + 2 * npml, ny=nyp + 2 * npml, npml=npml, nt=nt,
                                 dx=dx, dy=dx, dt=15e-12), f0)
        eps, sig = layered_blob_model(seed + k, nxp, nyp, dx)
        eps_i, sig_i = smooth(eps, 0.2, dx), np.exp(smooth(np.log(sig), 0.2, dx))
        nrec = max(8, nxp // 8)
        src, rec = surface_acquisition(ns, nrec, nxp, dx, npml)
        out.append(Workload(f"instance{k}_{g.nx}x{g.ny}_nt{nt}_{ns}shots", g, f0, src, rec,
                            pad_edges(eps, npml), pad_edges(sig, npml),
                            pad_edges(eps_i, npml), pad_edges(sig_i, npml), seed=seed + k))
    return out


def large_checkpointed(seed: int = 4000, nshots: int = 16, nt: int = 8000) -> Workload:
    """2048x1024 cells (+30-cell CPML), dx 0.005 m, dt 8 ps, nt 8000, 1 GHz Ricker,
    16 shots, 400 receivers; eps_r 2-25, sigma 0.1-50 mS/m."""
    npml, nxp, nyp, dx, f0 = 30, 2048, 1024, 0.005, 1e9
    g = default_pml(GridSpec(nx=nxp + 2 * npml, ny=nyp + 2 * npml, npml=npml, nt=nt, dx=dx,
                             dy=dx, dt=8e-12), f0)
    eps, sig = layered_blob_model(seed, nxp, nyp, dx, eps_range=(2.0, 25.0),
                                  sig_range_mS=(0.1, 50.0))
    eps_i, sig_i = smooth(eps, 0.2, dx), np.exp(smooth(np.log(sig), 0.2, dx))
    src, rec = surface_acquisition(nshots, 400, nxp, dx, npml)
    return Workload(f"large_{g.nx}x{g.ny}_{nshots}shots_nt{nt}", g, f0, src, rec,
                    pad_edges(eps, npml), pad_edges(sig, npml), pad_edges(eps_i, npml),
                    pad_edges(sig_i, npml), seed=seed)


def preconditioner_model(seed: int, nshots: int = 16, nt: int = 1500, nxp: int = 256,
                         nyp: int = 128, npml: int = 20, nrec: int = 64) -> Workload:
    """256x128 cells (+20-cell CPML), dx 0.01 m, dt 15 ps, nt 1500, 400 MHz, 16 shots, 64
    receivers (smaller grids for tests through nxp, nyp, npml, nrec)."""
    dx, f0 = 0.01, 400e6
    g = default_pml(GridSpec(nx=nxp + 2 * npml, ny=nyp + 2 * npml, npml=npml, nt=nt, dx=dx,
                             dy=dx, dt=15e-12), f0)
    eps, sig = layered_blob_model(seed, nxp, nyp, dx)
    eps_i, sig_i = smooth(eps, 0.2, dx), np.exp(smooth(np.log(sig), 0.2, dx))
    src, rec = surface_acquisition(nshots, nrec, nxp, dx, npml)
    return Workload(f"precond_{g.nx}x{g.ny}_{nshots}shots_nt{nt}", g, f0, src, rec,
                    pad_edges(eps, npml), pad_edges(sig, npml), pad_edges(eps_i, npml),
                    pad_edges(sig_i, npml), seed=seed)


def small_random(seed: int, nxp: int = 40, nyp: int = 30, npml: int = 6, nt: int = 160,
                 nshots: int = 2, nrec: int = 7, dx: float = 0.02, f0: float = 300e6,
                 kappa_max: float = 1.0, with_pec: bool = False) -> Workload:
    """Small heterogeneous lossy case for parity and pin tests (ragged sizes on purpose)."""
    dt = 0.9 * cfl_dt_max(dx, dx)
    g = default_pml(GridSpec(nx=nxp + 2 * npml, ny=nyp + 2 * npml, npml=npml, nt=nt, dx=dx,
                             dy=dx, dt=dt), f0)
    g = replace(g, pml_kappa_max=kappa_max)
    eps, sig = layered_blob_model(seed, nxp, nyp, dx, sig_range_mS=(1.0, 30.0))
    rng = np.random.default_rng(seed + 7)
    eps_t, sig_t = pad_edges(eps, npml), pad_edges(sig, npml)
    if with_pec:
        j0, i0 = npml + nyp // 2, npml + nxp // 2
        sig_t[j0:j0 + 2, i0:i0 + 3] = 1e3  # a small metal object (sigma > 100 S/m)
    src = np.zeros((nshots, 1, 2), dtype=np.int32)
    rec = np.zeros((nshots, nrec, 2), dtype=np.int32)
    for s in range(nshots):
        src[s, 0] = [npml + int(rng.integers(1, nxp - 1)), npml + int(rng.integers(1, 4))]
        rec[s, :, 0] = npml + rng.integers(0, nxp, size=nrec)
        rec[s, :, 1] = npml + rng.integers(0, nyp, size=nrec)
    eps_i = pad_edges(smooth(eps, 0.1, dx), npml)
    sig_i = pad_edges(np.exp(smooth(np.log(sig), 0.1, dx)), npml)
    return Workload(f"small_{g.nx}x{g.ny}_s{seed}", g, f0, src, rec, eps_t, sig_t, eps_i,
                    sig_i, seed=seed)
