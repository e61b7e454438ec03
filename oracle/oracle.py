"""FP64 CPU oracle for the 2-D TM FDTD forward model and its exact discrete adjoint.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of
``bench.py`` may import this module.  It shares no code with the CUDA library; the heavy
loops live in ``fdtd_oracle.c`` (plain C, double precision), and this file adds the pieces
that are easier to state with numpy/scipy:

* :func:`ricker` -- the Ricker source wavelet (the paper's ``source_amplitudes =
  ['ricker', amplitude, f0]``, Sec. 4 tables; formula per the reading listed in the design
  notes: w(t) = A (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2), t0 = sqrt(2)/f0).
* :func:`line_source_trace` -- the analytic 2-D homogeneous-medium line-source solution
  (Hankel-function Green's function convolved with the source current), used to pin the
  oracle against the continuous Maxwell equations (Eqs. faraday, ampere).
* :func:`forward`, :func:`misfit_and_gradient`, :func:`tangent`, :func:`forward_shot`,
  :func:`adjoint_shot` -- ctypes wrappers of the C routines.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

EPS0 = 8.8541878128e-12  # F/m
MU0 = 1.25663706212e-6  # H/m
C0 = 1.0 / np.sqrt(EPS0 * MU0)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fdtd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
# A test may point the wrapper at a deliberately broken build of this same source (the
# mutation test plants mistakes in a copy of fdtd_oracle.c to show the pins catch them).
_OVERRIDE = os.environ.get("GPRFWI_ORACLE_LIB")
_lock = threading.Lock()
_lib = None


def build(force: bool = False, src: str = _SRC, out: str | None = None) -> str:
    """Compile ``fdtd_oracle.c`` with gcc into ``oracle/_build/liboracle.so``."""
    if _OVERRIDE and out is None:
        return _OVERRIDE
    if out is not None:
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", "-o", tmp, src,
                        "-lm"], check=True)
        os.replace(tmp, out)
        return out
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrGrid(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("npml", ctypes.c_int32),
        ("nt", ctypes.c_int32), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
        ("dt", ctypes.c_double), ("pml_order", ctypes.c_int32),
        ("pml_sigma_max", ctypes.c_double), ("pml_kappa_max", ctypes.c_double),
        ("pml_alpha_max", ctypes.c_double), ("pml_eps_ref", ctypes.c_double),
    ]


@dataclass
class Grid:
    """Padded grid: arrays are [ny][nx] with the CPML (width npml) inside them."""
    nx: int
    ny: int
    npml: int
    nt: int
    dx: float
    dy: float
    dt: float
    pml_order: int = 3
    pml_sigma_max: float = 0.0
    pml_kappa_max: float = 1.0
    pml_alpha_max: float = 0.0
    pml_eps_ref: float = 1.0

    def c_struct(self) -> OrGrid:
        return OrGrid(self.nx, self.ny, self.npml, self.nt, self.dx, self.dy, self.dt,
                      self.pml_order, self.pml_sigma_max, self.pml_kappa_max,
                      self.pml_alpha_max, self.pml_eps_ref)


def as_grid(g) -> Grid:
    """Accept any object with the Grid attributes (e.g. a workload descriptor)."""
    if isinstance(g, Grid):
        return g
    return Grid(**{k: getattr(g, k) for k in Grid.__dataclass_fields__})


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            d, i32 = ctypes.c_double, ctypes.c_int32
            pd, pi = P(d), P(i32)
            g = P(OrGrid)
            lib.or_forward_shot.argtypes = [g, pd, pd, ctypes.c_int, pi, pd, ctypes.c_int, pi,
                                            pd, pd, pd, pd, pd]
            lib.or_adjoint_shot.argtypes = [g, pd, pd, ctypes.c_int, pi, ctypes.c_int, pi,
                                            pd, pd, pd, pd, pd, pd, pd, pd]
            lib.or_tangent_shot.argtypes = [g, pd, pd, pd, pd, ctypes.c_int, pi, pd,
                                            ctypes.c_int, pi, pd]
            lib.or_forward.argtypes = [g, pd, pd, ctypes.c_int, ctypes.c_int, pi, pd,
                                       ctypes.c_int, pi, pd, ctypes.c_int]
            lib.or_misfit_gradient.argtypes = [g, pd, pd, ctypes.c_int, ctypes.c_int, pi, pd,
                                               ctypes.c_int, pi, pd, pd, pd, pd, pd,
                                               ctypes.c_int]
            lib.or_forward_te_shot.argtypes = [g, pd, pd, ctypes.c_int, ctypes.c_int, pi, pd,
                                               ctypes.c_int, pi, pd, pd, pd, pd]
            lib.or_adjoint_te_shot.argtypes = [g, pd, pd, ctypes.c_int, ctypes.c_int, pi, pd,
                                               pd, pd, pd, pd]
            for f in (lib.or_forward_shot, lib.or_adjoint_shot, lib.or_tangent_shot,
                      lib.or_forward, lib.or_misfit_gradient, lib.or_forward_te_shot,
                      lib.or_adjoint_te_shot):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _pd(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _pi(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None and a.shape != tuple(shape):
        a = a.reshape(shape)
    return a


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _check(rc, name):
    if rc != 0:
        raise RuntimeError(f"oracle {name} failed (out of memory?)")


# ------------------------------------------------------------------------------------------
# Source wavelet
# ------------------------------------------------------------------------------------------
def ricker(f0: float, dt: float, nt: int, amp: float = 1.0, t0: float | None = None) -> np.ndarray:
    """Ricker wavelet sampled at t = n dt, n = 0..nt-1 (FP64)."""
    if t0 is None:
        t0 = np.sqrt(2.0) / f0
    t = np.arange(nt, dtype=np.float64) * dt - t0
    z = (np.pi * f0 * t) ** 2
    return amp * (1.0 - 2.0 * z) * np.exp(-z)


# ------------------------------------------------------------------------------------------
# Single-shot routines
# ------------------------------------------------------------------------------------------
def forward_shot(grid, eps_r, sigma, src, wav, rec, history=False, qhistory=False,
                 energy=False, fields=False):
    """One shot.  src [nsrc,2], wav [nsrc,nt], rec [nrec,2] (cell indices i, j).

    Returns a dict with ``traces`` [nt, nrec] and optionally ``ez_hist`` [nt+1, ny, nx],
    ``q_hist`` [nt, ny, nx], ``energy`` [nt], ``h_traces`` [nt, nrec, 2] (Hx^{n-1/2},
    Hy^{n-1/2} at the receiver cells' staggered nodes, sampled with Ez^n)."""
    g = as_grid(grid)
    lib = _load()
    shape = (g.ny, g.nx)
    e, s = _f64(eps_r, shape), _f64(sigma, shape)
    src, rec = _i32(src).reshape(-1, 2), _i32(rec).reshape(-1, 2)
    wav = _f64(wav).reshape(len(src), g.nt)
    out = {"traces": np.zeros((g.nt, len(rec)))}
    if history:
        out["ez_hist"] = np.zeros((g.nt + 1,) + shape)
    if qhistory:
        out["q_hist"] = np.zeros((g.nt,) + shape)
    if energy:
        out["energy"] = np.zeros(g.nt)
    if fields:
        out["h_traces"] = np.zeros((g.nt, len(rec), 2))
    rc = lib.or_forward_shot(ctypes.byref(g.c_struct()), _pd(e), _pd(s), len(src), _pi(src),
                             _pd(wav), len(rec), _pi(rec), _pd(out["traces"]),
                             _pd(out.get("h_traces")), _pd(out.get("ez_hist")),
                             _pd(out.get("q_hist")), _pd(out.get("energy")))
    _check(rc, "forward_shot")
    return out


def forward_te_shot(grid, eps_r, sigma, polarisation, src, wav, rec, energy=False,
                    history=False):
    """One shot of the TE mode (``polarisation`` 0: x-directed source current on Ex,
    1: y-directed on Ey).  Returns ``traces`` [nt, nrec, 3] (Ex^n, Ey^n, Hz^{n-1/2} at the
    receiver cells' nodes) and optionally ``energy`` [nt] and ``ex_hist``, ``ey_hist``
    [nt+1, ny, nx]."""
    g = as_grid(grid)
    lib = _load()
    shape = (g.ny, g.nx)
    e, s = _f64(eps_r, shape), _f64(sigma, shape)
    src, rec = _i32(src).reshape(-1, 2), _i32(rec).reshape(-1, 2)
    wav = _f64(wav).reshape(len(src), g.nt)
    out = {"traces": np.zeros((g.nt, len(rec), 3))}
    if energy:
        out["energy"] = np.zeros(g.nt)
    if history:
        out["ex_hist"] = np.zeros((g.nt + 1,) + shape)
        out["ey_hist"] = np.zeros((g.nt + 1,) + shape)
    rc = lib.or_forward_te_shot(ctypes.byref(g.c_struct()), _pd(e), _pd(s), int(polarisation),
                                len(src), _pi(src), _pd(wav), len(rec), _pi(rec),
                                _pd(out["traces"]), _pd(out.get("energy")),
                                _pd(out.get("ex_hist")), _pd(out.get("ey_hist")))
    if rc == -2:
        raise ValueError("polarisation must be 0 (x) or 1 (y)")
    _check(rc, "forward_te_shot")
    return out


def adjoint_te_shot(grid, eps_r, sigma, polarisation, rec, resid, ex_hist, ey_hist):
    """Exact adjoint of :func:`forward_te_shot` for the residual of the source's own
    component, resid [nt, nrec]; returns (dJ/deps_r, dJ/dsigma) [ny, nx]."""
    g = as_grid(grid)
    lib = _load()
    shape = (g.ny, g.nx)
    e, s = _f64(eps_r, shape), _f64(sigma, shape)
    rec = _i32(rec).reshape(-1, 2)
    r = _f64(resid).reshape(g.nt, len(rec))
    xh = _f64(ex_hist).reshape((g.nt + 1,) + shape)
    yh = _f64(ey_hist).reshape((g.nt + 1,) + shape)
    ge, gs = np.zeros(shape), np.zeros(shape)
    rc = lib.or_adjoint_te_shot(ctypes.byref(g.c_struct()), _pd(e), _pd(s), int(polarisation),
                                len(rec), _pi(rec), _pd(r), _pd(xh), _pd(yh), _pd(ge), _pd(gs))
    if rc == -2:
        raise ValueError("polarisation must be 0 (x) or 1 (y)")
    _check(rc, "adjoint_te_shot")
    return ge, gs


def misfit_and_gradient_te(grid, eps_r, sigma, polarisation, src, wav, rec, observed):
    """J = 1/2 sum (d - o)^2 over the source component's traces of every shot, and its
    gradients summed over shots (in shot order).  src [nshots,nsrc,2], wav [nshots,nsrc,nt],
    rec [nshots,nrec,2], observed [nshots,nt,nrec]."""
    src = np.asarray(src)
    J = 0.0
    ge = gs = None
    for k in range(len(src)):
        out = forward_te_shot(grid, eps_r, sigma, polarisation, src[k], wav[k], rec[k],
                              history=True)
        r = out["traces"][:, :, polarisation] - np.asarray(observed[k], dtype=np.float64)
        J += 0.5 * float(np.sum(r * r))
        a, b = adjoint_te_shot(grid, eps_r, sigma, polarisation, rec[k], r, out["ex_hist"],
                               out["ey_hist"])
        ge = a if ge is None else ge + a
        gs = b if gs is None else gs + b
    return J, ge, gs


def adjoint_shot(grid, eps_r, sigma, src, rec, resid, ez_hist, q_hist=None):
    """Exact discrete adjoint of :func:`forward_shot` driven by ``resid`` [nt, nrec].

    Returns a dict: ``g_eps_r``, ``g_sigma`` (zero-lag form), ``gc_eps_r``, ``gc_sigma``
    (coefficient form, only if ``q_hist`` is given) and ``g_wav`` [nsrc, nt]."""
    g = as_grid(grid)
    lib = _load()
    shape = (g.ny, g.nx)
    e, s = _f64(eps_r, shape), _f64(sigma, shape)
    src, rec = _i32(src).reshape(-1, 2), _i32(rec).reshape(-1, 2)
    resid = _f64(resid).reshape(g.nt, len(rec))
    ez_hist = _f64(ez_hist)
    qh = _f64(q_hist) if q_hist is not None else None
    out = {"g_eps_r": np.zeros(shape), "g_sigma": np.zeros(shape),
           "g_wav": np.zeros((len(src), g.nt))}
    if qh is not None:
        out["gc_eps_r"] = np.zeros(shape)
        out["gc_sigma"] = np.zeros(shape)
    rc = lib.or_adjoint_shot(ctypes.byref(g.c_struct()), _pd(e), _pd(s), len(src), _pi(src),
                             len(rec), _pi(rec), _pd(resid), _pd(ez_hist), _pd(qh),
                             _pd(out["g_eps_r"]), _pd(out["g_sigma"]),
                             _pd(out.get("gc_eps_r")), _pd(out.get("gc_sigma")),
                             _pd(out["g_wav"]))
    _check(rc, "adjoint_shot")
    return out


def tangent(grid, eps_r, sigma, d_eps_r, d_sigma, src, wav, rec):
    """Tangent-linear traces [nt, nrec] of one shot along (d_eps_r, d_sigma)."""
    g = as_grid(grid)
    lib = _load()
    shape = (g.ny, g.nx)
    args = [_f64(a, shape) for a in (eps_r, sigma, d_eps_r, d_sigma)]
    src, rec = _i32(src).reshape(-1, 2), _i32(rec).reshape(-1, 2)
    wav = _f64(wav).reshape(len(src), g.nt)
    out = np.zeros((g.nt, len(rec)))
    rc = lib.or_tangent_shot(ctypes.byref(g.c_struct()), *[_pd(a) for a in args], len(src),
                             _pi(src), _pd(wav), len(rec), _pi(rec), _pd(out))
    _check(rc, "tangent")
    return out


# ------------------------------------------------------------------------------------------
# Multi-shot routines.  src [nshots,nsrc,2], wav [nshots,nsrc,nt], rec [nshots,nrec,2].
# ------------------------------------------------------------------------------------------
def forward(grid, eps_r, sigma, src, wav, rec, nthreads: int = 1) -> np.ndarray:
    """Traces [nshots, nt, nrec] of all shots."""
    g = as_grid(grid)
    lib = _load()
    shape = (g.ny, g.nx)
    e, s = _f64(eps_r, shape), _f64(sigma, shape)
    src, rec = _i32(src), _i32(rec)
    ns, nsrc, nrec = src.shape[0], src.shape[1], rec.shape[1]
    wav = _f64(wav).reshape(ns, nsrc, g.nt)
    out = np.zeros((ns, g.nt, nrec))
    rc = lib.or_forward(ctypes.byref(g.c_struct()), _pd(e), _pd(s), ns, nsrc, _pi(src),
                        _pd(wav), nrec, _pi(rec), _pd(out), int(nthreads))
    _check(rc, "forward")
    return out


def misfit_and_gradient(grid, eps_r, sigma, src, wav, rec, observed, nthreads: int = 1,
                        return_traces: bool = False):
    """J = 1/2 sum (d - o)^2 and its exact gradients (dJ/deps_r, dJ/dsigma) summed over
    shots.  Returns (J, g_eps_r, g_sigma[, traces])."""
    g = as_grid(grid)
    lib = _load()
    shape = (g.ny, g.nx)
    e, s = _f64(eps_r, shape), _f64(sigma, shape)
    src, rec = _i32(src), _i32(rec)
    ns, nsrc, nrec = src.shape[0], src.shape[1], rec.shape[1]
    wav = _f64(wav).reshape(ns, nsrc, g.nt)
    obs = _f64(observed).reshape(ns, g.nt, nrec)
    J = np.zeros(1)
    ge, gs = np.zeros(shape), np.zeros(shape)
    tr = np.zeros((ns, g.nt, nrec)) if return_traces else None
    rc = lib.or_misfit_gradient(ctypes.byref(g.c_struct()), _pd(e), _pd(s), ns, nsrc,
                                _pi(src), _pd(wav), nrec, _pi(rec), _pd(obs), _pd(J),
                                _pd(ge), _pd(gs), _pd(tr), int(nthreads))
    _check(rc, "misfit_gradient")
    if return_traces:
        return float(J[0]), ge, gs, tr
    return float(J[0]), ge, gs


# ------------------------------------------------------------------------------------------
# Analytic 2-D line-source solution (pin for the continuous equations)
# ------------------------------------------------------------------------------------------
def line_source_hy_trace(current: np.ndarray, dt: float, x: float, eps_r: float,
                         sigma: float, pad: int = 8) -> np.ndarray:
    """Hy(x, 0, t_n), t_n = n dt, of the same line current at a point on the +x axis.

    Faraday's law with the e^{+j w t} convention, j w mu0 H = -curl E, gives for E = Ez z:
    Hy = (1 / (j w mu0)) dEz/dx; with Ez = -(w mu0 / 4) I H0^(2)(k rho) and
    dH0^(2)(z)/dz = -H1^(2)(z) this is Hy = -(j k / 4) I(w) H1^(2)(k x) on the axis."""
    from scipy.special import hankel2

    n = len(current)
    nfft = int(2 ** np.ceil(np.log2(n * pad)))
    I = np.fft.rfft(current, nfft)
    w = 2.0 * np.pi * np.fft.rfftfreq(nfft, dt)
    H = np.zeros_like(I)
    wk = w[1:]
    eps = EPS0 * eps_r
    k = np.sqrt(wk * wk * MU0 * eps - 1j * wk * MU0 * sigma)
    k = np.where(k.imag > 0, -k, k)
    H[1:] = -(1j * k / 4.0) * I[1:] * hankel2(1, k * x)
    return np.fft.irfft(H, nfft)[:n]


def line_source_trace(current: np.ndarray, dt: float, rho: float, eps_r: float,
                      sigma: float, pad: int = 8) -> np.ndarray:
    """Ez(rho, t_n), t_n = n dt, radiated by an infinite line current I(t_n) = current[n]
    (amperes) in a homogeneous medium (eps_r, sigma, mu0).

    With the e^{+j w t} convention the field obeys (lap + k^2) Ez = j w mu0 I delta, with
    k^2 = w^2 mu0 eps - j w mu0 sigma, whose outgoing solution is
    Ez = -(w mu0 / 4) I(w) H0^(2)(k rho)  (2-D Green's function -(j/4) H0^(2)(k rho)).
    The time series is obtained by an FFT of the zero-padded current."""
    from scipy.special import hankel2

    n = len(current)
    nfft = int(2 ** np.ceil(np.log2(n * pad)))
    I = np.fft.rfft(current, nfft)  # sum_n i(t_n) e^{-j w t_n}: e^{+jwt} convention
    w = 2.0 * np.pi * np.fft.rfftfreq(nfft, dt)
    E = np.zeros_like(I)
    wk = w[1:]
    eps = EPS0 * eps_r
    k = np.sqrt(wk * wk * MU0 * eps - 1j * wk * MU0 * sigma)
    k = np.where(k.imag > 0, -k, k)  # decaying branch: Im k <= 0 for e^{-j k rho}
    E[1:] = -(wk * MU0 / 4.0) * I[1:] * hankel2(0, k * rho)
    return np.fft.irfft(E, nfft)[:n]


def dipole_line_source_trace(current: np.ndarray, dt: float, rho: float, eps_r: float,
                             sigma: float, along: bool, pad: int = 8) -> np.ndarray:
    """E component parallel to an infinite x-directed line current I(t_n) = current[n]
    (the TE mode's source), at distance rho on the line through the source perpendicular to
    the current (``along`` False) or along it (``along`` True), homogeneous medium.

    With the e^{+j w t} convention the vector potential A = x mu0 I G, G = -(j/4)
    H0^(2)(k rho), gives E = -j w (A + grad div A / k^2), so
    Ex = -j w mu0 I (G + d^2 G / dx^2 / k^2).  Off the current's line (x = 0) the second
    derivative is G'(rho) / rho, and with dH0^(2)/dz = -H1^(2):
        Ex = -(w mu0 / 4) I [H0^(2)(k rho) - H1^(2)(k rho) / (k rho)];
    along it the second derivative is G''(rho), and with H0'' = -H0 + H1 / z:
        Ex = -(w mu0 / 4) I H1^(2)(k rho) / (k rho)."""
    from scipy.special import hankel2

    n = len(current)
    nfft = int(2 ** np.ceil(np.log2(n * pad)))
    I = np.fft.rfft(current, nfft)
    w = 2.0 * np.pi * np.fft.rfftfreq(nfft, dt)
    E = np.zeros_like(I)
    wk = w[1:]
    eps = EPS0 * eps_r
    k = np.sqrt(wk * wk * MU0 * eps - 1j * wk * MU0 * sigma)
    k = np.where(k.imag > 0, -k, k)
    z = k * rho
    shape = hankel2(1, z) / z if along else hankel2(0, z) - hankel2(1, z) / z
    E[1:] = -(wk * MU0 / 4.0) * I[1:] * shape
    return np.fft.irfft(E, nfft)[:n]
