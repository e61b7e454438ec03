"""Why the adjoint does not rebuild the forward wavefield by running the forward step
backwards (boundary-strip reconstruction) and uses checkpoints instead.

The E update of Algorithm 1 is Ez^{n+1} = Ca Ez^n + Cb Q^n with Ca = (1 - a) / (1 + a),
a = sigma dt / (2 eps) (Sec. 3.2 coefficient listing).  Undoing it gives
Ez^n = (Ez^{n+1} - Cb Q^n) / Ca, and with the H updates undone as well the reversed scheme is
exact in exact arithmetic.  In a lossy medium, though, the reversal turns the wave's damping
into growth: a perturbation of the final state (rounding, in practice) grows like e^{a n}
over n reversed steps, the inverse of the amplitude decay e^{-a n} of the forward lossy wave.
For the configurations' conductivities that is about e^11 (540x290 workload, 20 mS/m at
eps_r 3, nt 2000) and e^90 (2048x1024 workload, 50 mS/m at eps_r 2, nt 8000): FP32 rounding
would swamp the reconstructed field.  In a lossless medium the reversal stays bounded.

The reversed step here is written from Algorithm 1's update order for a PEC box without a
CPML (the CPML memories would need 1/b with b < 1 as well); the forward history comes from the
oracle.
"""
import numpy as np
import pytest

from oracle import oracle as O

EPS0 = 8.8541878128e-12
MU0 = 1.25663706212e-6


def box(nx, ny, nt, eps_r, sigma, dx=0.01):
    dt = 0.9 * dx / (299792458.0 * np.sqrt(2.0))
    g = O.Grid(nx=nx, ny=ny, npml=0, nt=nt, dx=dx, dy=dx, dt=dt)
    e = np.full((ny, nx), float(eps_r))
    s = np.full((ny, nx), float(sigma))
    return g, e, s


def coefficients(g, e, s):
    eps = EPS0 * e
    a = s * g.dt / (2.0 * eps)
    ca = (1.0 - a) / (1.0 + a)
    cb = (g.dt / eps) / (1.0 + a)
    return ca, cb


def h_from_history(g, ez_hist):
    """H^{nt - 1/2} from the Ez history: H starts at zero and each step adds the curl term."""
    ch = g.dt / MU0
    hx = np.zeros(ez_hist.shape[1:])
    hy = np.zeros(ez_hist.shape[1:])
    for ez in ez_hist[:-1]:                      # Ez^0 .. Ez^{nt-1}
        hx[:-1, :] -= ch * (ez[1:, :] - ez[:-1, :]) / g.dy
        hy[:, :-1] += ch * (ez[:, 1:] - ez[:, :-1]) / g.dx
    return hx, hy


def reverse_step(g, ez, hx, hy, ca, cb, src, w):
    """(Ez^{n+1}, H^{n+1/2}) -> (Ez^n, H^{n-1/2}) for step n of Algorithm 1 (PEC box)."""
    ch = g.dt / MU0
    q = np.zeros_like(ez)
    q[1:-1, 1:-1] = (hy[1:-1, 1:-1] - hy[1:-1, :-2]) / g.dx - (hx[1:-1, 1:-1] - hx[:-2, 1:-1]) / g.dy
    for (i, j), wn in zip(src, w):
        q[j, i] -= wn / (g.dx * g.dy)
    ez0 = np.zeros_like(ez)                      # the PEC ring stays zero
    ez0[1:-1, 1:-1] = (ez[1:-1, 1:-1] - cb[1:-1, 1:-1] * q[1:-1, 1:-1]) / ca[1:-1, 1:-1]
    hx0 = hx.copy()
    hy0 = hy.copy()
    hx0[:-1, :] += ch * (ez0[1:, :] - ez0[:-1, :]) / g.dy
    hy0[:, :-1] -= ch * (ez0[:, 1:] - ez0[:, :-1]) / g.dx
    return ez0, hx0, hy0


def run_reverse(g, e, s, src, wav, ez_end, hx, hy, steps):
    ca, cb = coefficients(g, e, s)
    ez, out = ez_end, [ez_end]
    for n in range(g.nt - 1, g.nt - 1 - steps, -1):
        ez, hx, hy = reverse_step(g, ez, hx, hy, ca, cb, src, wav[:, n])
        out.append(ez)
    return out                                   # Ez^{nt}, Ez^{nt-1}, ...


@pytest.fixture(scope="module")
def lossless():
    g, e, s = box(48, 40, 300, 4.0, 0.0)
    src = np.array([[20, 17]])
    wav = O.ricker(1.5e9, g.dt, g.nt)[None, :]
    hist = O.forward_shot(g, e, s, src, wav, np.array([[30, 25]]), history=True)["ez_hist"]
    return g, e, s, src, wav, hist


def test_reversed_scheme_reproduces_the_history_without_loss(lossless):
    """Exact start state: the reversed steps give back the oracle's Ez history (FP64)."""
    g, e, s, src, wav, hist = lossless
    hx, hy = h_from_history(g, hist)
    rec = run_reverse(g, e, s, src, wav, hist[-1], hx, hy, g.nt)
    ref = np.linalg.norm(hist, axis=(1, 2)).max()
    err = max(np.abs(rec[k] - hist[g.nt - k]).max() for k in range(len(rec)))
    assert err <= 1e-9 * ref


def test_perturbation_stays_bounded_without_loss(lossless):
    g, e, s, src, wav, hist = lossless
    hx, hy = h_from_history(g, hist)
    rng = np.random.default_rng(5)
    d = 1e-6 * np.abs(hist[-1]).max() * rng.standard_normal(hist[-1].shape)
    d[[0, -1], :] = 0.0
    d[:, [0, -1]] = 0.0
    a = run_reverse(g, e, s, src, wav, hist[-1], hx, hy, g.nt)
    b = run_reverse(g, e, s, src, wav, hist[-1] + d, hx, hy, g.nt)
    growth = [np.linalg.norm(y - x) / np.linalg.norm(d) for x, y in zip(a, b)]
    assert max(growth) < 3.0


@pytest.mark.parametrize("sigma", [0.02, 0.04])
def test_perturbation_grows_like_the_inverse_damping_with_loss(sigma):
    """The growth over k reversed steps matches ((1 + a) / (1 - a))^{k/2} ~ e^{a k},
    a = sigma dt / (2 eps) (each oscillating mode of the lossy step has |lambda|^2 = Ca, the
    determinant of the one-step map), within 25%, far above the lossless bound; e^{2 a k}
    would be off by the same factor again."""
    g, e, s = box(48, 40, 600, 3.0, sigma)
    src = np.array([[20, 17]])
    wav = O.ricker(1.5e9, g.dt, g.nt)[None, :]
    hist = O.forward_shot(g, e, s, src, wav, np.array([[30, 25]]), history=True)["ez_hist"]
    hx, hy = h_from_history(g, hist)
    rng = np.random.default_rng(6)
    d = 1e-6 * np.abs(hist[-1]).max() * rng.standard_normal(hist[-1].shape)
    d[[0, -1], :] = 0.0
    d[:, [0, -1]] = 0.0
    a = run_reverse(g, e, s, src, wav, hist[-1], hx, hy, g.nt)
    b = run_reverse(g, e, s, src, wav, hist[-1] + d, hx, hy, g.nt)
    # |dEz| alone oscillates as energy moves between E and H: compare its envelope (the
    # largest value in a window of 40 steps) near the end state and near the start
    norms = np.array([np.linalg.norm(y - x) for x, y in zip(a, b)])
    k0 = int(np.argmax(norms[:40]))
    k1 = len(norms) - 40 + int(np.argmax(norms[-40:]))
    measured = norms[k1] / norms[k0]
    a_coef = sigma * g.dt / (2.0 * EPS0 * 3.0)
    predicted = ((1.0 + a_coef) / (1.0 - a_coef)) ** ((k1 - k0) / 2.0)
    assert predicted > 50.0
    assert predicted / 1.25 <= measured <= predicted * 1.25
