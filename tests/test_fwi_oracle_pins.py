"""Pins of the FWI-driver oracle (TV term of Algorithm 3, L-BFGS) against independent
mathematics: the ROF minimiser by Chambolle's dual projection algorithm, and the dense
BFGS inverse-Hessian recursion."""
import numpy as np
import pytest

from oracle import fwi_oracle as F


def test_two_loop_equals_dense_bfgs():
    """The two-loop recursion applies the BFGS inverse Hessian built from the same pairs
    (H0 = gamma I with gamma from the newest pair)."""
    rng = np.random.default_rng(0)
    n, m = 12, 5
    A = rng.standard_normal((n, n))
    A = A @ A.T + n * np.eye(n)  # SPD: s'y > 0 for y = A s
    S = [rng.standard_normal(n) for _ in range(m)]
    Y = [A @ s for s in S]
    g = rng.standard_normal(n)
    gamma = S[-1] @ Y[-1] / (Y[-1] @ Y[-1])
    H = gamma * np.eye(n)
    for s, y in zip(S, Y):
        rho = 1.0 / (y @ s)
        V = np.eye(n) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    np.testing.assert_allclose(F.lbfgs_direction(g, S, Y), -H @ g, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(F.lbfgs_direction(g, [], []), -g)


def _chambolle_rof(f, lam, iters=20000, tau=0.124):
    """Chambolle (2004) dual projection for min_u 1/2 |u - f|^2 + lam TV(u) (isotropic,
    circular differences): u = f - lam * div p, div = -D^T."""
    px = np.zeros_like(f)
    py = np.zeros_like(f)
    for _ in range(iters):
        div = -(F.dxt(px) + F.dyt(py))
        w = div - f / lam
        gx, gy = F.dx_fwd(w), F.dy_fwd(w)
        nrm = np.sqrt(gx * gx + gy * gy)
        px = (px + tau * gx) / (1.0 + tau * nrm)
        py = (py + tau * gy) / (1.0 + tau * nrm)
    return f + lam * (F.dxt(px) + F.dyt(py))


def test_split_bregman_reaches_the_rof_minimiser():
    rng = np.random.default_rng(1)
    clean = np.zeros((12, 16))
    clean[3:9, 4:11] = 1.0
    f = clean + 0.2 * rng.standard_normal(clean.shape)
    lam = 0.15
    # one neighbour average per iteration (Algorithm 3) is stable for small mu
    u_sb = F.tv_denoise_split_bregman(f, lam, mu=0.2, iters=4000)
    u_ch = _chambolle_rof(f, lam)
    assert np.abs(u_sb - u_ch).max() < 2e-3
    # a real denoiser: closer to the clean image, smaller TV
    assert np.linalg.norm(u_sb - clean) < np.linalg.norm(f - clean)
    assert F.tv_value(u_sb) < F.tv_value(f)


def test_tv_gradient_without_regularisation_is_zero():
    rng = np.random.default_rng(2)
    X = 3 + rng.random((10, 14))
    G = rng.standard_normal((10, 14))
    np.testing.assert_allclose(F.tv_gradient(X, G, lam=0.0, mu=0.2, iters=30, weight=0.5), G,
                               rtol=0, atol=1e-12 * np.abs(G).max())


def test_tv_gradient_points_towards_smoother_model():
    """Adding the TV term moves a descent step towards a model with smaller TV."""
    rng = np.random.default_rng(3)
    X = 4 + (np.arange(16)[None, :] > 7) * 2.0 + 0.3 * rng.standard_normal((12, 16))
    G = np.zeros_like(X)
    G[0, 0] = 1.0  # sets the scale only
    out = F.tv_gradient(X, G, lam=0.05, mu=0.2, iters=200, weight=1.0)
    step = -(out - G)
    step *= 0.5 * np.abs(X - F.tv_denoise_split_bregman(X / np.abs(X).max(), 0.05, 0.2, 200)
                         * np.abs(X).max()).max() / np.abs(step).max()
    assert F.tv_value(X + step) < F.tv_value(X)
