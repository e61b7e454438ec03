"""FP64 numpy oracle for the FWI driver pieces: the TV term of Algorithm 3 and L-BFGS.

TEST INFRASTRUCTURE ONLY (see oracle.py).  Shares no code with the CUDA library or the
driver in the package.

TV (Algorithm 3, Sec. 3.4), read as split Bregman for min_u 1/2 |u - x|^2 + lam TV(u),
TV(u) = sum sqrt((Dx u)^2 + (Dy u)^2), circular differences, on x = X / max|X|, starting
from u = x, Z = D x, B = 0 (so that lam = 0 leaves x unchanged), then per iteration:
    u <- (x + mu D^T (Z - B) + mu * (sum of the 4 neighbours of u)) / (1 + 4 mu)   (Jacobi)
    Z <- shrink(D u + B, lam / mu)                                                 (isotropic)
    B <- B + D u - Z
then the TV gradient weight * max|G| * (x - u) (normalised units) is added to G.

L-BFGS (Nocedal & Wright, Algorithm 7.4): the two-loop recursion for d = -H g with the
initial scaling gamma = s'y / y'y of the newest pair.
"""
from __future__ import annotations

import numpy as np


def dx_fwd(u):
    return np.roll(u, -1, axis=1) - u


def dy_fwd(u):
    return np.roll(u, -1, axis=0) - u


def dxt(v):
    """Transpose of dx_fwd: v(i-1) - v(i)."""
    return np.roll(v, 1, axis=1) - v


def dyt(v):
    return np.roll(v, 1, axis=0) - v


def tv_value(u):
    return float(np.sum(np.sqrt(dx_fwd(u) ** 2 + dy_fwd(u) ** 2)))


def tv_denoise_split_bregman(x, lam, mu, iters):
    """Approximate minimiser of 1/2 |u - x|^2 + lam TV(u) (the steps listed above)."""
    x = np.asarray(x, dtype=np.float64)
    u = x.copy()
    zx = dx_fwd(x)
    zy = dy_fwd(x)
    bx = np.zeros_like(x)
    by = np.zeros_like(x)
    for _ in range(iters):
        rhs = x + mu * (dxt(zx - bx) + dyt(zy - by))
        nb = np.roll(u, 1, 1) + np.roll(u, -1, 1) + np.roll(u, 1, 0) + np.roll(u, -1, 0)
        u = (rhs + mu * nb) / (1.0 + 4.0 * mu)
        sx = dx_fwd(u) + bx
        sy = dy_fwd(u) + by
        mag = np.sqrt(sx * sx + sy * sy)
        f = np.where(mag > lam / mu, (mag - lam / mu) / np.where(mag > 0, mag, 1.0), 0.0)
        zx, zy = f * sx, f * sy
        bx, by = sx - zx, sy - zy
    return u


def tv_gradient(X, G, lam, mu, iters, weight):
    """G + weight * max|G| * (x - u): x = X / max|X|, u its TV-denoised version."""
    X = np.asarray(X, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    s = np.abs(X).max()
    x = X / s if s > 0 else np.zeros_like(X)
    u = tv_denoise_split_bregman(x, lam, mu, iters)
    return G + weight * np.abs(G).max() * (x - u)


def lbfgs_direction(g, s_list, y_list):
    """d = -H g by the two-loop recursion over the stored pairs (oldest first)."""
    q = np.array(g, dtype=np.float64)
    alphas = []
    for s, y in zip(reversed(s_list), reversed(y_list)):
        rho = 1.0 / np.dot(y, s)
        a = rho * np.dot(s, q)
        q = q - a * y
        alphas.append((rho, a))
    if s_list:
        s, y = s_list[-1], y_list[-1]
        q = q * (np.dot(s, y) / np.dot(y, y))
    for (s, y), (rho, a) in zip(zip(s_list, y_list), reversed(alphas)):
        b = rho * np.dot(y, q)
        q = q + s * (a - b)
    return -q
