"""Learned gradient preconditioner: a U-Net that turns the raw FWI gradient into a model
update, its training data, training loop, and the misfit-guarded step used by the FWI
driver.

The paper motivates learned methods as a way to cut the number of expensive Maxwell
solutions (Sec. 1) but trains none; this module is the library's own design:

* input (4 channels, physical cells only, channels last): g_eps_r / max|g_eps_r|,
  g_sigma / max|g_sigma|, eps_r / 10, and log10 of the illumination (sum over shots and
  steps of Ez^2, normalised by its maximum and floored at 1e-6) / 6 + 1;
* output (2 channels): (eps_true - eps_r) / eps_scale and (sigma_true - sigma) / sig_scale;
* training pairs: seeded random models (the preconditioner workload generator); each pair is
  taken at a model m = m0 + a (m_true - m0) between the smoothed starting model m0 and the
  truth (a = 0 for half of the pairs, else uniform in [0, 0.8), drawn from the seed), so the
  network also sees the gradients of later FWI iterates: the gradient of the L2 misfit at m
  and the illumination of m, computed by the FDTD/adjoint kernels, against the remaining
  update (1 - a)(m_true - m0); the pairs stay resident in device memory;
* use in FWI: the network's update is tried first (full, then half size); it is kept only
  if the true FDTD misfit decreases, otherwise the plain L-BFGS step is taken (see
  :class:`FWI`); at most two updates are kept per band by default;
* a sequence of networks: network k proposes the update after k kept ones; the second is
  fine-tuned from the first on pairs taken at the model the first network's update reaches
  (:func:`generate_stage_pairs`).

Feature scaling, cropping and batching are a few elementwise tensor operations (PyTorch as
plumbing); the network runs in the library's BF16 kernels (:mod:`.unet`), the gradients in
its FDTD kernels.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np
import torch

from .unet import UNet

EPS_FEATURE_SCALE = 10.0
ILLUM_FLOOR = 1e-6


@dataclass
class PreconditionerScales:
    eps_scale: float = 1.0    # target channel 0 = delta eps_r / eps_scale
    sig_scale: float = 1e-2   # target channel 1 = delta sigma / sig_scale (S/m)


def crop(a: torch.Tensor, npml: int) -> torch.Tensor:
    return a[npml:a.shape[0] - npml, npml:a.shape[1] - npml]


def features(ge, gs, eps, illum, npml: int, out: torch.Tensor | None = None) -> torch.Tensor:
    """[H, W, 4] FP32 network input from full-grid [ny, nx] arrays (see module docstring)."""
    ge, gs, eps, ill = (crop(a, npml) for a in (ge, gs, eps, illum))
    H, W = ge.shape
    x = out if out is not None else torch.empty(H, W, 4, dtype=torch.float32, device=ge.device)
    x[..., 0] = ge / ge.abs().max().clamp_min(1e-30)
    x[..., 1] = gs / gs.abs().max().clamp_min(1e-30)
    x[..., 2] = eps / EPS_FEATURE_SCALE
    x[..., 3] = torch.log10((ill / ill.max().clamp_min(1e-30)).clamp_min(ILLUM_FLOOR)) / 6.0 + 1.0
    return x


def targets(eps, sig, eps_true, sig_true, npml: int, scales: PreconditionerScales,
            out: torch.Tensor | None = None) -> torch.Tensor:
    de = crop(eps_true - eps, npml)
    ds = crop(sig_true - sig, npml)
    H, W = de.shape
    t = out if out is not None else torch.empty(H, W, 2, dtype=torch.float32, device=de.device)
    t[..., 0] = de / scales.eps_scale
    t[..., 1] = ds / scales.sig_scale
    return t


class LearnedPreconditioner:
    """A U-Net over the physical region of an FDTD grid (padding npml cells on each side), or
    a sequence of them: network k proposes the update after k learned updates of the band
    have been kept (the last one serves any later stage)."""

    def __init__(self, net, npml: int, scales: PreconditionerScales | None = None):
        self.nets = list(net) if isinstance(net, (list, tuple)) else [net]
        net = self.nets[0]
        self.net = net
        self.npml = npml
        self.scales = scales or PreconditionerScales()
        self._x = torch.empty(1, net.height, net.width, 4, dtype=torch.float32, device=net.device)

    def update(self, ge, gs, eps, illum, stage: int = 0):
        """(delta eps_r, delta sigma) on the full grid (zero in the absorbing layer)."""
        features(ge, gs, eps, illum, self.npml, out=self._x[0])
        y = self.nets[min(stage, len(self.nets) - 1)].forward(self._x)[0]
        p = self.npml
        de = torch.zeros_like(ge)
        ds = torch.zeros_like(gs)
        de[p:de.shape[0] - p, p:de.shape[1] - p] = y[..., 0] * self.scales.eps_scale
        ds[p:ds.shape[0] - p, p:ds.shape[1] - p] = y[..., 1] * self.scales.sig_scale
        return de, ds


def pair_fractions(seeds) -> np.ndarray:
    """The fraction a of the way from the start model to the truth at which each seed's
    training pair is taken: 0 for half of the seeds, else uniform in [0, 0.8)."""
    out = np.empty(len(seeds))
    for i, s in enumerate(seeds):
        r = np.random.default_rng([int(s), 77])
        out[i] = 0.0 if r.random() < 0.5 else 0.8 * r.random()
    return out


def generate_pairs(fd, models, N: int, wavelet, scales: PreconditionerScales, npml: int,
                   progress=None, fractions=None):
    """Training pairs for N models from the iterable ``models``, each (eps_true, sig_true,
    eps_init, sig_init) as device or host [ny, nx] arrays sharing the geometry of ``fd``,
    taken at m0 + a (m_true - m0) with a = fractions[i] (0 if not given).  Returns
    X [N, H, W, 4] and T [N, H, W, 2] on the device (and the seconds spent)."""
    ny, nx = fd.shape
    H, W = ny - 2 * npml, nx - 2 * npml
    dev = fd.device
    X = torch.empty(N, H, W, 4, dtype=torch.float32, device=dev)
    T = torch.empty(N, H, W, 2, dtype=torch.float32, device=dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for i, (et, st, ei, si) in enumerate(models):
        et, st, ei, si = (torch.as_tensor(a, dtype=torch.float32).to(dev) for a in (et, st, ei, si))
        if fractions is not None and fractions[i] > 0:
            a = float(fractions[i])
            ei = (ei + a * (et - ei)).contiguous()
            si = (si + a * (st - si)).contiguous()
        obs = fd.forward_model(et, st, wavelet)
        _, illum = fd.forward_model(ei, si, wavelet, illumination=True)
        _, ge, gs = fd.misfit_and_gradient(ei, si, wavelet, obs)
        features(ge, gs, ei, illum, npml, out=X[i])
        targets(ei, si, et, st, npml, scales, out=T[i])
        if progress:
            progress(i)
    torch.cuda.synchronize(dev)
    return X, T, time.perf_counter() - t0


def generate_stage_pairs(fd, models, N: int, wavelet, scales: PreconditionerScales, npml: int,
                         pre: "LearnedPreconditioner", mask, fractions=None, progress=None):
    """Training pairs for the next network of a sequence: for each of the N models (as in
    :func:`generate_pairs`), apply ``pre``'s update at the start model as the FWI driver does
    (masked, then eps_r >= 1, sigma >= 0), and pair the gradient at the updated model (with
    the start model's illumination, which the driver keeps for the band) with the remaining
    update to the truth.  Returns X, T on the device and the seconds spent."""
    ny, nx = fd.shape
    H, W = ny - 2 * npml, nx - 2 * npml
    dev = fd.device
    m = mask.to(device=dev, dtype=torch.float32)
    X = torch.empty(N, H, W, 4, dtype=torch.float32, device=dev)
    T = torch.empty(N, H, W, 2, dtype=torch.float32, device=dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for i, (et, st, ei, si) in enumerate(models):
        et, st, ei, si = (torch.as_tensor(a, dtype=torch.float32).to(dev) for a in (et, st, ei, si))
        if fractions is not None and fractions[i] > 0:
            a = float(fractions[i])
            ei = (ei + a * (et - ei)).contiguous()
            si = (si + a * (st - si)).contiguous()
        obs = fd.forward_model(et, st, wavelet)
        _, illum = fd.forward_model(ei, si, wavelet, illumination=True)
        _, ge, gs = fd.misfit_and_gradient(ei, si, wavelet, obs)
        de, ds = pre.update(ge, gs, ei, illum)
        e1 = (ei + de * m).clamp_min(1.0).contiguous()
        s1 = (si + ds * m).clamp_min(0.0).contiguous()
        _, ge1, gs1 = fd.misfit_and_gradient(e1, s1, wavelet, obs)
        features(ge1, gs1, e1, illum, npml, out=X[i])
        targets(e1, s1, et, st, npml, scales, out=T[i])
        if progress:
            progress(i)
    torch.cuda.synchronize(dev)
    return X, T, time.perf_counter() - t0


def train(net: UNet, X, T, epochs: int, batch: int, lr: float, seed: int = 0,
          lr_decay: float = 0.5, decay_every: int | None = None, log=None):
    """Adam on minibatches of (X, T) resident on the device; returns per-epoch mean losses."""
    N = X.shape[0]
    g = torch.Generator().manual_seed(seed)
    xb = torch.empty((batch,) + tuple(X.shape[1:]), dtype=torch.float32, device=X.device)
    tb = torch.empty((batch,) + tuple(T.shape[1:]), dtype=torch.float32, device=X.device)
    losses = []
    for ep in range(epochs):
        if decay_every and ep and ep % decay_every == 0:
            lr *= lr_decay
        perm = torch.randperm(N, generator=g).to(X.device)
        acc = torch.zeros(1, dtype=torch.float64, device=X.device)
        nb = 0
        for b0 in range(0, N - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            torch.index_select(X, 0, idx, out=xb)
            torch.index_select(T, 0, idx, out=tb)
            loss = net.train_step(xb, tb, lr=lr)
            acc += loss
            nb += 1
        losses.append(float(acc.item()) / max(nb, 1))
        if log:
            log(ep, losses[-1])
    return losses


def validation_loss(net: UNet, X, T, batch: int) -> float:
    """Mean loss over (X, T) without updating the network."""
    acc, nb = 0.0, 0
    for b0 in range(0, X.shape[0] - batch + 1, batch):
        loss, _ = net.loss_and_grad(X[b0:b0 + batch].contiguous(), T[b0:b0 + batch].contiguous())
        acc += float(loss.item())
        nb += 1
    return acc / max(nb, 1)


def _model_arrays(seed_nt):
    from .workloads import preconditioner_model
    wl = preconditioner_model(int(seed_nt[0]), nt=int(seed_nt[1]))
    return (np.asarray(wl.eps_true, np.float32), np.asarray(wl.sig_true, np.float32),
            np.asarray(wl.eps_init, np.float32), np.asarray(wl.sig_init, np.float32))


def seeded_models(seeds, nt: int, workers: int = 0):
    """(eps_true, sig_true, eps_init, sig_init) of the preconditioner workload for each seed,
    in order.  With ``workers`` > 0 the host-side generation runs in a pool of spawned
    processes (spawned, not forked: the parent already holds a CUDA context) and overlaps
    the GPU work that consumes the models."""
    jobs = [(int(s), nt) for s in seeds]
    if workers <= 0:
        for j in jobs:
            yield _model_arrays(j)
        return
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(workers) as pool:
        yield from pool.imap(_model_arrays, jobs, chunksize=8)
