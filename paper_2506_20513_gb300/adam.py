"""Staged-learning-rate Adam inversion: the optimisation loop of the paper's demonstration.

The paper updates eps_r and sigma with Adam, one learning rate per parameter (Sec. 2.3), in
an epoch loop (Sec. 3.1): one forward model and its gradient per epoch, the gradient zeroed
in the rows of the sources, the optimiser step, then eps_r >= 1 and sigma >= 0 enforced.
Its optimisation strategy (Sec. 3.4) adds TV regularisation, multiscale bands and a staged
learning rate; the cross-hole example (Results) runs a first stage on eps_r alone and then
updates eps_r and sigma together with smaller rates.

This driver runs that loop on the library's entry points: ``gf_misfit_and_gradient`` per
epoch, ``gf_tv_gradient`` for the TV term, ``gf_adam_update`` for the masked, bias-corrected,
clamped update of each parameter (one kernel each).  The schedule is a sequence of
:class:`Stage` s (epochs, rate of eps_r, rate of sigma, Ricker peak of the stage's data); a
rate of 0 freezes that parameter (its moments are left as they are).  Each parameter keeps
its own Adam state and step count across stages, as one optimiser whose rates change.

Loss: J = 1/2 sum (d - o)^2 divided by 1/2 sum o^2 of the stage's observed data.  Adam's
step is invariant to the scale of the loss except through its eps; dividing by the data's
energy gives eps the same meaning for every acquisition (the paper's mean-squared error is
another fixed rescaling of the same sum).
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import torch

from . import _lib
from .fdtd import FDTD, ricker


@dataclass
class Stage:
    epochs: int
    lr_eps: float          # learning rate of eps_r (0: frozen in this stage)
    lr_sig: float          # learning rate of sigma in S/m (0: frozen)
    f0: float | None = None  # Ricker peak frequency of this stage's data (None: the previous)


@dataclass
class AdamConfig:
    # the cross-hole schedule: eps_r alone for 50 epochs, then both (Results)
    stages: tuple = (Stage(50, 0.2, 0.0), Stage(100, 0.1, 1e-4))
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    tv: bool = False
    tv_lambda: float = 0.02
    tv_mu: float = 0.2
    tv_iters: int = 20
    tv_weight: float = 0.1
    eps_min: float = 1.0
    sigma_min: float = 0.0


@dataclass
class AdamHistory:
    misfit: list = field(default_factory=list)    # normalised J at the start of each epoch
    seconds: list = field(default_factory=list)   # wall time per epoch (synchronised)
    stage: list = field(default_factory=list)


def stage_of(stages, epoch: int) -> int:
    """Index of the stage that epoch (0-based) falls in; -1 past the last."""
    end = 0
    for i, s in enumerate(stages):
        end += s.epochs
        if epoch < end:
            return i
    return -1


class StagedAdam:
    """The staged Adam loop on an :class:`FDTD` context (or a sharded one).

    ``observed(f0)`` returns the observed traces [nshots, nt, nrec] (device FP32) for data of
    Ricker peak f0; ``mask`` [ny, nx] (1 = free, 0 = fixed) zeroes the update where the model
    must not move (the absorbing layer, the rows of the sources); ``f0`` is the data's peak
    frequency for stages that name none."""

    def __init__(self, fdtd: FDTD, observed, mask: torch.Tensor, f0: float,
                 config: AdamConfig | None = None):
        self.fd = fdtd
        self.observed = observed
        self.f0 = f0
        self.cfg = config or AdamConfig()
        dev = fdtd.device
        self.mask = mask.to(device=dev, dtype=torch.float32).contiguous()
        ny, nx = fdtd.shape
        self._tv_scratch = None
        if self.cfg.tv:
            nb = self.fd.lib.gf_tv_scratch_bytes(nx, ny)
            self._tv_scratch = torch.empty(nb, dtype=torch.uint8, device=dev)
        z = lambda: torch.zeros((ny, nx), dtype=torch.float32, device=dev)
        self.m = {"eps": z(), "sig": z()}
        self.v = {"eps": z(), "sig": z()}
        self.t = {"eps": 0, "sig": 0}

    def _tv(self, model, grad):
        ny, nx = self.fd.shape
        c = self.cfg
        rc = self.fd.lib.gf_tv_gradient(nx, ny, model.data_ptr(), grad.data_ptr(),
                                        self._tv_scratch.data_ptr(), c.tv_lambda, c.tv_mu,
                                        c.tv_iters, c.tv_weight, self.fd._stream())
        _lib.check(self.fd.lib, None, rc)

    def _update(self, key, x, g, lr, gscale, xmin):
        c = self.cfg
        self.t[key] += 1
        rc = self.fd.lib.gf_adam_update(x.numel(), x.data_ptr(), g.data_ptr(),
                                        self.m[key].data_ptr(), self.v[key].data_ptr(),
                                        self.mask.data_ptr(), gscale, lr, c.beta1, c.beta2,
                                        c.eps, self.t[key], xmin, self.fd._stream())
        _lib.check(self.fd.lib, None, rc)

    def step(self, eps, sig, wav, obs, lr_eps: float, lr_sig: float, obs_energy: float):
        """One epoch in place on (eps, sig): gradient, TV, masked Adam updates.  Returns the
        normalised misfit at the model before the update."""
        J, ge, gs = self.fd.misfit_and_gradient(eps, sig, wav, obs)
        if self.cfg.tv:
            if lr_eps > 0:
                self._tv(eps, ge)
            if lr_sig > 0:
                self._tv(sig, gs)
        inv = 1.0 / obs_energy
        if lr_eps > 0:
            self._update("eps", eps, ge, lr_eps, inv, self.cfg.eps_min)
        if lr_sig > 0:
            self._update("sig", sig, gs, lr_sig, inv, self.cfg.sigma_min)
        return float(J.item()) * inv

    def run(self, eps0: torch.Tensor, sig0: torch.Tensor, callback=None):
        """Every stage in turn from (eps0, sig0); returns (eps_r, sigma, history)."""
        c = self.cfg
        dev = self.fd.device
        g = self.fd.grid
        eps = eps0.to(device=dev, dtype=torch.float32).clone().contiguous()
        sig = sig0.to(device=dev, dtype=torch.float32).clone().contiguous()
        hist = AdamHistory()
        f0 = self.f0
        epoch = 0
        for si, st in enumerate(c.stages):
            f0 = st.f0 if st.f0 is not None else f0
            wav = torch.tensor(ricker(f0, g.dt, g.nt), device=dev)
            obs = self.observed(f0)
            energy = 0.5 * float((obs.double() ** 2).sum())
            if not energy > 0:
                raise ValueError("observed data of zero energy")
            for _ in range(st.epochs):
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                J = self.step(eps, sig, wav, obs, st.lr_eps, st.lr_sig, energy)
                torch.cuda.synchronize(dev)
                hist.misfit.append(J)
                hist.seconds.append(time.perf_counter() - t0)
                hist.stage.append(si)
                if callback:
                    callback(epoch, J, eps, sig)
                epoch += 1
        return eps, sig, hist
