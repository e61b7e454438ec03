"""Dual-parameter FWI driver: L-BFGS with optional TV regularisation and multiscale bands.

The paper drives its CUDA forward/adjoint with a PyTorch optimiser (Adam in its demo script,
Sec. 3.1), with a TV term (Algorithm 3), multiscale inversion through its ``freq`` option
(Sec. 3.4), gradient zeroing near the sources and clamping to eps_r >= 1, sigma >= 0.  This
driver keeps those pieces around a limited-memory BFGS update:

* every misfit, gradient and TV evaluation runs in the CUDA library (``gf_misfit``,
  ``gf_misfit_and_gradient``, ``gf_tv_gradient``); the L-BFGS two-loop recursion and the
  line search are a few vector operations on the GPU (PyTorch tensors as plumbing);
* variables x = (eps_r, sigma / sigma_ref) on the masked cells; the gradient in x is
  (g_eps_r, sigma_ref g_sigma);
* line search: backtracking with the Armijo condition; the first step of each band is
  scaled so that the largest eps_r change equals ``first_step`` (relative to max eps_r);
  after each step eps_r and sigma are clamped to their physical ranges (Sec. 3.1);
* multiscale: a sequence of bands (Ricker peak frequency, iterations); the L-BFGS memory is
  reset at each band change;
* optional learned preconditioner (:class:`.precond.LearnedPreconditioner`): each iteration
  first tries the network's update computed from the raw gradient, the model and the
  illumination of the band's starting model (full size, then half); the update is kept only
  if the FDTD misfit decreases, otherwise the plain L-BFGS step is taken and the network is
  not consulted again in that band (its prediction no longer helps there, and each try costs
  a forward model); after ``learned_max`` kept updates (default 2) the rest of the band is
  plain L-BFGS too.  The k-th update of a band comes from the preconditioner's k-th network
  where it holds several.  Accepted steps of either kind feed the L-BFGS memory.
"""
from __future__ import annotations

import ctypes
import json
import time
from dataclasses import dataclass, field

import torch

from . import _lib
from .fdtd import FDTD, ricker


@dataclass
class FWIConfig:
    bands: tuple = ((400e6, 50),)      # (Ricker peak frequency, L-BFGS iterations)
    memory: int = 10                   # stored (s, y) pairs
    sigma_ref: float = 1e-2            # S/m: sigma enters the variables as sigma / sigma_ref
    first_step: float = 0.02           # first step changes eps_r by this fraction of max eps_r
    armijo: float = 1e-4
    backtracks: int = 8
    tv: bool = False
    tv_lambda: float = 0.02
    tv_mu: float = 0.2
    tv_iters: int = 20
    tv_weight: float = 0.1
    eps_min: float = 1.0
    sigma_min: float = 0.0
    # learned step: scales of the network's update tried in turn (each costs one misfit
    # evaluation); after a rejection the network is consulted again once this many L-BFGS
    # iterations have passed (0 = not again in this band)
    learned_scales: tuple = (1.0, 0.5)
    learned_retry: int = 0
    # most learned updates kept per band before the rest is plain L-BFGS (0 = no limit)
    learned_max: int = 2


@dataclass
class FWIHistory:
    misfit: list = field(default_factory=list)        # J at the start of each iteration
    evaluations: list = field(default_factory=list)   # FDTD evaluations per iteration
                                                      # (misfit-only or misfit + gradient)
    passes: list = field(default_factory=list)        # forward-equivalent time loops per
                                                      # iteration: a misfit-only evaluation is
                                                      # 1 (forward), a gradient 2 (+ adjoint)
    seconds: list = field(default_factory=list)       # wall time per iteration (synchronised)
    band: list = field(default_factory=list)
    learned: list = field(default_factory=list)       # True where the learned update was kept


class FWI:
    """L-BFGS inversion of (eps_r, sigma) on an :class:`FDTD` context.

    ``observed(f0)`` returns the observed traces [nshots, nt, nrec] (device FP32) for the
    band with Ricker peak frequency f0; ``mask`` [ny, nx] (1 = free, 0 = fixed) zeroes the
    gradient where the model must not move (the absorbing layer, the rows of the sources)."""

    def __init__(self, fdtd: FDTD, observed, mask: torch.Tensor, config: FWIConfig | None = None,
                 preconditioner=None):
        self.fd = fdtd
        self.pre = preconditioner
        self.observed = observed
        self.cfg = config or FWIConfig()
        self.mask = mask.to(device=fdtd.device, dtype=torch.float32)
        ny, nx = fdtd.shape
        self._tv_scratch = None
        if self.cfg.tv:
            nb = self.fd.lib.gf_tv_scratch_bytes(nx, ny)
            self._tv_scratch = torch.empty(nb, dtype=torch.uint8, device=fdtd.device)
        self._J = torch.empty(1, dtype=torch.float64, device=fdtd.device)
        self.passes = 0   # forward-equivalent time loops run so far (misfit 1, gradient 2)

    # -- evaluations through the library ---------------------------------------------------
    def _misfit(self, eps, sig, wav, obs) -> float:
        self.passes += 1
        return float(self.fd.misfit(eps, sig, wav, obs, out=self._J).item())

    def _tv(self, model, grad):
        ny, nx = self.fd.shape
        c = self.cfg
        for t in (model, grad):
            if t.shape != (ny, nx) or t.dtype != torch.float32 or not t.is_contiguous() \
                    or t.device != self.fd.device:
                raise ValueError("TV needs contiguous float32 [ny, nx] tensors on the device")
        rc = self.fd.lib.gf_tv_gradient(nx, ny, model.data_ptr(), grad.data_ptr(),
                                        self._tv_scratch.data_ptr(), c.tv_lambda, c.tv_mu,
                                        c.tv_iters, c.tv_weight, self.fd._stream())
        _lib.check(self.fd.lib, None, rc)

    def gradient(self, eps, sig, wav, obs, raw: bool = False):
        """J and the masked gradient in the variables x = (eps_r, sigma / sigma_ref) (and the
        raw model gradients with ``raw``)."""
        J, ge, gs = self.fd.misfit_and_gradient(eps, sig, wav, obs)
        self.passes += 2
        if raw:
            ge0, gs0 = ge.clone(), gs.clone()
        if self.cfg.tv:
            self._tv(eps, ge)
            self._tv(sig, gs)
        gx = torch.cat([(ge * self.mask).reshape(-1), (gs * self.mask * self.cfg.sigma_ref).reshape(-1)])
        return (float(J.item()), gx, ge0, gs0) if raw else (float(J.item()), gx)

    # -- the iteration ---------------------------------------------------------------------
    def _split(self, x):
        n = x.numel() // 2
        ny, nx = self.fd.shape
        eps = x[:n].reshape(ny, nx).clamp_min(self.cfg.eps_min).contiguous()
        sig = (x[n:].reshape(ny, nx) * self.cfg.sigma_ref).clamp_min(self.cfg.sigma_min).contiguous()
        return eps, sig

    def run(self, eps0: torch.Tensor, sig0: torch.Tensor, callback=None,
            stop_misfit: float | None = None, checkpoint: str | None = None,
            checkpoint_every: int = 0, resume: str | None = None, log: str | None = None):
        """Iterate every band; with ``stop_misfit`` stop as soon as J <= stop_misfit.

        ``checkpoint`` / ``checkpoint_every``: after every that many iterations of a band, save
        the FWI state (model, gradient, misfit, L-BFGS pairs, band and iteration, the
        learned step's state and the history so far) to that file.  ``resume``: continue from
        such a file instead of starting at (eps0, sig0); a resumed run continues exactly as the
        uninterrupted one would (every kernel is deterministic).  ``log``: append one JSON line
        per iteration (band, iteration, misfit, evaluations, seconds, learned)."""
        c = self.cfg
        dev = self.fd.device
        hist = FWIHistory()
        learned = self.pre is not None
        x = torch.cat([eps0.reshape(-1).double(), (sig0.reshape(-1) / c.sigma_ref).double()])
        x = x.to(dev)
        st = torch.load(resume, map_location=dev, weights_only=False) if resume else None
        if st is not None:
            for k in ("misfit", "evaluations", "passes", "seconds", "band", "learned"):
                getattr(hist, k).extend(st["hist"].get(k, []))
        logf = open(log, "a") if log else None
        J = float("nan")
        for bi, (f0, iters) in enumerate(c.bands):
            if st is not None and bi < st["band_index"]:
                continue
            wav = torch.tensor(ricker(f0, self.fd.grid.dt, self.fd.grid.nt), device=dev)
            obs = self.observed(f0)
            ge = gs = illum = None
            if st is not None and bi == st["band_index"]:
                x, g, J = st["x"].to(dev), st["g"].to(dev), st["J"]
                S = [t.to(dev) for t in st["S"]]
                Y = [t.to(dev) for t in st["Y"]]
                first, use_net, it0 = st["first"], st["use_net"], st["iteration"]
                n_kept = st.get("n_kept", 0)
                retry_at = st.get("retry_at", -1)
                if learned:
                    ge, gs, illum = (st[k].to(dev) for k in ("ge", "gs", "illum"))
                eps, sig = self._split(x.float())
                st = None
            else:
                S, Y = [], []
                eps, sig = self._split(x.float())
                if learned:
                    _, illum = self.fd.forward_model(eps, sig, wav, illumination=True)
                    J, g, ge, gs = self.gradient(eps, sig, wav, obs, raw=True)
                else:
                    J, g = self.gradient(eps, sig, wav, obs)
                g = g.double()
                first = True
                use_net = learned   # the network is tried until its update is rejected
                n_kept = 0          # learned updates kept in this band (selects the network)
                retry_at = -1       # iteration at which a rejected network is tried again
                it0 = 0
            n = x.numel() // 2
            for it in range(it0, iters):
                if stop_misfit is not None and J <= stop_misfit:
                    break
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                p0 = self.passes
                tries = 0
                kept = False
                if learned and not use_net and 0 <= retry_at <= it:
                    use_net, retry_at = True, -1
                if use_net:
                    de, ds = self.pre.update(ge, gs, eps, illum, stage=n_kept)
                    d_l = torch.cat([(de * self.mask).reshape(-1).double(),
                                     (ds * self.mask / c.sigma_ref).reshape(-1).double()])
                    J_c = float("inf")
                    g_net = None
                    for si, scale in enumerate(c.learned_scales):
                        e_c, s_c = self._split((x + scale * d_l).float())
                        if si == 0:
                            # the full-size update with its gradient, reused when it is kept
                            J_c, g_net, ge_net, gs_net = self.gradient(e_c, s_c, wav, obs,
                                                                       raw=True)
                        else:
                            J_c = self._misfit(e_c, s_c, wav, obs)
                            g_net = None
                        tries += 1
                        if J_c < J:
                            break
                    if J_c < J:
                        kept = True
                        n_kept += 1
                        eps, sig = e_c, s_c
                        if 0 < c.learned_max <= n_kept:
                            use_net = False
                    else:
                        use_net = False
                        if c.learned_retry > 0:
                            retry_at = it + c.learned_retry
                if not kept:
                    # two-loop recursion (Nocedal & Wright, Algorithm 7.4)
                    q = g.clone()
                    alphas = []
                    for s_, y_ in zip(reversed(S), reversed(Y)):
                        rho = 1.0 / torch.dot(y_, s_)
                        a = rho * torch.dot(s_, q)
                        q -= a * y_
                        alphas.append((rho, a))
                    if S:
                        q *= torch.dot(S[-1], Y[-1]) / torch.dot(Y[-1], Y[-1])
                    for (s_, y_), (rho, a) in zip(zip(S, Y), reversed(alphas)):
                        b = rho * torch.dot(y_, q)
                        q += s_ * (a - b)
                    d = -q
                    slope = float(torch.dot(g, d))
                    if slope >= 0:  # not a descent direction: restart from steepest descent
                        S, Y, d, first = [], [], -g, True
                        slope = float(torch.dot(g, d))
                    alpha = 1.0
                    if first:
                        peak = float(d[:n].abs().max())
                        if peak > 0:
                            alpha = c.first_step * float(x[:n].max()) / peak
                    accepted = False
                    for bt in range(c.backtracks):
                        eps, sig = self._split((x + alpha * d).float())
                        if bt == 0 and not first:
                            # an L-BFGS step is usually accepted at alpha = 1: evaluate the first
                            # trial with its gradient (the same J as the misfit-only forward)
                            # and reuse both when Armijo holds; backtracking evaluates misfits
                            if learned:
                                J_new, g_try, ge_try, gs_try = self.gradient(eps, sig, wav, obs,
                                                                             raw=True)
                            else:
                                J_new, g_try = self.gradient(eps, sig, wav, obs)
                        else:
                            J_new = self._misfit(eps, sig, wav, obs)
                            g_try = None
                        tries += 1
                        if J_new <= J + c.armijo * alpha * slope:
                            accepted = True
                            break
                        alpha *= 0.5
                    if not accepted:
                        self._record(hist, logf, f0, it, J, tries, self.passes - p0,
                                     time.perf_counter() - t0, False)
                        eps, sig = self._split(x.float())
                        break
                # the accepted model (projected onto the physical ranges), then its gradient
                x_new = torch.cat([eps.reshape(-1).double(), (sig.reshape(-1) / c.sigma_ref).double()])
                if kept and g_net is not None:
                    J_next, g_new, ge, gs = J_c, g_net, ge_net, gs_net
                elif not kept and g_try is not None:
                    J_next, g_new = J_new, g_try
                    if learned:
                        ge, gs = ge_try, gs_try
                else:
                    if learned:
                        J_next, g_new, ge, gs = self.gradient(eps, sig, wav, obs, raw=True)
                    else:
                        J_next, g_new = self.gradient(eps, sig, wav, obs)
                    tries += 1
                g_new = g_new.double()
                s_k, y_k = x_new - x, g_new - g
                if float(torch.dot(s_k, y_k)) > 1e-12 * float(torch.dot(s_k, s_k)) ** 0.5:
                    S.append(s_k)
                    Y.append(y_k)
                    if len(S) > c.memory:
                        S.pop(0)
                        Y.pop(0)
                torch.cuda.synchronize(dev)
                self._record(hist, logf, f0, it, J, tries, self.passes - p0,
                             time.perf_counter() - t0, kept)
                x, g, J, first = x_new, g_new, J_next, False
                if checkpoint and checkpoint_every > 0 and (it + 1) % checkpoint_every == 0:
                    state = dict(band_index=bi, iteration=it + 1, x=x.cpu(), g=g.cpu(), J=J,
                                 S=[t.cpu() for t in S], Y=[t.cpu() for t in Y], first=first,
                                 use_net=use_net, retry_at=retry_at, n_kept=n_kept,
                                 hist={k: list(getattr(hist, k)) for k in
                                       ("misfit", "evaluations", "passes", "seconds", "band",
                                        "learned")})
                    if learned:
                        state.update(ge=ge.cpu(), gs=gs.cpu(), illum=illum.cpu())
                    torch.save(state, checkpoint)
                if callback:
                    callback(it, J, x)
        if logf:
            logf.close()
        eps, sig = self._split(x.float())
        hist.final_misfit = J
        return eps, sig, hist

    @staticmethod
    def _record(hist, logf, f0, it, J, evals, passes, seconds, learned):
        hist.misfit.append(J)
        hist.evaluations.append(evals)
        hist.passes.append(passes)
        hist.seconds.append(seconds)
        hist.band.append(f0)
        hist.learned.append(learned)
        if logf:
            logf.write(json.dumps({"band_f0": f0, "iteration": it, "misfit": J,
                                   "evaluations": evals, "passes": passes, "seconds": seconds,
                                   "learned": learned}) + "\n")
            logf.flush()


def interior_mask(grid, rows_below_top: int = 0) -> torch.Tensor:
    """1 on the physical cells below the first ``rows_below_top`` physical rows, 0 in the
    absorbing layer (the paper zeroes the gradient of the rows holding its sources,
    Sec. 3.1)."""
    m = torch.zeros(grid.ny, grid.nx)
    p = grid.npml
    m[p + rows_below_top:grid.ny - p, p:grid.nx - p] = 1.0
    return m
