"""Shot sharding over ranks with a sum all-reduce of (J, g_eps_r, g_sigma).

The misfit is a sum over shots (Eq. objective) and so are its zero-lag gradients (Sec. 2.2):
each shot's forward and adjoint time loops are independent of every other shot's.  One
inversion of S shots on W GPUs therefore splits its shots over the ranks, each rank runs the
library's ``gf_misfit_and_gradient`` on its own subset, and one collective sums the partial
misfits and gradients.  Every rank ends with the same (J, g_eps_r, g_sigma), so the model
update that follows (L-BFGS, TV, clamping) runs replicated on each rank and no model is
broadcast.

* partition: round-robin, shot s on rank s mod W (ranks take shots spread across the
  surface, so the per-rank cost stays even when the CPML strips make edge shots dearer);
* reduction: one ``all_reduce(SUM)`` over a float64 vector [J, g_eps_r, g_sigma] (FP64 so
  that the cross-rank sum adds no rounding beyond the per-rank FP32 gradients; 2 x 8 bytes
  per cell, small beside a gradient's time loops);
* the process group is the caller's (NCCL with device tensors on GPUs, gloo with host
  tensors on the CPU); with no process group the sharding is the identity.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def shard_shots(nshots: int, rank: int, world: int) -> np.ndarray:
    """Indices of the shots that ``rank`` of ``world`` runs: rank, rank + world, ..."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("need 0 <= rank < world")
    return np.arange(rank, nshots, world, dtype=np.int64)


def _group_size(group) -> tuple[int, int]:
    if not (dist.is_available() and dist.is_initialized()):
        return 0, 1
    return dist.get_rank(group), dist.get_world_size(group)


def allreduce_sum(J: torch.Tensor, ge: torch.Tensor, gs: torch.Tensor, group=None):
    """Sum (J, g_eps_r, g_sigma) over the ranks of ``group`` in one collective; returns the
    summed tensors in the inputs' dtypes and devices (every rank gets the same values)."""
    _, world = _group_size(group)
    if world == 1:
        return J, ge, gs
    if J.numel() != 1:
        raise ValueError("J must hold one value")
    flat = torch.cat([J.reshape(-1).double(), ge.reshape(-1).double(),
                      gs.reshape(-1).double()])
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    n = ge.numel()
    return (flat[:1].to(J.dtype).reshape(J.shape),
            flat[1:1 + n].to(ge.dtype).reshape(ge.shape),
            flat[1 + n:].to(gs.dtype).reshape(gs.shape))


class ShardedGradient:
    """The gradient of one multi-shot acquisition with its shots split over the ranks.

    ``src`` [nshots][nsrc][2] and ``rec`` [nshots][nrec][2] describe the whole acquisition;
    this rank builds an evaluator on its round-robin share: by default an
    :class:`~.fdtd.FDTD` context on ``device``, or ``context(grid, src_share, rec_share)``.
    Calls take the whole acquisition's wavelet [nshots, nsrc, nt] (or [nt]) and observed
    traces [nshots, nt, nrec] and return the all-reduced (J, g_eps_r, g_sigma), the same on
    every rank.  The object stands in for an FDTD context in :class:`~.fwi.FWI`, which then
    runs one inversion replicated on every rank over the summed gradients."""

    def __init__(self, grid, src, rec, device=None, tiling=None, group=None, context=None,
                 share: tuple[int, int] | None = None):
        """``share`` = (rank, world) builds that rank's share without a process group (the
        collectives then sum over nothing: for running the shares one after the other)."""
        self.group = group
        self.rank, self.world = share if share is not None else _group_size(group)
        src = np.asarray(src)
        rec = np.asarray(rec)
        self.nshots = src.shape[0]
        self.shots = shard_shots(self.nshots, self.rank, self.world)
        if self.shots.size == 0:
            raise ValueError(f"rank {self.rank} has no shots: {self.nshots} shots on "
                             f"{self.world} ranks")
        if context is None:
            from .fdtd import FDTD
            self.fd = FDTD(grid, src[self.shots], rec[self.shots], device=device, tiling=tiling)
        else:
            self.fd = context(grid, src[self.shots], rec[self.shots])
        self._idx = torch.as_tensor(self.shots, device=self.fd.device)

    def __getattr__(self, name):
        # grid, shape, device, lib, tiling(), status() ... of the rank's own context
        if name == "fd":
            raise AttributeError(name)
        return getattr(self.fd, name)

    def close(self):
        self.fd.close()

    def _share(self, wavelet, observed):
        w = wavelet if wavelet.dim() == 1 else wavelet.to(self.fd.device)[self._idx]
        return w, observed.to(self.fd.device)[self._idx]

    def local(self, eps_r, sigma, wavelet, observed):
        """This rank's partial (J, g_eps_r, g_sigma) over its own shots (no collective)."""
        return self.fd.misfit_and_gradient(eps_r, sigma, *self._share(wavelet, observed))

    def misfit_and_gradient(self, eps_r, sigma, wavelet, observed):
        return allreduce_sum(*self.local(eps_r, sigma, wavelet, observed), group=self.group)

    def misfit(self, eps_r, sigma, wavelet, observed, out=None):
        """J summed over all ranks' shots (FP64 tensor of one value)."""
        J = self.fd.misfit(eps_r, sigma, *self._share(wavelet, observed), out=out)
        _, world = _group_size(self.group)
        if world > 1:
            dist.all_reduce(J, op=dist.ReduceOp.SUM, group=self.group)
        return J
