"""The paper's calling convention: ``compute(device, dx, ny, nx, nz, time_windows, source,
source_location, source_step, receiver_location, receiver_step, pmlthick, source_amplitudes,
step, epsilon, sigma, miu, nsrc, nrx, freq, dt)`` (Sec. 3.1 demo listing, parameter tables
of Sec. 4), returning ``(traces, t)`` and differentiable with respect to epsilon and sigma.

Readings of the parameters (the paper lists names and example values only):

* the model arrays include the absorbing layer (pmlthick cells on each side, Sec. 3.1 demo
  strips them before saving) and are indexed [x][y][z] with nz = 1 (2-D TM; the demo zeroes
  ``grad[:, :pmlthick+1, :]``, the rows near the surface sources, so the second axis is depth);
* positions are metres from the array origin, converted to cells by rounding x/dx half up;
* shot s (s = 0 .. step-1) has its source at source_location + s * source_step; the nrx
  receivers of every shot are at receiver_location + r * receiver_step (r = 0 .. nrx-1);
* source = ['hertzian', 'z']: a z-polarised line source (TM mode, Ez traces, differentiable);
  ['hertzian', 'x'] or ['hertzian', 'y']: an x- or y-polarised one (TE mode, traces of Ex or
  Ey, not differentiable here: the TE gradient call, gf_misfit_and_gradient_te, takes
  observed traces, not the arbitrary trace cotangent autograd passes); source_amplitudes =
  ['ricker', A, f0]: a Ricker wavelet of amplitude A and peak frequency f0, replaced by
  ``freq`` when that is given (a multiscale band, Sec. 3.4);
* time_windows / dt steps (rounded); miu must be 1 (relative permeability is not inverted).

Every step runs in the library's kernels through :class:`FDTDFunction`; this module only
converts the arguments.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .fdtd import FDTD, FDTDFunction, ricker
from .workloads import GridSpec, default_pml

_contexts: dict = {}


def _cell(x: float, d: float) -> int:
    return int(math.floor(x / d + 0.5))


def paper_geometry(dx, dy, nx, ny, source_location, source_step, receiver_location,
                   receiver_step, step, nsrc, nrx):
    """Source and receiver cells (i, j) of every shot: src [step][nsrc][2], rec [step][nrx][2]."""
    if nsrc != 1:
        raise ValueError("one source per shot is supported (nsrc = 1)")
    src = np.zeros((step, 1, 2), dtype=np.int32)
    rec = np.zeros((step, nrx, 2), dtype=np.int32)
    for s in range(step):
        src[s, 0] = (_cell(source_location[0] + s * source_step[0], dx),
                     _cell(source_location[1] + s * source_step[1], dy))
        for r in range(nrx):
            rec[s, r] = (_cell(receiver_location[0] + r * receiver_step[0], dx),
                         _cell(receiver_location[1] + r * receiver_step[1], dy))
    for name, a in (("source", src), ("receiver", rec)):
        i, j = a[..., 0], a[..., 1]
        if (i < 1).any() or (j < 1).any() or (i > nx - 2).any() or (j > ny - 2).any():
            raise ValueError(f"a {name} lies outside the updated grid (1..nx-2, 1..ny-2)")
    return src, rec


def compute(device, dx, ny, nx, nz, time_windows, source, source_location, source_step,
            receiver_location, receiver_step, pmlthick, source_amplitudes, step, epsilon,
            sigma, miu, nsrc, nrx, freq, dt, dy=None):
    """traces [step, nt, nrx] (differentiable in epsilon and sigma) and the time axis."""
    if nz != 1:
        raise ValueError("2-D only: nz must be 1")
    pols = {"x": 0, "y": 1, "z": None}
    if len(source) != 2 or source[0] != "hertzian" or source[1] not in pols:
        raise ValueError("source must be ['hertzian', 'x' | 'y' | 'z']")
    pol = pols[source[1]]
    if pol is not None and torch.is_grad_enabled() and (
            getattr(epsilon, "requires_grad", False) or getattr(sigma, "requires_grad", False)):
        raise ValueError("compute() runs the x- and y-polarised (TE) model without autograd "
                         "(FDTD.misfit_and_gradient_te gives its gradients): run it without "
                         "gradients (torch.no_grad() or detached epsilon and sigma)")
    kind, amp, f0 = source_amplitudes
    if kind != "ricker":
        raise ValueError("only Ricker source amplitudes are supported")
    mu = miu if isinstance(miu, torch.Tensor) else torch.as_tensor(miu)
    if not torch.all(mu == 1):
        raise ValueError("relative permeability must be 1")
    f0 = float(freq) if freq else float(f0)
    dy = dx if dy is None else dy
    nt = int(round(time_windows / dt))
    dev = torch.device(device) if not isinstance(device, torch.device) else device
    if dev.type == "cuda" and dev.index is None:
        dev = torch.device("cuda", torch.cuda.current_device())
    for name, t in (("epsilon", epsilon), ("sigma", sigma)):
        if tuple(t.shape) != (nx, ny, 1):
            raise ValueError(f"{name} must be [nx, ny, 1] = [{nx}, {ny}, 1]")
    src, rec = paper_geometry(dx, dy, nx, ny, source_location, source_step, receiver_location,
                              receiver_step, step, nsrc, nrx)
    # one context per source kind: a TE call would drop the TM forward an autograd backward
    # still needs
    key = (str(dev), nx, ny, pmlthick, nt, dx, dy, dt, f0, src.tobytes(), rec.tobytes(),
           pol is None)
    fd = _contexts.get(key)
    if fd is None:
        g = default_pml(GridSpec(nx=nx, ny=ny, npml=pmlthick, nt=nt, dx=dx, dy=dy, dt=dt), f0)
        fd = FDTD(g, src, rec, device=dev)
        _contexts[key] = fd
    wav = torch.tensor(float(amp) * ricker(f0, dt, nt), dtype=torch.float32, device=dev)
    eps2 = epsilon[:, :, 0].transpose(0, 1).to(dev, torch.float32).contiguous()
    sig2 = sigma[:, :, 0].transpose(0, 1).to(dev, torch.float32).contiguous()
    if pol is None:
        traces = FDTDFunction.apply(eps2, sig2, fd, wav)
    else:
        # the source's own component of the TE traces (Ex for 'x', Ey for 'y')
        traces = fd.forward_model_te(eps2, sig2, wav, pol)[..., pol].contiguous()
    t = torch.arange(nt, dtype=torch.float64) * dt
    return traces, t
