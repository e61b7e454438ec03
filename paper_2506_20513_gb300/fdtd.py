"""PyTorch-facing API over the C ABI (device memory, streams and autograd glue only).

* :class:`FDTD` wraps one ``gf_ctx``: ``forward_model`` (traces), ``misfit_and_gradient``
  (Eq. objective and its exact gradients), ``forward``/``adjoint`` for autograd.
* :class:`FDTDFunction` is the ``torch.autograd.Function`` hookup the paper describes
  (Sec. 2.3): forward = Algorithm 1, backward = Algorithm 2, both in the CUDA kernels.
* :func:`ricker` calls the library's host helper.

Workspaces are allocated through PyTorch (``torch.empty(..., dtype=uint8)``) and handed to
the library with ``gf_set_workspace``, so device memory stays under PyTorch's allocator.
There is no CPU path: CUDA tensors are required and a missing library raises.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from .workloads import GridSpec


def _grid_desc(g: GridSpec) -> _lib.GridDesc:
    return _lib.GridDesc(g.nx, g.ny, g.npml, g.nt, g.dx, g.dy, g.dt, g.pml_order,
                         g.pml_sigma_max, g.pml_kappa_max, g.pml_alpha_max, g.pml_eps_ref)


def ricker(f0: float, dt: float, nt: int, amp: float = 1.0, lib_path: str | None = None) -> np.ndarray:
    """Ricker wavelet [nt] (FP32) from the library's host helper ``gf_ricker``."""
    lib = _lib.load(lib_path)
    out = np.zeros(nt, dtype=np.float32)
    rc = lib.gf_ricker(out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), nt, dt, f0, amp)
    _lib.check(lib, None, rc)
    return out


def _dev_f32(t: torch.Tensor, shape, name: str, device: torch.device) -> torch.Tensor:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.device != device:
        raise ValueError(f"{name} must live on {device} (got {t.device})")
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t.contiguous()


@dataclass
class Tiling:
    """Interior tile size and time steps per launch (0 = library default / largest that
    fits) and the tile-kernel variant (None = keep)."""
    tile_w: int = 0
    tile_h: int = 0
    steps: int = 0
    variant: int | None = None


class FDTD:
    """One acquisition on one grid: ``nshots`` shots advanced together on ``device``."""

    def __init__(self, grid: GridSpec, src, rec, device=None, tiling: Tiling | None = None,
                 lib_path: str | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("FDTD needs a CUDA device (the library has no CPU path)")
        self.lib = _lib.load(lib_path)
        self.grid = grid
        self.device = torch.device(device if device is not None else "cuda", 0) \
            if not isinstance(device, torch.device) else device
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        src = np.ascontiguousarray(src, dtype=np.int32)
        rec = np.ascontiguousarray(rec, dtype=np.int32)
        if src.ndim != 3 or rec.ndim != 3 or src.shape[2] != 2 or rec.shape[2] != 2 \
                or src.shape[0] != rec.shape[0]:
            raise ValueError("src must be [nshots][nsrc][2], rec [nshots][nrec][2]")
        self.nshots, self.nsrc, self.nrec = src.shape[0], src.shape[1], rec.shape[1]
        self._src, self._rec = src, rec
        acq = _lib.Acquisition(self.nshots, self.nsrc, self.nrec,
                               src.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                               rec.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        gd = _grid_desc(grid)
        ctx = ctypes.c_void_p()
        rc = self.lib.gf_create(ctypes.byref(ctx), ctypes.byref(gd), ctypes.byref(acq),
                                self.device.index)
        _lib.check(self.lib, None, rc)
        self.ctx = ctx
        self._ws = None
        self._ws_full = False
        if tiling is not None:
            self.set_tiling(tiling)

    # -- housekeeping ------------------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            self.lib.gf_destroy(self.ctx)
            self.ctx = None
            self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tiling(self, t: Tiling):
        if t.variant is not None:
            _lib.check(self.lib, self.ctx, self.lib.gf_set_variant(self.ctx, t.variant))
        _lib.check(self.lib, self.ctx, self.lib.gf_set_tiling(self.ctx, t.tile_w, t.tile_h, t.steps))
        # the workspace holds per-tile counters: its size follows the tiling
        self._ws = None
        self._ws_full = False

    def tiling(self) -> Tiling:
        v = [ctypes.c_int() for _ in range(4)]
        _lib.check(self.lib, self.ctx, self.lib.gf_get_tiling(self.ctx, *[ctypes.byref(x) for x in v]))
        return Tiling(*[x.value for x in v])

    def set_storage(self, checkpoint_every: int = 0, reconstruct: bool = False):
        """0: keep the full forward wavefield; k > 0: checkpoint every k steps and recompute
        each segment during the adjoint (same results, less memory, one extra forward); with
        ``reconstruct`` the recomputation keeps only a boundary ring per step and the adjoint
        runs the updates backwards inside each segment (experimental: its error grows with k
        and the conductivity)."""
        mode = ((_lib.GF_STORE_RECONSTRUCT if reconstruct else _lib.GF_STORE_CHECKPOINT)
                if checkpoint_every > 0 else _lib.GF_STORE_FULL)
        _lib.check(self.lib, self.ctx, self.lib.gf_set_storage(self.ctx, mode, checkpoint_every))
        self._store_mode = mode
        self._ws = None
        self._ws_full = False

    def workspace_bytes(self, forward_only: bool = False) -> int:
        n = ctypes.c_size_t()
        _lib.check(self.lib, self.ctx, self.lib.gf_workspace_size(
            self.ctx, getattr(self, "_store_mode", _lib.GF_STORE_FULL), int(forward_only),
            ctypes.byref(n)))
        return n.value

    def _workspace(self, full: bool):
        if self._ws is not None and (self._ws_full or not full):
            return
        nbytes = self.workspace_bytes(forward_only=not full)
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self._ws.data_ptr()
        aligned = (base + 255) // 256 * 256
        _lib.check(self.lib, self.ctx, self.lib.gf_set_workspace(self.ctx, aligned, nbytes))
        self._ws_full = full

    @property
    def shape(self):
        return (self.grid.ny, self.grid.nx)

    @property
    def trace_shape(self):
        return (self.nshots, self.grid.nt, self.nrec)

    def _stream(self):
        return torch.cuda.current_stream(self.device).cuda_stream

    def _model(self, eps_r, sigma):
        return (_dev_f32(eps_r, self.shape, "eps_r", self.device),
                _dev_f32(sigma, self.shape, "sigma", self.device))

    def _wavelet(self, wavelet):
        w = wavelet
        if w.dim() == 1:
            w = w.reshape(1, 1, -1).expand(self.nshots, self.nsrc, -1)
        return _dev_f32(w.contiguous(), (self.nshots, self.nsrc, self.grid.nt), "wavelet",
                        self.device)

    def status(self):
        """Synchronise and raise if a kernel flagged an invalid model or non-finite data."""
        _lib.check(self.lib, self.ctx, self.lib.gf_status(self.ctx, self._stream()))

    # -- the calls of the paper's statement of the problem ---------------------------------
    def forward_model(self, eps_r, sigma, wavelet, illumination: bool = False,
                      fields: bool = False):
        """traces [nshots, nt, nrec] (Ez), then the illumination [ny, nx] if asked, then the
        receivers' magnetic components [nshots, nt, nrec, 2] (Hx^{n-1/2}, Hy^{n-1/2} at the
        staggered nodes of each receiver cell) if ``fields``."""
        e, s = self._model(eps_r, sigma)
        w = self._wavelet(wavelet)
        self._workspace(full=False)
        tr = torch.empty(self.trace_shape, dtype=torch.float32, device=self.device)
        ill = torch.empty(self.shape, dtype=torch.float32, device=self.device) if illumination else None
        if fields:
            h = torch.empty(self.trace_shape + (2,), dtype=torch.float32, device=self.device)
            rc = self.lib.gf_forward_model_fields(
                self.ctx, e.data_ptr(), s.data_ptr(), w.data_ptr(), tr.data_ptr(), h.data_ptr(),
                ill.data_ptr() if ill is not None else None, self._stream())
        else:
            rc = self.lib.gf_forward_model(self.ctx, e.data_ptr(), s.data_ptr(), w.data_ptr(),
                                           tr.data_ptr(), ill.data_ptr() if ill is not None else None,
                                           self._stream())
        _lib.check(self.lib, self.ctx, rc)
        out = (tr,) + ((ill,) if illumination else ()) + ((h,) if fields else ())
        return out if len(out) > 1 else tr

    def forward_model_te(self, eps_r, sigma, wavelet, polarisation: int = 0):
        """Traces of the TE mode [nshots, nt, nrec, 3] (Ex^n, Ey^n, Hz^{n-1/2} at each receiver
        cell's nodes) for x-directed (``polarisation`` 0) or y-directed (1) sources."""
        e, s = self._model(eps_r, sigma)
        w = self._wavelet(wavelet)
        self._workspace(full=False)
        tr = torch.empty(self.trace_shape + (3,), dtype=torch.float32, device=self.device)
        rc = self.lib.gf_forward_model_te(self.ctx, e.data_ptr(), s.data_ptr(), w.data_ptr(),
                                          int(polarisation), tr.data_ptr(), self._stream())
        _lib.check(self.lib, self.ctx, rc)
        return tr

    def misfit_and_gradient_te(self, eps_r, sigma, wavelet, observed, polarisation: int = 0,
                               return_traces: bool = False):
        """TE mode: J = 1/2 sum (d - o)^2 over the source component's traces (observed
        [nshots, nt, nrec]: Ex for ``polarisation`` 0, Ey for 1), dJ/deps_r and dJ/dsigma
        [ny, nx]; with ``return_traces`` also the traces [nshots, nt, nrec, 3]."""
        e, s = self._model(eps_r, sigma)
        w = self._wavelet(wavelet)
        o = _dev_f32(observed, self.trace_shape, "observed", self.device)
        self._workspace(full=False)
        J = torch.empty(1, dtype=torch.float64, device=self.device)
        ge = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        gs = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        tr = torch.empty(self.trace_shape + (3,), dtype=torch.float32, device=self.device) \
            if return_traces else None
        rc = self.lib.gf_misfit_and_gradient_te(
            self.ctx, e.data_ptr(), s.data_ptr(), w.data_ptr(), int(polarisation), o.data_ptr(),
            J.data_ptr(), ge.data_ptr(), gs.data_ptr(),
            tr.data_ptr() if tr is not None else None, self._stream())
        _lib.check(self.lib, self.ctx, rc)
        return (J, ge, gs, tr) if return_traces else (J, ge, gs)

    def misfit_te(self, eps_r, sigma, wavelet, observed, polarisation: int = 0,
                  out: torch.Tensor | None = None):
        """TE mode: J = 1/2 sum (d - o)^2 over the source component's traces only (a
        line-search evaluation), FP64 device scalar."""
        e, s = self._model(eps_r, sigma)
        w = self._wavelet(wavelet)
        o = _dev_f32(observed, self.trace_shape, "observed", self.device)
        self._workspace(full=False)
        J = out if out is not None else torch.empty(1, dtype=torch.float64, device=self.device)
        if J.dtype != torch.float64 or J.device != self.device or J.numel() < 1:
            raise ValueError("out must be a float64 tensor on the context's device")
        rc = self.lib.gf_misfit_te(self.ctx, e.data_ptr(), s.data_ptr(), w.data_ptr(),
                                   int(polarisation), o.data_ptr(), J.data_ptr(), self._stream())
        _lib.check(self.lib, self.ctx, rc)
        return J

    def misfit_and_gradient(self, eps_r, sigma, wavelet, observed, return_traces: bool = False):
        """J = 1/2 sum (d - o)^2 (FP64 device scalar), dJ/deps_r and dJ/dsigma [ny, nx].

        Host (CPU) tensors are accepted: they are copied to the device, and the results are
        copied back to host memory (the end-to-end path)."""
        host = not eps_r.is_cuda
        if host:
            nb = True
            eps_r = eps_r.to(self.device, non_blocking=nb)
            sigma = sigma.to(self.device, non_blocking=nb)
            wavelet = wavelet.to(self.device, non_blocking=nb)
            observed = observed.to(self.device, non_blocking=nb)
        e, s = self._model(eps_r, sigma)
        w = self._wavelet(wavelet)
        o = _dev_f32(observed, self.trace_shape, "observed", self.device)
        self._workspace(full=True)
        J = torch.empty(1, dtype=torch.float64, device=self.device)
        ge = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        gs = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        tr = torch.empty(self.trace_shape, dtype=torch.float32, device=self.device) \
            if return_traces else None
        rc = self.lib.gf_misfit_and_gradient(self.ctx, e.data_ptr(), s.data_ptr(), w.data_ptr(),
                                             o.data_ptr(), J.data_ptr(), ge.data_ptr(),
                                             gs.data_ptr(), tr.data_ptr() if tr is not None else None,
                                             self._stream())
        _lib.check(self.lib, self.ctx, rc)
        if host:
            out = [J.to("cpu"), ge.to("cpu"), gs.to("cpu")]
            if return_traces:
                out.append(tr.to("cpu"))
            return tuple(out)
        return (J, ge, gs, tr) if return_traces else (J, ge, gs)

    def misfit(self, eps_r, sigma, wavelet, observed, out: torch.Tensor | None = None):
        """J = 1/2 sum (d - o)^2 only (a line-search evaluation), FP64 device scalar."""
        e, s = self._model(eps_r, sigma)
        w = self._wavelet(wavelet)
        o = _dev_f32(observed, self.trace_shape, "observed", self.device)
        self._workspace(full=False)
        J = out if out is not None else torch.empty(1, dtype=torch.float64, device=self.device)
        if J.dtype != torch.float64 or J.device != self.device or J.numel() < 1:
            raise ValueError("out must be a float64 tensor on the context's device")
        rc = self.lib.gf_misfit(self.ctx, e.data_ptr(), s.data_ptr(), w.data_ptr(), o.data_ptr(),
                                J.data_ptr(), self._stream())
        _lib.check(self.lib, self.ctx, rc)
        return J

    def forward(self, eps_r, sigma, wavelet):
        """Traces, keeping the wavefield for a following :meth:`adjoint`."""
        e, s = self._model(eps_r, sigma)
        w = self._wavelet(wavelet)
        self._workspace(full=True)
        tr = torch.empty(self.trace_shape, dtype=torch.float32, device=self.device)
        rc = self.lib.gf_forward(self.ctx, e.data_ptr(), s.data_ptr(), w.data_ptr(), tr.data_ptr(),
                                 None, getattr(self, "_store_mode", _lib.GF_STORE_FULL),
                                 self._stream())
        self._last_wavelet = w  # the recomputation of a checkpointed adjoint reads it
        _lib.check(self.lib, self.ctx, rc)
        return tr

    def adjoint(self, eps_r, sigma, resid):
        """dL/deps_r, dL/dsigma for the trace cotangent ``resid`` of the last forward."""
        e, s = self._model(eps_r, sigma)
        r = _dev_f32(resid.contiguous(), self.trace_shape, "resid", self.device)
        ge = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        gs = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        rc = self.lib.gf_adjoint(self.ctx, e.data_ptr(), s.data_ptr(), r.data_ptr(), ge.data_ptr(),
                                 gs.data_ptr(), self._stream())
        _lib.check(self.lib, self.ctx, rc)
        return ge, gs


class TEMode:
    """An :class:`FDTD` context seen through the TE mode of one source polarisation (0: x,
    1: y): ``misfit`` and ``misfit_and_gradient`` have the TM signatures and run the TE
    calls, so that the FWI driver (:class:`~.fwi.FWI`, without a learned preconditioner)
    inverts the source component's traces.  Everything else is the context's."""

    def __init__(self, fdtd: FDTD, polarisation: int):
        if polarisation not in (0, 1):
            raise ValueError("polarisation must be 0 (x) or 1 (y)")
        self.fd = fdtd
        self.polarisation = polarisation

    def __getattr__(self, name):
        if name == "fd":
            raise AttributeError(name)
        return getattr(self.fd, name)

    def misfit(self, eps_r, sigma, wavelet, observed, out=None):
        return self.fd.misfit_te(eps_r, sigma, wavelet, observed, self.polarisation, out=out)

    def misfit_and_gradient(self, eps_r, sigma, wavelet, observed):
        return self.fd.misfit_and_gradient_te(eps_r, sigma, wavelet, observed, self.polarisation)

    def forward_model(self, eps_r, sigma, wavelet, illumination: bool = False):
        if illumination:
            raise ValueError("no TE illumination: the learned preconditioner is TM-only")
        return self.fd.forward_model_te(eps_r, sigma, wavelet,
                                        self.polarisation)[..., self.polarisation].contiguous()


class FDTDFunction(torch.autograd.Function):
    """traces = FDTDFunction.apply(eps_r, sigma, fdtd, wavelet); backward runs the adjoint."""

    @staticmethod
    def forward(ctx, eps_r, sigma, fdtd: FDTD, wavelet):
        tr = fdtd.forward(eps_r.detach(), sigma.detach(), wavelet)
        ctx.fdtd = fdtd
        ctx.save_for_backward(eps_r, sigma)
        return tr

    @staticmethod
    def backward(ctx, grad_traces):
        eps_r, sigma = ctx.saved_tensors
        ge, gs = ctx.fdtd.adjoint(eps_r.detach(), sigma.detach(), grad_traces.float())
        return ge, gs, None, None


def autotune(fdtd: FDTD, eps_r, sigma, wavelet, cache_path: str | None = None,
             probe_steps: int = 0) -> Tiling:
    """Pick the fastest tiling / kernel variant for this context's shape (cached on disk)."""
    e, s = fdtd._model(eps_r, sigma)
    w = fdtd._wavelet(wavelet)
    # the candidates' workspaces differ in size (per-tile counters): let the library hold its
    # own while it probes them
    _lib.check(fdtd.lib, fdtd.ctx, fdtd.lib.gf_set_workspace(fdtd.ctx, None, 0))
    fdtd._ws = None
    fdtd._ws_full = False
    path = cache_path.encode() if cache_path else None
    rc = fdtd.lib.gf_autotune(fdtd.ctx, e.data_ptr(), s.data_ptr(), w.data_ptr(), path,
                              probe_steps, fdtd._stream())
    _lib.check(fdtd.lib, fdtd.ctx, rc)
    fdtd._ws = None  # the chosen tiling may need another workspace size
    fdtd._ws_full = False
    return fdtd.tiling()


class FDTDBatch:
    """Many independent instances (possibly different grids, shots, nt) advanced together:
    mode 0 one after the other, 1 concurrently on one stream each, 2 as one CUDA graph of
    those streams, 3 the persistent multi-instance schedule (the instances' persistent passes
    merged into single cooperative launches; every instance on variant 3), 4 mode 3 as one
    CUDA graph."""

    def __init__(self, fdtds):
        self.fds = list(fdtds)
        self.lib = self.fds[0].lib
        self.device = self.fds[0].device
        arr = (ctypes.c_void_p * len(self.fds))(*[f.ctx.value for f in self.fds])
        b = ctypes.c_void_p()
        _lib.check(self.lib, None, self.lib.gf_batch_create(ctypes.byref(b), arr, len(self.fds)))
        self.batch = b
        self.J = torch.zeros(len(self.fds), dtype=torch.float64, device=self.device)
        self.ge = [torch.zeros(f.shape, dtype=torch.float32, device=self.device) for f in self.fds]
        self.gs = [torch.zeros(f.shape, dtype=torch.float32, device=self.device) for f in self.fds]

    def close(self):
        if getattr(self, "batch", None):
            self.lib.gf_batch_destroy(self.batch)
            self.batch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def misfit_and_gradient(self, eps_r, sigma, wavelet, observed, mode: int = 2):
        """Lists of per-instance device tensors in; (J [n], [g_eps_r], [g_sigma]) out.  The
        output tensors are reused by every call (a replayed graph writes the same buffers);
        pass the same input tensors to replay without re-capturing."""
        n = len(self.fds)
        ins = []
        for k, f in enumerate(self.fds):
            e, s = f._model(eps_r[k], sigma[k])
            w = f._wavelet(wavelet[k])
            o = _dev_f32(observed[k], f.trace_shape, "observed", f.device)
            f._workspace(full=True)
            ins.append((e, s, w, o))
        self._keep = ins  # the tensors must outlive the asynchronous (or replayed) work
        P = lambda xs: (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
        rc = self.lib.gf_batch_misfit_and_gradient(
            self.batch, P([x[0] for x in ins]), P([x[1] for x in ins]), P([x[2] for x in ins]),
            P([x[3] for x in ins]), self.J.data_ptr(), P(self.ge), P(self.gs), mode,
            torch.cuda.current_stream(self.device).cuda_stream)
        if rc != _lib.GF_OK:
            msg = self.lib.gf_batch_last_error(self.batch)
            raise _lib.GfError(rc, msg.decode() if msg else "")
        return self.J, self.ge, self.gs
