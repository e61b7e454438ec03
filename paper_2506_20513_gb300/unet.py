"""U-Net of the learned gradient preconditioner (binding of include/gprfwi_unet.h).

Argument marshalling only: forward, loss, backward and Adam run in the library's BF16
tensor-core kernels.  Tensors are channels-last FP32 on the network's device:
x [n, H, W, cin], y and targets [n, H, W, cout], masks [n, H, W].
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib


class UNet:
    def __init__(self, levels: int = 4, base: int = 32, cin: int = 4, cout: int = 2,
                 height: int = 128, width: int = 256, max_batch: int = 16, device=None,
                 lib_path: str | None = None):
        self.lib = _lib.load(lib_path)
        self.device = torch.device(device if device is not None else "cuda:0")
        if self.device.type != "cuda":
            raise ValueError("the U-Net runs on a CUDA device")
        self.desc = _lib.UNetDesc(levels, base, cin, cout, height, width, max_batch)
        self.levels, self.base, self.cin, self.cout = levels, base, cin, cout
        self.height, self.width, self.max_batch = height, width, max_batch
        n = self.lib.gf_unet_param_count(ctypes.byref(self.desc))
        if n < 0:
            raise _lib.GfError(_lib.GF_EINVAL, "invalid U-Net description")
        self.param_count = int(n)
        self._net = ctypes.c_void_p()
        idx = self.device.index if self.device.index is not None else torch.cuda.current_device()
        self._check(self.lib.gf_unet_create(ctypes.byref(self._net), ctypes.byref(self.desc),
                                            idx), None)
        self._loss = torch.zeros(1, dtype=torch.float64, device=self.device)

    def _check(self, rc, net):
        _lib.check(self.lib, net, rc, self.lib.gf_unet_last_error)

    def _stream(self):
        return torch.cuda.current_stream(self.device).cuda_stream

    def close(self):
        if getattr(self, "_net", None) and self._net.value:
            torch.cuda.synchronize(self.device)
            self.lib.gf_unet_destroy(self._net)
            self._net = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- parameters ------------------------------------------------------------------------
    def init_params(self, seed: int) -> torch.Tensor:
        """He-normal weights (std sqrt(2 / fan_in)), biases N(0, 0.01^2), drawn on the host
        from a seeded generator, uploaded and set."""
        rng = np.random.default_rng(seed)
        c = [self.base * 2 ** l for l in range(self.levels)]
        shapes = []
        ci = self.cin
        for l in range(self.levels):
            shapes += [(3, ci, c[l]), (3, c[l], c[l])]
            ci = c[l]
        for l in range(self.levels - 2, -1, -1):
            shapes += [(3, c[l + 1] + c[l], c[l]), (3, c[l], c[l])]
        shapes.append((1, c[0], self.cout))
        parts = []
        for k, ci, co in shapes:
            parts.append(rng.standard_normal(k * k * ci * co) * np.sqrt(2.0 / (k * k * ci)))
            parts.append(0.01 * rng.standard_normal(co))
        p = torch.from_numpy(np.concatenate(parts).astype(np.float32)).to(self.device)
        assert p.numel() == self.param_count
        self.set_params(p)
        return p

    def set_params(self, params: torch.Tensor):
        p = self._vec(params, self.param_count, "params")
        self._check(self.lib.gf_unet_set_params(self._net, p.data_ptr(), self._stream()),
                    self._net)
        self._keep = p

    def get_params(self) -> torch.Tensor:
        out = torch.empty(self.param_count, dtype=torch.float32, device=self.device)
        self._check(self.lib.gf_unet_get_params(self._net, out.data_ptr(), self._stream()),
                    self._net)
        return out

    # -- compute ---------------------------------------------------------------------------
    def _vec(self, t, n, name):
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or t.device != self.device \
                or not t.is_contiguous() or t.numel() != n:
            raise ValueError(f"{name} must be a contiguous float32 tensor of {n} values on "
                             f"{self.device}")
        return t

    def _images(self, t, c, name):
        if t.dim() != 4 or tuple(t.shape[1:]) != (self.height, self.width, c):
            raise ValueError(f"{name} must be [n, {self.height}, {self.width}, {c}]")
        n = t.shape[0]
        if not 1 <= n <= self.max_batch:
            raise ValueError(f"{name}: n = {n} outside 1..{self.max_batch}")
        return self._vec(t, t.numel(), name)

    def forward(self, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        x = self._images(x, self.cin, "x")
        n = x.shape[0]
        y = out if out is not None else torch.empty(n, self.height, self.width, self.cout,
                                                    dtype=torch.float32, device=self.device)
        self._images(y, self.cout, "y")
        self._check(self.lib.gf_unet_forward(self._net, n, x.data_ptr(), y.data_ptr(),
                                             self._stream()), self._net)
        return y

    __call__ = forward

    def loss_and_grad(self, x, target, mask=None, grads: bool = False):
        """(loss as a device FP64 tensor [1], parameter gradient or None)."""
        x = self._images(x, self.cin, "x")
        n = x.shape[0]
        t = self._images(target, self.cout, "target")
        if t.shape[0] != n:
            raise ValueError("x and target hold different numbers of images")
        mp = 0
        if mask is not None:
            m = self._vec(mask, n * self.height * self.width, "mask")
            mp = m.data_ptr()
        g = torch.empty(self.param_count, dtype=torch.float32, device=self.device) if grads \
            else None
        self._check(self.lib.gf_unet_loss_and_grad(self._net, n, x.data_ptr(), t.data_ptr(), mp,
                                                   self._loss.data_ptr(),
                                                   g.data_ptr() if g is not None else None,
                                                   self._stream()), self._net)
        return self._loss, g

    def adam_step(self, lr: float, beta1: float = 0.9, beta2: float = 0.999,
                  eps: float = 1e-8):
        self._check(self.lib.gf_unet_adam_step(self._net, lr, beta1, beta2, eps,
                                               self._stream()), self._net)

    def train_step(self, x, target, mask=None, lr: float = 1e-3):
        loss, _ = self.loss_and_grad(x, target, mask)
        self.adam_step(lr)
        return loss

    @property
    def kernel_launches(self) -> int:
        return int(self.lib.gf_unet_kernel_launches(self._net))

    def set_gemm(self, mode: int):
        """1: tcgen05 with TMA-loaded operands (default); 2: tcgen05 with thread-staged
        operands; 0: mma.sync only."""
        self._check(self.lib.gf_unet_set_gemm(self._net, int(mode)), self._net)

    def set_wait_budget(self, polls: int):
        """Failure-path hook: polls per tensor-core GEMM wait (0 = built-in limit)."""
        self._check(self.lib.gf_unet_set_wait_budget(self._net, int(polls)), self._net)

    def status(self):
        """Synchronise and raise if a tensor-core GEMM gave up waiting (outputs invalid)."""
        self._check(self.lib.gf_unet_status(self._net, self._stream()), self._net)

    def profile(self, enable: bool = True):
        """Bracket every GEMM launch with CUDA events (see :meth:`profile_read`)."""
        self._check(self.lib.gf_unet_profile(self._net, int(enable)), self._net)

    def profile_read(self):
        """(GEMM milliseconds, GEMM launches, algorithmic FLOPs) since the last read."""
        ms, n, fl = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double()
        self._check(self.lib.gf_unet_profile_read(self._net, ctypes.byref(ms), ctypes.byref(n),
                                                  ctypes.byref(fl)), self._net)
        return ms.value, n.value, fl.value
