"""ctypes binding of ``include/gprfwi.h`` and ``include/gprfwi_unet.h``: the C ABI under the
same names.

Argument marshalling only.  Array arguments are integer addresses (device pointers from
``torch.Tensor.data_ptr()``); ``stream`` is a ``cudaStream_t`` as an integer.  Every compute
step runs in the CUDA kernels of ``libgprfwi.so``; this module never computes anything and
raises if the library is missing.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_LIB = os.path.join(_HERE, "_build", "libgprfwi.so")

GF_OK = 0
GF_EINVAL = -1
GF_ECFL = -2
GF_ENOMEM = -3
GF_ECUDA = -4
GF_ENONFINITE = -5
GF_ETIMEOUT = -6
GF_ESTATE = -7
GF_STORE_FULL = 0
GF_STORE_CHECKPOINT = 1
GF_STORE_RECONSTRUCT = 2

ERROR_NAMES = {
    GF_EINVAL: "GF_EINVAL", GF_ECFL: "GF_ECFL", GF_ENOMEM: "GF_ENOMEM", GF_ECUDA: "GF_ECUDA",
    GF_ENONFINITE: "GF_ENONFINITE", GF_ETIMEOUT: "GF_ETIMEOUT", GF_ESTATE: "GF_ESTATE",
}

# Every entry point declared in include/gprfwi.h and include/gprfwi_unet.h.
EXPORTS = (
    "gf_create", "gf_destroy", "gf_last_error", "gf_workspace_size", "gf_set_workspace",
    "gf_set_tiling", "gf_set_variant", "gf_set_storage", "gf_get_tiling", "gf_forward_model", "gf_forward_model_fields", "gf_forward_model_te", "gf_misfit_and_gradient_te", "gf_misfit_te", "gf_forward", "gf_adjoint", "gf_misfit_and_gradient",
    "gf_status", "gf_ricker", "gf_version", "gf_kernel_launches", "gf_set_wait_budget", "gf_set_lanes", "gf_profile",
    "gf_profile_read", "gf_profile_read_span", "gf_forward_model_noalloc", "gf_misfit", "gf_tv_scratch_bytes",
    "gf_tv_gradient", "gf_adam_update", "gf_autotune", "gf_batch_create", "gf_batch_destroy",
    "gf_batch_last_error", "gf_batch_misfit_and_gradient",
    "gf_unet_param_count", "gf_unet_create", "gf_unet_destroy", "gf_unet_last_error",
    "gf_unet_set_params", "gf_unet_get_params", "gf_unet_forward", "gf_unet_loss_and_grad",
    "gf_unet_adam_step", "gf_unet_kernel_launches", "gf_unet_profile", "gf_unet_profile_read",
    "gf_unet_set_gemm", "gf_unet_status", "gf_unet_set_wait_budget",
)
GF_KERNEL_FWD = 0
GF_KERNEL_ADJ = 1
GF_KERNEL_AUX = 2


class GridDesc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("npml", ctypes.c_int32),
        ("nt", ctypes.c_int32), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
        ("dt", ctypes.c_double), ("pml_order", ctypes.c_int32),
        ("pml_sigma_max", ctypes.c_double), ("pml_kappa_max", ctypes.c_double),
        ("pml_alpha_max", ctypes.c_double), ("pml_eps_ref", ctypes.c_double),
    ]


class Acquisition(ctypes.Structure):
    _fields_ = [
        ("nshots", ctypes.c_int32), ("nsrc", ctypes.c_int32), ("nrec", ctypes.c_int32),
        ("src_ij", ctypes.POINTER(ctypes.c_int32)), ("rec_ij", ctypes.POINTER(ctypes.c_int32)),
    ]


class UNetDesc(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("levels", "base", "cin", "cout", "height", "width", "max_batch")]


class GfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lock = threading.Lock()
_libs: dict = {}


def load(path: str | None = None) -> ctypes.CDLL:
    """Load (once) and declare the library at ``path`` (default: the in-tree build)."""
    path = os.path.abspath(path or DEFAULT_LIB)
    with _lock:
        if path in _libs:
            return _libs[path]
        if not os.path.exists(path):
            raise ImportError(
                f"libgprfwi.so not found at {path}: build it first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(path)
        vp, i, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        P = ctypes.POINTER
        decl = {
            "gf_create": (i, [P(vp), P(GridDesc), P(Acquisition), i]),
            "gf_destroy": (None, [vp]),
            "gf_last_error": (ctypes.c_char_p, [vp]),
            "gf_workspace_size": (i, [vp, i, i, P(sz)]),
            "gf_set_workspace": (i, [vp, vp, sz]),
            "gf_set_tiling": (i, [vp, i, i, i]),
            "gf_set_variant": (i, [vp, i]),
            "gf_set_storage": (i, [vp, i, i]),
            "gf_get_tiling": (i, [vp, P(i), P(i), P(i), P(i)]),
            "gf_forward_model": (i, [vp, vp, vp, vp, vp, vp, vp]),
            "gf_forward_model_fields": (i, [vp, vp, vp, vp, vp, vp, vp, vp]),
            "gf_forward_model_te": (i, [vp, vp, vp, vp, i, vp, vp]),
            "gf_misfit_and_gradient_te": (i, [vp, vp, vp, vp, i, vp, vp, vp, vp, vp, vp]),
            "gf_misfit_te": (i, [vp, vp, vp, vp, i, vp, vp, vp]),
            "gf_forward": (i, [vp, vp, vp, vp, vp, vp, i, vp]),
            "gf_adjoint": (i, [vp, vp, vp, vp, vp, vp, vp]),
            "gf_misfit_and_gradient": (i, [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
            "gf_status": (i, [vp, vp]),
            "gf_ricker": (i, [P(ctypes.c_float), i, ctypes.c_double, ctypes.c_double,
                              ctypes.c_double]),
            "gf_version": (ctypes.c_char_p, []),
            "gf_kernel_launches": (ctypes.c_longlong, [vp]),
            "gf_set_wait_budget": (i, [vp, ctypes.c_longlong]),
            "gf_set_lanes": (i, [vp, i]),
            "gf_profile": (i, [vp, i]),
            "gf_profile_read": (i, [vp, i, P(ctypes.c_double), P(ctypes.c_longlong)]),
            "gf_profile_read_span": (i, [vp, i, P(ctypes.c_double), P(ctypes.c_double),
                                         P(ctypes.c_longlong)]),
            "gf_misfit": (i, [vp, vp, vp, vp, vp, vp, vp]),
            "gf_tv_scratch_bytes": (sz, [i, i]),
            "gf_tv_gradient": (i, [i, i, vp, vp, vp, ctypes.c_float, ctypes.c_float, i,
                                   ctypes.c_float, vp]),
            "gf_adam_update": (i, [ctypes.c_longlong, vp, vp, vp, vp, vp] + [ctypes.c_float] * 5
                               + [i, ctypes.c_float, vp]),
            "gf_autotune": (i, [vp, vp, vp, vp, ctypes.c_char_p, i, vp]),
            "gf_batch_create": (i, [P(vp), P(vp), i]),
            "gf_batch_destroy": (None, [vp]),
            "gf_batch_last_error": (ctypes.c_char_p, [vp]),
            "gf_batch_misfit_and_gradient": (i, [vp, P(vp), P(vp), P(vp), P(vp), vp, P(vp), P(vp),
                                                 i, vp]),
            "gf_forward_model_noalloc": (i, [P(GridDesc), P(Acquisition), i, vp, vp, vp, vp,
                                             vp]),
            "gf_unet_param_count": (ctypes.c_longlong, [P(UNetDesc)]),
            "gf_unet_create": (i, [P(vp), P(UNetDesc), i]),
            "gf_unet_destroy": (None, [vp]),
            "gf_unet_last_error": (ctypes.c_char_p, [vp]),
            "gf_unet_set_params": (i, [vp, vp, vp]),
            "gf_unet_get_params": (i, [vp, vp, vp]),
            "gf_unet_forward": (i, [vp, i, vp, vp, vp]),
            "gf_unet_loss_and_grad": (i, [vp, i, vp, vp, vp, vp, vp, vp]),
            "gf_unet_adam_step": (i, [vp, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                      ctypes.c_float, vp]),
            "gf_unet_kernel_launches": (ctypes.c_longlong, [vp]),
            "gf_unet_profile": (i, [vp, i]),
            "gf_unet_set_gemm": (i, [vp, i]),
            "gf_unet_status": (i, [vp, vp]),
            "gf_unet_set_wait_budget": (i, [vp, ctypes.c_uint]),
            "gf_unet_profile_read": (i, [vp, P(ctypes.c_double), P(ctypes.c_longlong),
                                         P(ctypes.c_double)]),
        }
        for name, (res, args) in decl.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _libs[path] = lib
        return lib


def check(lib, ctx, rc: int, last_error=None) -> None:
    if rc != GF_OK:
        msg = (last_error or lib.gf_last_error)(ctx)
        raise GfError(rc, msg.decode() if msg else "")
