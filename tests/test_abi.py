"""C-ABI checks that need no GPU: the library loads, exports every symbol that
include/gprfwi.h declares, and its host-side validation and helpers behave (no compute)."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_2506_20513_gb300 import _lib, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in ("gprfwi.h", "gprfwi_unet.h")]


@pytest.fixture(scope="module")
def lib():
    from paper_2506_20513_gb300 import build as B
    return _lib.load(B.build_library())


def header_symbols():
    text = "".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gf_[a-z_]+)\s*\(", text)))


def test_header_declares_what_binding_lists():
    assert header_symbols() == sorted(_lib.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in header_symbols():
        assert hasattr(lib, name), name
    assert lib.gf_version().startswith(b"gprfwi-gb300")


def _create(lib, g, src, rec, nshots=1):
    gd = _lib.GridDesc(g.nx, g.ny, g.npml, g.nt, g.dx, g.dy, g.dt, g.pml_order, g.pml_sigma_max,
                       g.pml_kappa_max, g.pml_alpha_max, g.pml_eps_ref)
    src = np.ascontiguousarray(src, dtype=np.int32)
    rec = np.ascontiguousarray(rec, dtype=np.int32)
    acq = _lib.Acquisition(nshots, src.shape[1], rec.shape[1],
                           src.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                           rec.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    ctx = ctypes.c_void_p()
    rc = lib.gf_create(ctypes.byref(ctx), ctypes.byref(gd), ctypes.byref(acq), 0)
    if rc == 0:
        lib.gf_destroy(ctx)
    else:
        assert not ctx.value
    return rc


def test_create_rejects_cfl_violation(lib):
    g = W.GridSpec(nx=40, ny=30, npml=5, nt=10, dx=0.01, dy=0.01, dt=1.001 * W.cfl_dt_max(0.01, 0.01))
    assert _create(lib, g, [[[10, 10]]], [[[20, 12]]]) == _lib.GF_ECFL


@pytest.mark.parametrize("src,rec", [
    ([[[0, 10]]], [[[20, 12]]]),     # source on the PEC ring
    ([[[10, 10]]], [[[39, 12]]]),    # receiver on the PEC ring
    ([[[10, 30]]], [[[20, 12]]]),    # outside the grid
    ([[[10, 10]] * 9], [[[20, 12]]]),  # more than 8 sources per shot
])
def test_create_rejects_bad_geometry(lib, src, rec):
    g = W.GridSpec(nx=40, ny=30, npml=5, nt=10, dx=0.01, dy=0.01, dt=0.9 * W.cfl_dt_max(0.01, 0.01))
    assert _create(lib, g, src, rec) == _lib.GF_EINVAL


def test_create_rejects_bad_grid(lib):
    ok = dict(nx=40, ny=30, npml=5, nt=10, dx=0.01, dy=0.01, dt=1e-12)
    for bad in (dict(nt=0), dict(npml=15), dict(dx=0.0), dict(nx=2), dict(pml_kappa_max=0.5)):
        g = W.GridSpec(**{**ok, **bad})
        assert _create(lib, g, [[[10, 10]]], [[[20, 12]]]) == _lib.GF_EINVAL, bad


def test_null_arguments_are_rejected(lib):
    assert lib.gf_create(None, None, None, 0) == _lib.GF_EINVAL
    assert lib.gf_forward_model(None, None, None, None, None, None, None) == _lib.GF_EINVAL
    assert lib.gf_status(None, None) == _lib.GF_EINVAL
    lib.gf_destroy(None)
    assert lib.gf_last_error(None)
    assert lib.gf_batch_create(None, None, 0) == _lib.GF_EINVAL
    assert lib.gf_autotune(None, None, None, None, None, 0, None) == _lib.GF_EINVAL
    assert lib.gf_batch_misfit_and_gradient(None, None, None, None, None, None, None, None, 0,
                                            None) == _lib.GF_EINVAL
    lib.gf_batch_destroy(None)


def test_ricker_helper_closed_form(lib):
    """The host helper follows the Ricker closed form: peak at t0 = sqrt(2)/f0, zeros at
    t0 +- 1/(sqrt(2) pi f0)."""
    from paper_2506_20513_gb300.fdtd import ricker
    f0, dt, nt = 250e6, 1e-12, 20000
    w = ricker(f0, dt, nt, amp=3.0)
    t0 = math.sqrt(2) / f0
    assert w[int(round(t0 / dt))] == pytest.approx(3.0, rel=1e-6)
    nz = int((t0 + 1 / (math.sqrt(2) * math.pi * f0)) / dt)
    assert w[nz] > 0 > w[nz + 1]
    n = np.arange(nt) * dt - t0
    z = (math.pi * f0 * n) ** 2
    np.testing.assert_allclose(w, 3.0 * (1 - 2 * z) * np.exp(-z), rtol=0, atol=3e-6)


def _unet_desc(**kw):
    d = dict(levels=4, base=32, cin=4, cout=2, height=128, width=256, max_batch=16)
    d.update(kw)
    return _lib.UNetDesc(**d)


def test_unet_param_count_matches_oracle(lib):
    from oracle import unet_oracle as U
    for lv, b, ci, co in ((4, 32, 4, 2), (3, 8, 3, 5), (1, 16, 1, 1), (6, 8, 64, 64)):
        d = _unet_desc(levels=lv, base=b, cin=ci, cout=co, height=64, width=64, max_batch=1)
        assert lib.gf_unet_param_count(ctypes.byref(d)) == U.param_count(lv, b, ci, co)


@pytest.mark.parametrize("bad", [dict(levels=0), dict(levels=7), dict(base=12), dict(base=4),
                                 dict(base=64, levels=6), dict(cin=0), dict(cout=65),
                                 dict(height=100), dict(width=0), dict(max_batch=0),
                                 dict(max_batch=300)])
def test_unet_create_rejects_invalid_desc(lib, bad):
    d = _unet_desc(**bad)
    assert lib.gf_unet_param_count(ctypes.byref(d)) == -1
    net = ctypes.c_void_p()
    assert lib.gf_unet_create(ctypes.byref(net), ctypes.byref(d), 0) == _lib.GF_EINVAL
    assert not net.value
    assert lib.gf_unet_last_error(None)


def test_unet_null_arguments(lib):
    assert lib.gf_unet_create(None, None, 0) == _lib.GF_EINVAL
    assert lib.gf_unet_param_count(None) == -1
    assert lib.gf_unet_forward(None, 1, None, None, None) == _lib.GF_EINVAL
    assert lib.gf_unet_loss_and_grad(None, 1, None, None, None, None, None, None) == _lib.GF_EINVAL
    assert lib.gf_unet_adam_step(None, 1e-3, 0.9, 0.999, 1e-8, None) == _lib.GF_EINVAL
    assert lib.gf_unet_set_params(None, None, None) == _lib.GF_EINVAL
    assert lib.gf_unet_kernel_launches(None) == 0
    lib.gf_unet_destroy(None)


def test_create_rejects_empty_acquisitions(lib):
    """No shots, no sources or no receivers: GF_EINVAL before anything touches a device."""
    g = W.GridSpec(nx=40, ny=30, npml=5, nt=10, dx=0.01, dy=0.01, dt=0.9 * W.cfl_dt_max(0.01, 0.01))
    assert _create(lib, g, np.zeros((0, 1, 2)), np.zeros((0, 1, 2)), nshots=0) == _lib.GF_EINVAL
    assert _create(lib, g, [[[10, 10]]], np.zeros((1, 0, 2))) == _lib.GF_EINVAL
    assert _create(lib, g, np.zeros((1, 0, 2)), [[[20, 12]]]) == _lib.GF_EINVAL
