"""gf_forward_model_noalloc: the forward model for callers that may not allocate device
memory (their memory belongs to another runtime or a fixed pool, or they run under a hard
budget).  It must give the same traces as gf_forward_model (to FP32 rounding: it has its own
tiling) while keeping all its working memory in the library's static device array.  Calls in
a row, the first on a larger grid with a thicker CPML, more shots and more receivers, check
that the array's leftover contents from the previous call do not leak into the next one.  A
call on a capturing stream is refused without breaking the capture.

This file is collected last on purpose, so a run that stops at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2506_20513_gb300 import _lib, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

TRACE_TOL = 1e-4  # the traces tolerance of the parity tests


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_forward_matches_forward_model_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_20513_gb300 import FDTD
    from paper_2506_20513_gb300 import build as B
    lib = _lib.load(B.build_library())
    dev = torch.device("cuda", 0)
    wl = W.small_random(41, nxp=130, nyp=70, npml=8, nt=300, nshots=3, nrec=9, with_pec=True)
    g = wl.grid
    gd = _lib.GridDesc(g.nx, g.ny, g.npml, g.nt, g.dx, g.dy, g.dt, g.pml_order, g.pml_sigma_max,
                       g.pml_kappa_max, g.pml_alpha_max, g.pml_eps_ref)
    src = np.ascontiguousarray(wl.src, dtype=np.int32)
    rec = np.ascontiguousarray(wl.rec, dtype=np.int32)
    acq = _lib.Acquisition(wl.nshots, 1, wl.nrec,
                           src.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                           rec.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    t32 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    wav = t32(np.broadcast_to(O.ricker(wl.f0, g.dt, g.nt), (wl.nshots, 1, g.nt)))
    fd = FDTD(g, wl.src, wl.rec, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    for eps, sig in ((wl.eps_true, wl.sig_true), (wl.eps_init, wl.sig_init)):
        e, s = t32(eps), t32(sig)
        ref = fd.forward_model(e, s, wav)
        out = torch.full((wl.nshots, g.nt, wl.nrec), float("nan"), device=dev)
        rc = lib.gf_forward_model_noalloc(ctypes.byref(gd), ctypes.byref(acq), 0, e.data_ptr(),
                                          s.data_ptr(), wav.data_ptr(), out.data_ptr(), stream)
        assert rc == _lib.GF_OK, lib.gf_last_error(None)
        torch.cuda.synchronize(dev)
        assert torch.isfinite(out).all()
        assert rel(out.cpu().numpy(), ref.cpu().numpy()) <= TRACE_TOL
    fd.close()


def _acq(wl):
    src = np.ascontiguousarray(wl.src, dtype=np.int32)
    rec = np.ascontiguousarray(wl.rec, dtype=np.int32)
    acq = _lib.Acquisition(wl.nshots, 1, wl.nrec,
                           src.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                           rec.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return acq, (src, rec)


def _gd(g):
    return _lib.GridDesc(g.nx, g.ny, g.npml, g.nt, g.dx, g.dy, g.dt, g.pml_order,
                         g.pml_sigma_max, g.pml_kappa_max, g.pml_alpha_max, g.pml_eps_ref)


def test_noalloc_after_a_larger_call():
    """A large call (thick CPML, 5 shots, 14 receivers, longer nt) leaves CPML strips,
    receiver lists and state in the array; the small call after it must not see them."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_20513_gb300 import FDTD
    from paper_2506_20513_gb300 import build as B
    lib = _lib.load(B.build_library())
    dev = torch.device("cuda", 0)
    t32 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    big = W.small_random(43, nxp=150, nyp=90, npml=14, nt=260, nshots=5, nrec=14)
    small = W.small_random(44, nxp=60, nyp=40, npml=5, nt=150, nshots=2, nrec=5,
                           with_pec=True)
    for wl in (big, small):
        g = wl.grid
        gd = _gd(g)
        acq, keep = _acq(wl)
        wav = t32(np.broadcast_to(O.ricker(wl.f0, g.dt, g.nt), (wl.nshots, 1, g.nt)))
        e, s = t32(wl.eps_true), t32(wl.sig_true)
        out = torch.full((wl.nshots, g.nt, wl.nrec), float("nan"), device=dev)
        rc = lib.gf_forward_model_noalloc(ctypes.byref(gd), ctypes.byref(acq), 0, e.data_ptr(),
                                          s.data_ptr(), wav.data_ptr(), out.data_ptr(), stream)
        assert rc == _lib.GF_OK, lib.gf_last_error(None)
        torch.cuda.synchronize(dev)
        fd = FDTD(g, wl.src, wl.rec, device=dev)
        ref = fd.forward_model(e, s, wav)
        fd.close()
        assert torch.isfinite(out).all()
        assert rel(out.cpu().numpy(), ref.cpu().numpy()) <= TRACE_TOL


def test_noalloc_refuses_a_capturing_stream():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_20513_gb300 import build as B
    lib = _lib.load(B.build_library())
    dev = torch.device("cuda", 0)
    wl = W.small_random(45, nxp=40, nyp=30, npml=5, nt=50, nshots=1, nrec=3)
    g = wl.grid
    gd = _gd(g)
    acq, keep = _acq(wl)
    x = torch.zeros(16, device=dev)
    buf = torch.zeros(g.nx * g.ny + g.nt, device=dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        x.add_(1.0)
        stream = torch.cuda.current_stream(dev).cuda_stream
        rc = lib.gf_forward_model_noalloc(ctypes.byref(gd), ctypes.byref(acq), 0, buf.data_ptr(),
                                          buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), stream)
    assert rc == _lib.GF_EINVAL
    assert b"capturing" in lib.gf_last_error(None)
    graph.replay()
    torch.cuda.synchronize(dev)
    assert float(x[0]) == 1.0   # the capture survived: the graph holds the add


def test_noalloc_rejects_oversized_problem():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_20513_gb300 import build as B
    lib = _lib.load(B.build_library())
    wl = W.multishot_layered(nshots=32, nt=10)
    g = wl.grid
    gd = _lib.GridDesc(g.nx, g.ny, g.npml, g.nt, g.dx, g.dy, g.dt, g.pml_order, g.pml_sigma_max,
                       g.pml_kappa_max, g.pml_alpha_max, g.pml_eps_ref)
    src = np.ascontiguousarray(wl.src, dtype=np.int32)
    rec = np.ascontiguousarray(wl.rec, dtype=np.int32)
    acq = _lib.Acquisition(wl.nshots, 1, wl.nrec,
                           src.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                           rec.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    dummy = torch.zeros(1, device="cuda")
    rc = lib.gf_forward_model_noalloc(ctypes.byref(gd), ctypes.byref(acq), 0, dummy.data_ptr(),
                                      dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), None)
    assert rc == _lib.GF_ENOMEM
    assert b"scratch" in lib.gf_last_error(None)
