"""Reverse-time reconstruction inside checkpoint segments (storage mode GF_STORE_RECONSTRUCT):
each segment's recomputation keeps only the boundary ring (CPML strips and two cells more)
per step, and the adjoint runs the Yee updates backwards from the segment's last state.  In
a nearly lossless medium this reproduces the checkpointed gradient to FP32 rounding and
matches the oracle; in lossy media the reversed E update divides by Ca < 1 every step, so the
error grows with the segment length k and the conductivity, as e^{sigma dt k / eps}: the
table of that growth is printed and its monotonicity checked."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2506_20513_gb300 import _lib, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_20513_gb300 import build as B
    B.build_library()
    return torch.device("cuda", 0)


def t32(a, dev):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _case(sig_max_mS, seed=70):
    wl = W.small_random(seed, nxp=70, nyp=50, npml=8, nt=300, nshots=2, nrec=9)
    scale = sig_max_mS * 1e-3 / float(wl.sig_true.max())
    return wl, wl.sig_true * scale, wl.sig_init * scale


def _gradients(wl, sig_t, sig_i, dev, storage):
    from paper_2506_20513_gb300 import FDTD
    g = wl.grid
    wav = np.broadcast_to(O.ricker(wl.f0, g.dt, g.nt), (wl.nshots, 1, g.nt)).copy()
    fd = FDTD(g, wl.src, wl.rec, device=dev)
    obs = fd.forward_model(t32(wl.eps_true, dev), t32(sig_t, dev), t32(wav, dev))
    fd.set_storage(*storage)
    J, ge, gs = fd.misfit_and_gradient(t32(wl.eps_init, dev), t32(sig_i, dev), t32(wav, dev), obs)
    try:
        fd.status()
        out = float(J.item()), ge.cpu().numpy(), gs.cpu().numpy()
    except _lib.GfError as e:  # the reversed updates overflowed: the gradient is lost
        assert e.code == _lib.GF_ENONFINITE
        nan = np.full(fd.shape, np.nan)
        out = float(J.item()), nan, nan
    fd.close()
    return out, wav, obs.cpu().numpy()


@pytest.mark.parametrize("k", [1, 17, 60])
def test_reconstruction_in_a_nearly_lossless_medium(dev, k):
    wl, sig_t, sig_i = _case(0.05)
    (J, ge, gs), wav, obs = _gradients(wl, sig_t, sig_i, dev, (k, True))
    (Jc, gec, gsc), _, _ = _gradients(wl, sig_t, sig_i, dev, (k, False))
    assert J == Jc  # the forward pass is the same
    assert rel(ge, gec) <= 1e-4 and rel(gs, gsc) <= 1e-4
    J64, ge64, gs64 = O.misfit_and_gradient(wl.grid, wl.eps_init, sig_i, wl.src, wav, wl.rec, obs)
    assert rel(ge, ge64) <= 1e-3 and rel(gs, gs64) <= 1e-3


def test_reconstruction_error_grows_with_k_and_sigma(dev):
    """The reversed E update divides by Ca every step (1 / Ca = 1 + sigma dt / eps, about
    1.007 at 10 mS/m, 1.14 at 200 mS/m and 2 at 1 S/m on this grid: dt 42 ps, eps_r 3-12):
    rounding errors grow backwards through a segment wherever the true field does not grow
    with them.  Measured: up to 200 mS/m and k = 150 the gradient stays at FP32 rounding
    (about 2e-7); at 1 S/m it is 1.8e-7 at k = 10, 1.5e-6 at k = 40 and lost (overflow or
    1e7) at k = 150."""
    rows = {}
    for sig_max in (10.0, 200.0, 1000.0):
        wl, sig_t, sig_i = _case(sig_max)
        (_, gec, gsc), _, _ = _gradients(wl, sig_t, sig_i, dev, (300, False))
        for k in (10, 40, 150):
            (_, ge, gs), _, _ = _gradients(wl, sig_t, sig_i, dev, (k, True))
            rows[(sig_max, k)] = max(rel(ge, gec), rel(gs, gsc)) if np.isfinite(ge).all() \
                and np.isfinite(gs).all() else float("inf")
    print("\nsigma_max (mS/m), k, max rel-L2 gradient error vs checkpointing")
    for key, v in sorted(rows.items()):
        print(f"{key[0]:7.1f} {key[1]:4d} {v:.3e}")
    for sig_max in (10.0, 200.0):
        for k in (10, 40, 150):
            assert rows[(sig_max, k)] <= 1e-5
    assert rows[(1000.0, 10)] <= 1e-5
    assert rows[(1000.0, 40)] > 3 * rows[(1000.0, 10)]
    assert rows[(1000.0, 150)] > 1e-2
