"""Shot sharding on the GPU: the round-robin shares of one acquisition, run one after the
other on one device, sum to the gradient of the whole acquisition (FP32 rounding of a
different summation order), which matches the FP64 oracle at the gradient tolerance; without
a process group the sharded object is the plain context."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2506_20513_gb300 import workloads as W  # noqa: E402

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


@pytest.mark.parametrize("world", [2, 3])
def test_shares_sum_to_the_whole_acquisition(dev, world):
    from paper_2506_20513_gb300 import FDTD
    from paper_2506_20513_gb300.shard import ShardedGradient
    wl = W.small_random(31, nxp=70, nyp=46, npml=8, nt=220, nshots=5, nrec=9)
    g = wl.grid
    wav = np.broadcast_to(O.ricker(wl.f0, g.dt, g.nt), (wl.nshots, 1, g.nt)).copy()
    obs = O.forward(g, wl.eps_true, wl.sig_true, wl.src, wav, wl.rec)
    e, s, w, o = (t32(a, dev) for a in (wl.eps_init, wl.sig_init, wav, obs))
    full = FDTD(g, wl.src, wl.rec, device=dev)
    J, ge, gs = (x.cpu().numpy() for x in full.misfit_and_gradient(e, s, w, o))
    full.close()
    Js, ges, gss = 0.0, 0.0, 0.0
    shots = []
    for r in range(world):
        sg = ShardedGradient(g, wl.src, wl.rec, device=dev, share=(r, world))
        Jr, ger, gsr = sg.local(e, s, w, o)
        sg.status()
        Js, ges, gss = Js + float(Jr[0]), ges + ger.cpu().numpy(), gss + gsr.cpu().numpy()
        shots += sg.shots.tolist()
        sg.close()
    assert sorted(shots) == list(range(wl.nshots))
    assert Js == pytest.approx(float(J[0]), rel=1e-9)
    assert rel(ges, ge) <= 1e-5 and rel(gss, gs) <= 1e-5
    J64, ge64, gs64 = O.misfit_and_gradient(g, wl.eps_init, wl.sig_init, wl.src, wav, wl.rec, obs)
    assert rel(ges, ge64) <= 1e-3 and rel(gss, gs64) <= 1e-3
    assert Js == pytest.approx(J64, rel=1e-4)


def test_without_a_process_group_it_is_the_plain_context(dev):
    from paper_2506_20513_gb300 import FDTD
    from paper_2506_20513_gb300.shard import ShardedGradient
    wl = W.small_random(32, nxp=50, nyp=40, npml=6, nt=150, nshots=3, nrec=6)
    g = wl.grid
    wav = np.broadcast_to(O.ricker(wl.f0, g.dt, g.nt), (wl.nshots, 1, g.nt)).copy()
    obs = O.forward(g, wl.eps_true, wl.sig_true, wl.src, wav, wl.rec)
    e, s, w, o = (t32(a, dev) for a in (wl.eps_init, wl.sig_init, wav, obs))
    fd = FDTD(g, wl.src, wl.rec, device=dev)
    sg = ShardedGradient(g, wl.src, wl.rec, device=dev)
    a = [x.cpu() for x in fd.misfit_and_gradient(e, s, w, o)]
    b = [x.cpu() for x in sg.misfit_and_gradient(e, s, w, o)]
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    assert float(sg.misfit(e, s, w, o)[0]) == pytest.approx(float(a[0][0]), rel=1e-6)
    fd.close()
    sg.close()
