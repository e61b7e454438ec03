"""Uneven-instance batches (sequential, concurrent, CUDA graph) and the autotuner."""
import os

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


def _instances():
    # nt long enough that the 300 MHz Ricker (delay sqrt(2)/f0 = 4.7 ns) reaches receivers
    return [W.small_random(60, nxp=40, nyp=30, npml=5, nt=220, nshots=2, nrec=5),
            W.small_random(61, nxp=70, nyp=36, npml=6, nt=273, nshots=3, nrec=7, with_pec=True),
            W.small_random(62, nxp=52, nyp=61, npml=4, nt=251, nshots=1, nrec=4, kappa_max=2.0)]


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_batch_matches_single_instances_and_oracle(dev, mode):
    from paper_2506_20513_gb300 import FDTD, FDTDBatch
    wls = _instances()
    fds, args = [], []
    for k, wl in enumerate(wls):
        g = wl.grid
        fd = FDTD(g, wl.src, wl.rec, device=dev)
        if k == 1:
            fd.set_storage(30)  # one checkpointed instance in the batch
        wav = np.broadcast_to(O.ricker(wl.f0, g.dt, g.nt), (wl.nshots, 1, g.nt))
        obs = O.forward(g, wl.eps_true, wl.sig_true, wl.src, wav, wl.rec)
        args.append((t32(wl.eps_init, dev), t32(wl.sig_init, dev), t32(wav, dev), t32(obs, dev),
                     wav, obs))
        fds.append(fd)
    singles = [fd.misfit_and_gradient(*a[:4]) for fd, a in zip(fds, args)]
    batch = FDTDBatch(fds)
    for rep in range(2):  # the graph is captured on the first call, replayed on the second
        J, ge, gs = batch.misfit_and_gradient([a[0] for a in args], [a[1] for a in args],
                                              [a[2] for a in args], [a[3] for a in args], mode)
        torch.cuda.synchronize(dev)
        for k, (Js, ges, gss) in enumerate(singles):
            assert J[k].item() == Js.item()
            assert torch.equal(ge[k], ges) and torch.equal(gs[k], gss)
    for k, (wl, a) in enumerate(zip(wls, args)):
        J64, ge64, gs64 = O.misfit_and_gradient(wl.grid, wl.eps_init, wl.sig_init, wl.src, a[4],
                                                wl.rec, a[5])
        assert J64 > 1e-6  # the case carries signal
        rel = lambda x, y: np.linalg.norm(x.cpu().numpy() - y) / np.linalg.norm(y)
        assert rel(ge[k], ge64) <= 1e-3 and rel(gs[k], gs64) <= 1e-3
    batch.close()


def test_graph_replay_sees_new_input_values(dev):
    """Replaying the captured graph with new values in the same buffers recomputes."""
    from paper_2506_20513_gb300 import FDTD, FDTDBatch
    wls = _instances()[:2]
    fds = [FDTD(wl.grid, wl.src, wl.rec, device=dev) for wl in wls]
    ins = []
    for wl in wls:
        g = wl.grid
        wav = np.broadcast_to(O.ricker(wl.f0, g.dt, g.nt), (wl.nshots, 1, g.nt))
        obs = O.forward(g, wl.eps_true, wl.sig_true, wl.src, wav, wl.rec)
        ins.append([t32(wl.eps_init, dev), t32(wl.sig_init, dev), t32(wav, dev), t32(obs, dev)])
    batch = FDTDBatch(fds)
    J1 = batch.misfit_and_gradient(*[list(x) for x in zip(*ins)], mode=2)[0].clone()
    for x in ins:
        x[0].mul_(1.05)  # same tensors, new values
    J2, ge, gs = batch.misfit_and_gradient(*[list(x) for x in zip(*ins)], mode=2)
    torch.cuda.synchronize(dev)
    for k, fd in enumerate(fds):
        Jr, ger, gsr = fd.misfit_and_gradient(*ins[k])
        assert J2[k].item() == Jr.item() != J1[k].item()
        assert torch.equal(ge[k], ger)
    batch.close()


def test_autotune_picks_a_valid_tiling_and_caches_it(dev, tmp_path):
    from paper_2506_20513_gb300 import FDTD, autotune
    wl = W.small_random(63, nxp=120, nyp=80, npml=8, nt=100, nshots=2, nrec=6)
    g = wl.grid
    fd = FDTD(g, wl.src, wl.rec, device=dev)
    wav = t32(np.broadcast_to(O.ricker(wl.f0, g.dt, g.nt), (2, 1, g.nt)), dev)
    cache = str(tmp_path / "tune.txt")
    t1 = autotune(fd, t32(wl.eps_init, dev), t32(wl.sig_init, dev), wav, cache, probe_steps=24)
    assert os.path.exists(cache) and "nx=%d" % g.nx in open(cache).read()
    # staged window: 64 x 64 (variants 0, 2) or 64 x 32 (variant 1); even tile widths behind
    # a left halo of the steps rounded up to even
    kl = t1.steps + (t1.steps & 1)
    assert t1.steps >= 1 and t1.tile_w % 2 == 0 and kl + t1.tile_w + t1.steps <= 64
    assert t1.variant in (0, 1, 2)
    assert t1.tile_h + 2 * t1.steps <= (32 if t1.variant == 1 else 64)
    fd2 = FDTD(g, wl.src, wl.rec, device=dev)
    t2 = autotune(fd2, t32(wl.eps_init, dev), t32(wl.sig_init, dev), wav, cache, probe_steps=24)
    assert t2 == t1
    # the tuned context still computes the right gradient
    obs = O.forward(g, wl.eps_true, wl.sig_true, wl.src, wav.cpu().double().numpy(), wl.rec)
    J, ge, gs = fd2.misfit_and_gradient(t32(wl.eps_init, dev), t32(wl.sig_init, dev), wav,
                                        t32(obs, dev))
    J64, ge64, gs64 = O.misfit_and_gradient(g, wl.eps_init, wl.sig_init, wl.src,
                                            wav.cpu().double().numpy(), wl.rec, obs)
    assert np.linalg.norm(ge.cpu().numpy() - ge64) <= 1e-3 * np.linalg.norm(ge64)


def _flow_batch(dev, ks=(4, 6, 7)):
    from paper_2506_20513_gb300 import FDTD, Tiling
    wls = _instances()
    fds, args = [], []
    for k, wl in enumerate(wls):
        g = wl.grid
        fd = FDTD(g, wl.src, wl.rec, device=dev, tiling=Tiling(0, 0, ks[k], 3))
        if k == 1:
            fd.set_storage(30)  # one checkpointed instance in the batch
        wav = np.broadcast_to(O.ricker(wl.f0, g.dt, g.nt), (wl.nshots, 1, g.nt))
        obs = O.forward(g, wl.eps_true, wl.sig_true, wl.src, wav, wl.rec)
        args.append((t32(wl.eps_init, dev), t32(wl.sig_init, dev), t32(wav, dev), t32(obs, dev),
                     wav, obs))
        fds.append(fd)
    return wls, fds, args


@pytest.mark.parametrize("mode", [3, 4])
def test_persistent_batch_matches_single_instances_and_oracle(dev, mode):
    """Modes 3 and 4 merge the instances' persistent passes (different grids, shots, nt and
    time-block depths; one instance checkpointed, so its segment passes meet the others' full
    passes) into single cooperative launches: every gradient is bit-identical to the
    instance's own run (the per-item arithmetic and the per-cell summation order do not depend
    on which CTA runs an item) and matches the oracle."""
    from paper_2506_20513_gb300 import FDTDBatch
    wls, fds, args = _flow_batch(dev)
    singles = [fd.misfit_and_gradient(*a[:4]) for fd, a in zip(fds, args)]
    for fd in fds:
        fd.status()
    batch = FDTDBatch(fds)
    for rep in range(2):  # recorded on the first call, kept (and replayed) on the second
        J, ge, gs = batch.misfit_and_gradient([a[0] for a in args], [a[1] for a in args],
                                              [a[2] for a in args], [a[3] for a in args], mode)
        torch.cuda.synchronize(dev)
        for fd in fds:
            fd.status()
        for k, (Js, ges, gss) in enumerate(singles):
            assert J[k].item() == Js.item()
            assert torch.equal(ge[k], ges) and torch.equal(gs[k], gss)
    for k, (wl, a) in enumerate(zip(wls, args)):
        J64, ge64, gs64 = O.misfit_and_gradient(wl.grid, wl.eps_init, wl.sig_init, wl.src, a[4],
                                                wl.rec, a[5])
        rel = lambda x, y: np.linalg.norm(x.cpu().numpy() - y) / np.linalg.norm(y)
        assert rel(ge[k], ge64) <= 1e-3 and rel(gs[k], gs64) <= 1e-3
    batch.close()


def test_persistent_batch_wait_timeout_is_reported_and_recovered(dev):
    """With a dependency-wait budget of zero polls, the merged launches' waits that are not
    already satisfied give up: the CTAs end, the contexts report GF_ETIMEOUT and nothing hangs.
    With the budget restored (the recorded schedule carries it, so it is recorded again) the
    next call is exact."""
    from paper_2506_20513_gb300 import FDTDBatch, _lib
    wls, fds, args = _flow_batch(dev)
    singles = [[x.clone() for x in fd.misfit_and_gradient(*a[:4])] for fd, a in zip(fds, args)]
    batch = FDTDBatch(fds)
    cols = [[a[i] for a in args] for i in range(4)]
    for fd in fds:
        fd.lib.gf_set_wait_budget(fd.ctx, 0)
    batch.misfit_and_gradient(*cols, mode=3)
    torch.cuda.synchronize(dev)
    codes = []
    for fd in fds:
        try:
            fd.status()
            codes.append(_lib.GF_OK)
        except _lib.GfError as e:
            codes.append(e.code)
    assert _lib.GF_ETIMEOUT in codes
    assert all(c in (_lib.GF_OK, _lib.GF_ETIMEOUT) for c in codes)
    for fd in fds:
        fd.lib.gf_set_wait_budget(fd.ctx, 1 << 22)
    J, ge, gs = batch.misfit_and_gradient(*cols, mode=3)
    torch.cuda.synchronize(dev)
    for fd in fds:
        fd.status()
    for k, (Js, ges, gss) in enumerate(singles):
        assert J[k].item() == Js.item()
        assert torch.equal(ge[k], ges) and torch.equal(gs[k], gss)
    batch.close()


def test_persistent_batch_needs_the_persistent_variant(dev):
    from paper_2506_20513_gb300 import FDTD, FDTDBatch, _lib
    wls, fds, args = _flow_batch(dev)
    fds[2].set_tiling(type(fds[2].tiling())(0, 0, 5, 0))
    batch = FDTDBatch(fds)
    with pytest.raises(_lib.GfError) as e:
        batch.misfit_and_gradient(*[[a[i] for a in args] for i in range(4)], mode=3)
    assert e.value.code == _lib.GF_EINVAL
    batch.close()
