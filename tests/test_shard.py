"""Shot sharding with a sum all-reduce of (J, g_eps_r, g_sigma), on the CPU: the round-robin
partition covers every shot once, and two gloo ranks that each run their share (the FP64
oracle standing in for the per-rank FDTD context) and sum the results get the single-process
oracle gradient of the whole acquisition, on both ranks; an FWI iteration driven through the
sharded object takes the same step on both ranks."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2506_20513_gb300 import workloads as W  # noqa: E402
from paper_2506_20513_gb300.shard import ShardedGradient, allreduce_sum, shard_shots  # noqa: E402


def test_round_robin_partition_covers_every_shot_once():
    for nshots in (1, 2, 5, 32, 33):
        for world in (1, 2, 3, 4, 8):
            parts = [shard_shots(nshots, r, world) for r in range(world)]
            allshots = np.sort(np.concatenate(parts))
            assert np.array_equal(allshots, np.arange(nshots))
            sizes = [p.size for p in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_shots(4, 2, 2)


def test_without_a_process_group_the_reduction_is_the_identity():
    J = torch.tensor([2.5], dtype=torch.float64)
    ge, gs = torch.ones(3, 4), torch.full((3, 4), 2.0)
    assert allreduce_sum(J, ge, gs) == (J, ge, gs)


class OracleContext:
    """The parts of an FDTD context the sharded gradient and the FWI driver use, computed by
    the FP64 oracle on the host."""

    def __init__(self, grid, src, rec):
        self.grid, self.src, self.rec = grid, np.asarray(src), np.asarray(rec)
        self.device = torch.device("cpu")
        self.shape = (grid.ny, grid.nx)
        self.lib = None

    def misfit_and_gradient(self, eps, sig, wav, obs):
        w = np.broadcast_to(wav.numpy(), (self.src.shape[0], 1, self.grid.nt)) \
            if wav.dim() == 1 else wav.numpy()
        J, ge, gs = O.misfit_and_gradient(self.grid, eps.double().numpy(), sig.double().numpy(),
                                          self.src, w, self.rec, obs.numpy())
        return torch.tensor([J], dtype=torch.float64), torch.tensor(ge), torch.tensor(gs)

    def misfit(self, eps, sig, wav, obs, out=None):
        J = self.misfit_and_gradient(eps, sig, wav, obs)[0]
        if out is not None:
            out.copy_(J)
            return out
        return J

    def close(self):
        pass


def _case():
    wl = W.small_random(21, nxp=24, nyp=18, npml=5, nt=90, nshots=5, nrec=6)
    g = wl.grid
    wav = np.broadcast_to(O.ricker(wl.f0, g.dt, g.nt), (wl.nshots, 1, g.nt)).copy()
    obs = O.forward(g, wl.eps_true, wl.sig_true, wl.src, wav, wl.rec)
    return wl, wav, obs


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl, wav, obs = _case()
    sg = ShardedGradient(wl.grid, wl.src, wl.rec, context=OracleContext)
    e0, s0 = torch.tensor(wl.eps_init), torch.tensor(wl.sig_init)
    J, ge, gs = sg.misfit_and_gradient(e0, s0, torch.tensor(wav), torch.tensor(obs))
    Jm = sg.misfit(e0, s0, torch.tensor(wav), torch.tensor(obs))
    # two L-BFGS iterations of the FWI driver over the sharded gradient, replicated per rank
    from paper_2506_20513_gb300 import fwi as F
    torch.cuda.synchronize = lambda *a, **k: None
    drv = F.FWI(sg, lambda f0: torch.tensor(obs), F.interior_mask(wl.grid),
                F.FWIConfig(bands=((wl.f0, 2),)))
    eps, sig, hist = drv.run(e0.float(), s0.float())
    out[rank] = (sg.shots.tolist(), float(J[0]), ge.numpy(), gs.numpy(), float(Jm[0]),
                 eps.numpy(), hist.misfit)
    dist.destroy_process_group()


def test_two_gloo_ranks_sum_to_the_whole_acquisition_gradient():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    wl, wav, obs = _case()
    J, ge, gs = O.misfit_and_gradient(wl.grid, wl.eps_init, wl.sig_init, wl.src, wav, wl.rec, obs)
    assert res[0][0] == [0, 2, 4] and res[1][0] == [1, 3]
    for r in range(world):
        _, Jr, ger, gsr, Jmr = res[r][:5]
        assert Jr == pytest.approx(J, rel=1e-12)
        assert Jmr == pytest.approx(J, rel=1e-12)
        # the shares are summed in another order than the shots: FP64 rounding only
        assert np.abs(ger - ge).max() <= 1e-10 * np.abs(ge).max()
        assert np.abs(gsr - gs).max() <= 1e-10 * np.abs(gs).max()
    # both ranks hold bit-identical reduced values
    assert np.array_equal(res[0][2], res[1][2]) and np.array_equal(res[0][3], res[1][3])
    # the replicated inversion takes the same steps on both ranks and lowers the misfit
    assert np.array_equal(res[0][5], res[1][5])
    assert res[0][6] == res[1][6]
    assert res[0][6][0] == pytest.approx(J, rel=1e-6)
    assert res[0][6][-1] < res[0][6][0]
