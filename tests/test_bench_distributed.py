"""The multi-GPU path of bench.py on CPU: two gloo ranks share one acquisition over one
seeded model, each with its own round-robin half of the shots (weak scaling: the shots per
rank are fixed); the timing is reduced as the max over ranks."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.reduce_max(100.0 + 50.0 * rank, "cpu")
    wl = bench.workload(rank, nshots=4, nt=20, world=world)
    value = bench.job_value(wl.cell_updates(), world, ms)
    out[rank] = (ms, value, wl.src.tolist(), float(wl.eps_true.sum()), wl.grid.nx)
    dist.destroy_process_group()


def test_two_rank_weak_scaling_reduction():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    ms0, v0, s0, e0, nx0 = res[0]
    ms1, v1, s1, e1, nx1 = res[1]
    assert ms0 == ms1 == 150.0              # the slowest rank's time on every rank
    assert v0 == v1                          # whole-job value: all ranks' work / max time
    assert nx0 == nx1 and e0 == e1           # one model, one grid ...
    import bench
    whole = bench.workload(0, nshots=8, nt=20)
    assert len(s0) == len(s1) == 4           # ... 4 shots per rank (weak scaling) ...
    # ... which together are the whole 8-shot acquisition, split round-robin
    assert s0 == whole.src[0::2].tolist() and s1 == whole.src[1::2].tolist()
    wl = bench.workload(0, nshots=4, nt=20, world=2)
    assert v0 == pytest.approx(wl.cell_updates() * 2 / 0.150 / 1e9)
