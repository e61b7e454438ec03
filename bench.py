#!/usr/bin/env python
"""Benchmark: Gcell-updates/s of one dual-parameter FWI gradient (forward + adjoint).

One step = one ``misfit_and_gradient`` call over the 540x290-cell (20-cell CPML inside),
32-shot, nt = 2000, 100-receiver, 400 MHz layered + blob workload: the forward time loop
(Algorithm 1) with the full wavefield stored, the L2 misfit (Eq. objective) and the adjoint
time loop (Algorithm 2) accumulating the zero-lag gradients.  A cell-update is one cell
advanced one time step in one shot, counted once for the forward and once for the adjoint:
2 * N * nt * nshots per step.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle instead, on a
bounded sample of the same workload.  Under torchrun every rank runs its own 32-shot batch
(independent shots, no data-path collective: weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gcell-updates/s (fwd+adjoint) and s per dual-param FWI iteration vs HBM roofline"
UNIT = "Gcell-updates/s"
FALLBACK_HBM_GBS = 6800.0

# DRAM bytes (read + write) per cell-step of one launch, from `ncu --metrics
# dram__bytes_read.sum,dram__bytes_write.sum` of the same kernel code (kernel_source_tag),
# workload and tiling; see profiles/.  A change of the kernel code drops it.
# Warp instructions per cell-step of one launch (ncu InstructionStats, same keys): the
# kernels are bound by instruction issue, so the line also reports the issue roofline.
NCU_WARP_INST_PER_CELL_STEP: dict = {
    # profiles/adj_tile_multishot_540x290x32.md: 199.0 M warp instructions per K = 7 launch
    "adj@1085d4c1e613@540x290x32@default": 5.6732,
}
ISSUE_SLOTS_PER_SM_CLK = 4  # one warp instruction per scheduler per clock, 4 schedulers per SM

NCU_TRAFFIC_PER_CELL_STEP: dict = {
    # profiles/adj_tile_multishot_540x290x32.md: 339.3 MB per K = 7 launch
    "adj@1085d4c1e613@540x290x32@default": 9.6736,
}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nshots", type=int, default=32)
    ap.add_argument("--nt", type=int, default=2000)
    ap.add_argument("--tile", default="", help="tile_w,tile_h,steps_per_launch[,variant]")
    ap.add_argument("--workload", default="multishot",
                    choices=["multishot", "large", "uneven", "unet"],
                    help="multishot: 540x290, 32 shots, nt 2000 (default); large: 2108x1084, "
                         "16 shots, nt 8000 with checkpointing")
    ap.add_argument("--checkpoint", type=int, default=0,
                    help="checkpoint every k steps instead of storing the whole wavefield")
    ap.add_argument("--cpu-shots", type=int, default=0, help="oracle sample size (0 = auto)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--gemm", type=int, default=1, choices=[0, 1, 2],
                    help="U-Net workload: 1 = tcgen05 with TMA operand loads, 2 = tcgen05 with "
                         "thread-staged operands, 0 = explicit im2col and mma.sync GEMMs")
    ap.add_argument("--fwi-iters", type=int, default=10,
                    help="L-BFGS iterations timed for the s-per-FWI-iteration figure (0 = skip)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def workload(rank: int, nshots: int, nt: int, kind: str = "multishot"):
    from paper_2506_20513_gb300 import workloads as W
    if kind == "large":
        return W.large_checkpointed(seed=4000 + rank, nshots=min(nshots, 16), nt=nt)
    return W.multishot_layered(seed=1000 + rank, nshots=nshots, nt=nt)


def reduce_max(x: float, device) -> float:
    """Maximum of x over the ranks of the default process group (x itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(cells_per_rank: int, world: int, ms_max: float) -> float:
    """Whole-job Gcell-updates/s: every rank's work over the slowest rank's time."""
    return cells_per_rank * world / (ms_max / 1e3) / 1e9


def cpu_sample_shots(requested: int) -> int:
    if requested > 0:
        return requested
    cores = os.cpu_count() or 1
    try:
        mem_gb = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES") / 2 ** 30
    except (ValueError, OSError):
        mem_gb = 16.0
    # the oracle keeps each shot's FP64 wavefield history (~2.5 GB here) per thread
    return max(1, min(8, cores, int(mem_gb * 0.4 / 2.6)))


def run_oracle_sample(wl, shots: int):
    """Time the FP64 oracle gradient of `shots` shots (one OpenMP thread per shot)."""
    from oracle import oracle as O
    g = wl.grid
    wav = np.broadcast_to(O.ricker(wl.f0, g.dt, g.nt), (shots, 1, g.nt))
    obs = np.zeros((shots, g.nt, wl.nrec))
    t0 = time.perf_counter()
    O.misfit_and_gradient(g, wl.eps_init, wl.sig_init, wl.src[:shots], wav, wl.rec[:shots], obs,
                          nthreads=shots)
    dt = time.perf_counter() - t0
    cells = 2 * g.ncells * g.nt * shots
    return cells / dt / 1e9, dt


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    wl = workload(0, args.nshots, args.nt)
    shots = cpu_sample_shots(args.cpu_shots)
    for _ in range(args.warmup):
        run_oracle_sample(wl, shots)
    vals, times = [], []
    for _ in range(args.steps):
        v, t = run_oracle_sample(wl, shots)
        vals.append(v)
        times.append(t)
    value = 2 * wl.grid.ncells * wl.grid.nt * shots * args.steps / sum(times) / 1e9
    sample = (f"{shots} of {wl.nshots} shots per step (full {wl.grid.nx}x{wl.grid.ny} grid, "
              f"nt {wl.grid.nt}, forward + adjoint gradient), FP64 C oracle, one thread per shot")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "grid": f"{wl.grid.nx}x{wl.grid.ny}",
                   "shots_per_step": shots, "nt": wl.grid.nt, "nrec": wl.nrec},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": shots, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_tag():
    """sha1 prefix of gf_tile_kernels.cu without its // comments and blank lines: any change
    of the code drops the ncu figures keyed on it, an edit of a comment does not."""
    p = os.path.join(ROOT, "paper_2506_20513_gb300", "csrc", "gf_tile_kernels.cu")
    with open(p, encoding="utf-8") as f:
        lines = [re.sub(r"//.*$", "", line).rstrip() for line in f.read().splitlines()]
    code = "\n".join(line for line in lines if line.strip())
    return hashlib.sha1(code.encode()).hexdigest()[:12]


def algorithmic_bytes_per_launch(kind: str, wl, K: int) -> float:
    """Compulsory HBM bytes of one tile-kernel launch of K steps over all cells and shots:
    fields Ez, Hx, Hy read and written once (24 B), the model read once per cell (8 B,
    shared by the shots), CPML memories read and written in the strips (2 arrays x 8 B),
    plus per step: forward, the Ez history write (4 B); adjoint, the history read (4 B,
    K + 1 slots) and the per-shot gradient pair read and written once (16 B)."""
    g = wl.grid
    N, S = g.ncells, wl.nshots
    w = 2 * g.npml + 1
    strip_cells = w * g.ny + w * g.nx
    base = S * N * 24 + 8 * N + S * strip_cells * 16
    if kind == "fwd":
        return base + S * N * 4 * K
    return base + S * N * (16 + 4 * (K + 1))


def ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2506_20513_gb300 import FDTD, Tiling, _lib
    from paper_2506_20513_gb300.fdtd import ricker

    if args.workload == "large":
        if args.nt == 2000:
            args.nt = 8000
        if args.checkpoint <= 0:
            args.checkpoint = 100
        # the FP64 oracle would need ~146 GB of host memory per shot for this grid
        args.no_cpu_baseline = True
    wl = workload(rank, args.nshots, args.nt, args.workload)
    g = wl.grid
    tiling = Tiling(*[int(x) for x in args.tile.split(",")]) if args.tile else None
    fd = FDTD(g, wl.src, wl.rec, device=dev, tiling=tiling)
    if args.checkpoint > 0:
        fd.set_storage(args.checkpoint)
    t32 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    wav = t32(np.broadcast_to(ricker(wl.f0, g.dt, g.nt), (wl.nshots, 1, g.nt)))
    eps_t, sig_t = t32(wl.eps_true), t32(wl.sig_true)
    eps0, sig0 = t32(wl.eps_init), t32(wl.sig_init)
    obs = fd.forward_model(eps_t, sig_t, wav)
    fd.status()

    def step():
        return fd.misfit_and_gradient(eps0, sig0, wav, obs)

    for _ in range(args.warmup):
        step()
    fd.status()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    clocks = ClockSampler(torch.cuda.current_device())
    barrier()
    clocks.start()
    lib, ctx = fd.lib, fd.ctx
    launches0 = lib.gf_kernel_launches(ctx)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        J, ge, gs = step()
    e1.record()
    barrier()
    ms = e0.elapsed_time(e1)
    gpu_launches = lib.gf_kernel_launches(ctx) - launches0
    # the same K steps again with CUDA events around every launch on its stream, for the
    # per-kernel durations of the roofline (kept out of the timed region above: the events
    # cost about 1.5% of the step)
    lib.gf_profile(ctx, 1)
    for _ in range(args.steps):
        step()
    barrier()
    import ctypes
    prof = {}
    for name, kind in (("fwd", _lib.GF_KERNEL_FWD), ("adj", _lib.GF_KERNEL_ADJ),
                       ("aux", _lib.GF_KERNEL_AUX)):
        tot, cnt = ctypes.c_double(), ctypes.c_longlong()
        lib.gf_profile_read(ctx, kind, ctypes.byref(tot), ctypes.byref(cnt))
        prof[name] = (tot.value, cnt.value)
    lib.gf_profile(ctx, 0)
    clk = clocks.stop()
    fd.status()
    ms = reduce_max(ms, dev)
    cells = wl.cell_updates() * args.steps * world
    value = job_value(wl.cell_updates() * args.steps, world, ms)

    # roofline of the dominant tile kernel (its own launches, CUDA events on its stream)
    dom = max(("fwd", "adj"), key=lambda k: prof[k][0])
    tot_ms, cnt = prof[dom]
    nt = g.nt
    # launches of K steps except a possibly shorter last one: use the mean steps per launch
    per_launch_steps = nt / max(1, cnt / args.steps)
    algo = algorithmic_bytes_per_launch(dom, wl, per_launch_steps)
    avg_s = tot_ms / 1e3 / max(1, cnt)
    peak, peak_kind = hbm_peak()
    achieved = algo / avg_s / 1e9
    key = f"{dom}@{kernel_source_tag()}@{g.nx}x{g.ny}x{wl.nshots}@{args.tile or 'default'}"
    tpc = NCU_TRAFFIC_PER_CELL_STEP.get(key)
    traffic = tpc * wl.nshots * g.ncells * per_launch_steps if tpc else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "kernel": f"{dom}_tile",
            "peak_source": f"hbm_gbs of {peak_kind}",
            "avg_launch_us": avg_s * 1e6, "launches": cnt,
            "phase_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()}}
    ipc = NCU_WARP_INST_PER_CELL_STEP.get(key)
    if ipc:
        # the bound that holds the kernel: warp instructions issued per second against the
        # issue rate of all schedulers at the SM clock sampled during the timed region
        mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
        inst = ipc * wl.nshots * g.ncells * per_launch_steps
        peak_issue = torch.cuda.get_device_properties(dev).multi_processor_count * \
            ISSUE_SLOTS_PER_SM_CLK * mhz * 1e6
        roof["issue"] = {"achieved": inst / avg_s / 1e9, "peak": peak_issue / 1e9,
                         "unit": "G warp-instructions/s", "frac": inst / avg_s / peak_issue,
                         "warp_instructions_per_launch": inst,
                         "peak_source": "SMs x 4 schedulers x sampled SM clock"}
    if not args.checkpoint:
        # the whole step against the bytes an untiled stencil moves per cell-update (forward:
        # fields read+written 24 B, Ca/Cb 8 B, history write 4 B; adjoint: 24 + 8 B, history
        # read 4 B, gradient pair read+written 16 B; 44 B on average over the two)
        naive = (36.0 + 52.0) / 2
        eff = value / world * naive  # per GPU: Gcell/s x B = GB/s
        roof["effective"] = {"achieved": eff, "peak": peak, "unit": "GB/s", "frac": eff / peak,
                             "naive_bytes_per_cell_update": naive,
                             "meaning": "Gcell-updates/s x untiled bytes per cell-update"}

    # end to end through the public API with host (pinned) buffers
    e2e = None
    if not args.no_e2e:
        h = lambda t: t.detach().to("cpu").pin_memory()
        he, hs, hw, ho = h(eps0), h(sig0), h(wav), h(obs)
        fd.misfit_and_gradient(he, hs, hw, ho)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            Jh, geh, gsh = fd.misfit_and_gradient(he, hs, hw, ho)
        barrier()
        te = reduce_max(time.perf_counter() - t0, dev)
        h2d = sum(x.numel() * x.element_size() for x in (he, hs, hw, ho))
        d2h = Jh.numel() * 8 + geh.numel() * 4 + gsh.numel() * 4
        e2e = {"value": cells / te / 1e9, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    # seconds per dual-parameter FWI iteration (L-BFGS with its line-search evaluations)
    fwi = None
    if args.fwi_iters > 0:
        from paper_2506_20513_gb300.fwi import FWI, FWIConfig, interior_mask
        drv = FWI(fd, lambda f0: obs, interior_mask(g, rows_below_top=4),
                  FWIConfig(bands=((wl.f0, args.fwi_iters),)))
        # an untimed pass first: the FWI driver's first iterations otherwise include the one-time
        # loading of the PyTorch kernels its L-BFGS algebra uses (seconds on a fresh process)
        drv.run(eps0, sig0)
        _, _, hist = drv.run(eps0, sig0)
        fwi = {"iterations": len(hist.seconds),
               "s_per_iteration": sum(hist.seconds) / max(1, len(hist.seconds)),
               "evaluations_per_iteration": sum(hist.evaluations) / max(1, len(hist.evaluations)),
               "misfit_first_last": [hist.misfit[0], hist.final_misfit] if hist.misfit else None}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        shots = cpu_sample_shots(args.cpu_shots)
        v, t = run_oracle_sample(wl, shots)
        cpu = {"value": v, "unit": UNIT, "cores": shots, "kind": "oracle",
               "sample": (f"{shots} of {wl.nshots} shots, full grid and nt, forward + adjoint "
                          f"gradient, FP64 C oracle, one thread per shot, {t:.1f} s")}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": wl.name, "grid": f"{g.nx}x{g.ny}", "npml": g.npml,
                       "shots_per_gpu": wl.nshots, "nt": g.nt, "nrec": wl.nrec,
                       "cell_updates_per_step": wl.cell_updates() * world,
                       "s_per_gradient": ms / args.steps / 1e3,
                       "tiling": args.tile or "default 50,50,7,variant 0",
                       "l2": "inputs larger than L2: each step streams the "
                             f"{wl.nshots * g.nt * g.ncells * 4 / 1e9:.1f} GB wavefield "
                             "through HBM" if not args.checkpoint else
                             "inputs larger than L2: checkpoints and segment buffers of "
                             f"{fd.workspace_bytes() / 1e9:.1f} GB",
                       "storage": (f"checkpoint every {args.checkpoint} steps"
                                   if args.checkpoint else "full wavefield"),
                       "workspace_gb": fd.workspace_bytes() / 1e9,
                       "parallelism": f"shots x{world} (independent per GPU)",
                       "fwi": fwi},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    fd.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def uneven(args):
    """64 independent instances of uneven size (128-768 x 128-384 cells + 20-cell CPML, nt
    800-3000, 1-8 shots, checkpoints every 100 steps), each tuned by the autotuner, one
    gradient each per step: one after the other vs concurrently as one replayed CUDA graph."""
    import tempfile

    import torch
    from paper_2506_20513_gb300 import FDTD, FDTDBatch, autotune, workloads as W
    from paper_2506_20513_gb300.fdtd import ricker
    dev = torch.device("cuda", 0)
    insts = W.uneven_instances(count=args.nshots if args.nshots != 32 else 64)
    t32 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    cache = os.path.join(tempfile.gettempdir(), "gprfwi_autotune.txt")
    fds, ins = [], []
    t_tune = time.perf_counter()
    for wl in insts:
        g = wl.grid
        fd = FDTD(g, wl.src, wl.rec, device=dev)
        wav = t32(np.broadcast_to(ricker(wl.f0, g.dt, g.nt), (wl.nshots, 1, g.nt)))
        e0, s0 = t32(wl.eps_init), t32(wl.sig_init)
        autotune(fd, e0, s0, wav, cache, probe_steps=36)
        fd.set_storage(100)
        obs = fd.forward_model(t32(wl.eps_true), t32(wl.sig_true), wav)
        fds.append(fd)
        ins.append((e0, s0, wav, obs))
    torch.cuda.synchronize(dev)
    t_tune = time.perf_counter() - t_tune
    batch = FDTDBatch(fds)
    cols = [list(x) for x in zip(*ins)]
    cells = sum(w.cell_updates() for w in insts)
    out = {}
    for mode in (0, 2):
        for _ in range(max(1, args.warmup)):
            batch.misfit_and_gradient(*cols, mode=mode)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            batch.misfit_and_gradient(*cols, mode=mode)
        e1.record()
        torch.cuda.synchronize(dev)
        out[mode] = e0.elapsed_time(e1) / args.steps
    tilings = {}
    for fd in fds:
        t = fd.tiling()
        key = f"{t.tile_w}x{t.tile_h}/K{t.steps}/v{t.variant}"
        tilings[key] = tilings.get(key, 0) + 1
    line = {"metric": METRIC + " (uneven-instance batch)", "value": cells / (out[2] / 1e3) / 1e9,
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": out[2], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{len(insts)} uneven instances (128-768 x 128-384 + CPML, "
                                   "nt 800-3000, 1-8 shots), checkpoint every 100 steps",
                       "cell_updates_per_step": cells, "ms_sequential": out[0],
                       "ms_graph": out[2], "speedup_graph_vs_sequential": out[0] / out[2],
                       "autotune_s": t_tune, "tilings_chosen": tilings}}
    print(json.dumps(line), flush=True)
    batch.close()
    return 0


def bf16_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["bf16_tflops"]), "bf16_tflops (burst) of measured"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback"


def unet(args):
    """Training step of the learned preconditioner's U-Net (4 levels, 32 base channels,
    4 in / 2 out, 128 x 256 images, batch 16, BF16 kernels): forward, masked MSE, backward,
    Adam.  The roofline is the tensor-core one of its GEMM launches (algorithmic 2 M N K
    FLOPs over their CUDA-event time) against the measured cuBLAS bf16 rate."""
    import torch
    from oracle import unet_oracle as U
    from paper_2506_20513_gb300.unet import UNet
    dev = torch.device("cuda", 0)
    B, H, Wd = 16, 128, 256
    net = UNet(4, 32, 4, 2, H, Wd, max_batch=B, device=dev)
    net.set_gemm(args.gemm)
    net.init_params(1)
    g = torch.Generator().manual_seed(1)
    x = torch.randn(B, H, Wd, 4, generator=g).to(dev)
    t = torch.randn(B, H, Wd, 2, generator=g).to(dev)
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)  # > L2 (129 MB)
    for _ in range(max(3, args.warmup)):
        net.train_step(x, t, lr=1e-4)
    torch.cuda.synchronize(dev)
    net.profile(True)
    net.profile_read()
    l0 = net.kernel_launches
    clocks = ClockSampler(0)
    clocks.start()
    total = 0.0
    for _ in range(args.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        net.train_step(x, t, lr=1e-4)
        e1.record()
        torch.cuda.synchronize(dev)
        total += e0.elapsed_time(e1)
    clk = clocks.stop()
    net.status()
    gemm_ms, gemm_n, gemm_flops = net.profile_read()
    net.profile(False)
    launches = net.kernel_launches - l0
    ms = total / args.steps
    peak, peak_kind = bf16_peak()
    achieved = gemm_flops / (gemm_ms / 1e3) / 1e12
    fwd = U.flops_per_sample(4, 32, 4, 2, H, Wd)
    cpu = None
    if not args.no_cpu_baseline:
        rng = np.random.default_rng(0)
        p = U.init_params(rng, 4, 32, 4, 2)
        xs, ts = rng.standard_normal((1, H, Wd, 4)), rng.standard_normal((1, H, Wd, 2))
        t0 = time.perf_counter()
        U.loss_and_gradient(p, xs, ts, None, 4, 32, 4, 2)
        dt = time.perf_counter() - t0
        cpu = {"value": 1.0 / dt, "unit": "samples/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"one 128x256 sample, FP64 numpy forward + backward, {dt:.2f} s"}
    line = {"metric": "U-Net training samples/s (learned preconditioner) vs tensor roofline",
            "value": B * 1e3 / ms, "unit": "samples/s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "unet_4lvl_32ch_4to2_128x256_batch16",
                       "fwd_gflop_per_sample": fwd / 1e9,
                       "l2": "a 256 MB buffer is written before every timed step"},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                         "kernel": ("tc_gemm_kernel (tcgen05%s: K-major convolutions, MN-major "
                                    "weight gradients) + gemm_kernel (mma.sync, 1x1 and cin=4)"
                                    % (" + TMA" if args.gemm == 1 else "")
                                    if args.gemm else "gemm_kernel (mma.sync bf16)"),
                         "peak_source": peak_kind,
                         "gemm_ms_per_step": gemm_ms / args.steps,
                         "gemm_launches_per_step": gemm_n / args.steps},
            "cpu_baseline": cpu, "e2e": None, "gpu_launches": launches, "clocks": clk}
    print(json.dumps(line), flush=True)
    net.close()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "uneven":
        return uneven(args)
    if args.workload == "unet":
        return unet(args)
    return ours(args)


if __name__ == "__main__":
    sys.exit(main())
