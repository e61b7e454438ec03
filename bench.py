#!/usr/bin/env python
"""Benchmark: Gcell-updates/s of one dual-parameter FWI gradient (forward + adjoint).

One step = one ``misfit_and_gradient`` call over the 540x290-cell (20-cell CPML inside),
32-shot, nt = 2000, 100-receiver, 400 MHz layered + blob workload: the forward time loop
(Algorithm 1) with the full wavefield stored, the L2 misfit (Eq. objective) and the adjoint
time loop (Algorithm 2) accumulating the zero-lag gradients.  A cell-update is one cell
advanced one time step in one shot, counted once for the forward and once for the adjoint:
2 * N * nt * nshots per step.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle instead, on a
bounded sample of the same workload.  Under torchrun the ranks share one acquisition of
32 x N shots over one model, split round-robin (32 shots per GPU: weak scaling); every step
ends with an NCCL all-reduce of (J, g_eps_r, g_sigma), as one sharded inversion needs.
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

# Per-launch figures from one ncu capture of the tile kernels (`ncu --set full --clock-control
# none -k regex:<kernel>` on the multishot workload with nt = 70, default tiling, one shot lane:
# launches of all 32 shots), divided by the launch's cell-steps.
# Keyed on kernel_source_tag(): any change of the kernel code drops them (reported as null).
# DRAM bytes (read + write) per cell-step:
NCU_TRAFFIC_PER_CELL_STEP: dict = {
    "adj@1f1660801c10@540x290x32@default": 12.1320,   # 425.57 MB / 35.0784 M cell-steps
    "fwd@1f1660801c10@540x290x32@default": 8.0039,    # 280.77 MB
}
# Warp instructions per cell-step (the kernels are bound by instruction issue, so the line
# also reports the issue roofline):
NCU_WARP_INST_PER_CELL_STEP: dict = {
    "adj@1f1660801c10@540x290x32@default": 2.9761,    # 104.396 M warp instructions
    "fwd@1f1660801c10@540x290x32@default": 2.0820,    # 73.032 M
}
ISSUE_SLOTS_PER_SM_CLK = 4  # one warp instruction per scheduler per clock, 4 schedulers per SM
# the files holding the tile kernels' device code
KERNEL_SOURCES = ("gf_tile_kernels.cu", "gf_tile_common.cuh")


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
                    choices=["multishot", "large", "disc", "precond", "uneven", "unet"],
                    help="multishot: 540x290, 32 shots, nt 2000 (default); large: 2108x1084, "
                         "16 shots, nt 8000 with checkpointing")
    ap.add_argument("--checkpoint", type=int, default=0,
                    help="checkpoint every k steps instead of storing the whole wavefield")
    ap.add_argument("--lanes", type=int, default=2,
                    help="shot lanes: groups of shots whose passes run concurrently")
    ap.add_argument("--reconstruct", action="store_true",
                    help="with --checkpoint: reconstruct each segment backwards from a stored "
                         "boundary ring instead of keeping its Ez (experimental)")
    ap.add_argument("--cpu-shots", type=int, default=0, help="oracle sample size (0 = auto)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--gemm", type=int, default=1, choices=[0, 1, 2],
                    help="U-Net workload: 1 = tcgen05 with TMA operand loads, 2 = tcgen05 with "
                         "thread-staged operands, 0 = explicit im2col and mma.sync GEMMs")
    ap.add_argument("--fwi-iters", type=int, default=50,
                    help="L-BFGS iterations of the timed three-band FWI run (0 = skip)")
    ap.add_argument("--no-te", action="store_true",
                    help="skip the TE-mode forward model sub-record")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the 2108x1084, 16-shot, nt 8000 checkpointed-gradient sub-record")
    ap.add_argument("--large-checkpoint", type=int, default=200,
                    help="checkpoint interval of the large-grid sub-record")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def workload(rank: int, nshots: int, nt: int, kind: str = "multishot", world: int = 1):
    """This rank's share of one acquisition of nshots x world shots over one seeded model:
    shots split round-robin over the ranks (weak scaling: nshots per GPU)."""
    from dataclasses import replace
    from paper_2506_20513_gb300 import workloads as W
    from paper_2506_20513_gb300.shard import shard_shots
    if kind == "large":
        wl = W.large_checkpointed(seed=4000, nshots=min(nshots, 16) * world, nt=nt)
    elif kind == "disc":
        return W.single_shot_disc()
    elif kind == "precond":
        return W.preconditioner_model(5000000, nshots=16 * world, nt=nt)
    else:
        wl = W.multishot_layered(seed=1000, nshots=nshots * world, nt=nt)
    if world == 1:
        return wl
    mine = shard_shots(wl.nshots, rank, world)
    return replace(wl, src=wl.src[mine], rec=wl.rec[mine])


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


def host_cores() -> int:
    """Cores this process may run on (the box's nproc)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def cpu_sample_shots(requested: int, nshots: int) -> int:
    """Shots of the oracle sample: one OpenMP thread each, as many as there are cores and
    shots, fewer if host memory is short (each thread keeps its shot's FP64 wavefield
    history, about 2.6 GB on the 540x290, nt 2000 grid)."""
    if requested > 0:
        return min(requested, nshots)
    try:
        mem_gb = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES") / 2 ** 30
    except (ValueError, OSError):
        mem_gb = 16.0
    return max(1, min(nshots, host_cores(), int(mem_gb * 0.4 / 2.6)))


def run_oracle_sample(wl, shots: int):
    """Time the FP64 oracle gradient of the first `shots` shots (one OpenMP thread per shot)."""
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


def oracle_sample_text(wl, shots: int, seconds: float) -> str:
    g = wl.grid
    return (f"shots 0-{shots - 1} of the {wl.nshots}-shot batch (full {g.nx}x{g.ny} grid, "
            f"nt {g.nt}, forward + adjoint gradient), FP64 C oracle, one OpenMP thread per "
            f"shot on {shots} of {host_cores()} host cores, {seconds:.1f} s; the rate is over "
            f"the cells computed, so the whole batch would take "
            f"{seconds * wl.nshots / shots:.1f} s at it")


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    wl = workload(0, args.nshots, args.nt)
    shots = cpu_sample_shots(args.cpu_shots, wl.nshots)
    for _ in range(args.warmup):
        run_oracle_sample(wl, shots)
    vals, times = [], []
    for _ in range(args.steps):
        v, t = run_oracle_sample(wl, shots)
        vals.append(v)
        times.append(t)
    value = 2 * wl.grid.ncells * wl.grid.nt * shots * args.steps / sum(times) / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "grid": f"{wl.grid.nx}x{wl.grid.ny}",
                   "shots_per_step": shots, "nt": wl.grid.nt, "nrec": wl.nrec},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": shots, "nproc": host_cores(),
                         "kind": "oracle",
                         "sample": oracle_sample_text(wl, shots, sum(times) / len(times))},
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
    """sha1 prefix of the tile kernels' device code without its // comments and blank lines:
    any change of the code drops the ncu figures keyed on it, an edit of a comment does not."""
    code = []
    for name in KERNEL_SOURCES:
        p = os.path.join(ROOT, "paper_2506_20513_gb300", "csrc", name)
        with open(p, encoding="utf-8") as f:
            lines = [re.sub(r"//.*$", "", line).rstrip() for line in f.read().splitlines()]
        code.append("\n".join(line for line in lines if line.strip()))
    return hashlib.sha1("\n\f".join(code).encode()).hexdigest()[:12]


def algorithmic_bytes_per_launch(kind: str, wl, K: float, history: float = 1.0,
                                 shots: float | None = None) -> float:
    """Compulsory HBM bytes of one tile-kernel launch of K steps over all cells and the
    workload's shots (or ``shots`` of them: one lane's launch):
    fields Ez, Hx, Hy read and written once (24 B), the model read once per cell (Ca, Cb:
    8 B, shared by the shots), CPML memories read and written in the strips (2 arrays x 8 B),
    plus per step: forward, the Ez history write (4 B; ``history`` = the fraction of forward
    launches that store it, 0 for a misfit-only forward, 1/2 under checkpointing where the
    first pass keeps only the checkpoints); adjoint, the history read (4 B, K + 1 slots) and
    the per-shot gradient pair read and written once (16 B)."""
    g = wl.grid
    N, S = g.ncells, (wl.nshots if shots is None else shots)
    w = 2 * g.npml + 1
    strip_cells = w * g.ny + w * g.nx
    base = S * N * 24 + 8 * N + S * strip_cells * 16
    if kind == "fwd":
        return base + history * S * N * 4 * K
    return base + S * N * (16 + 4 * (K + 1))


def read_profile(lib, ctx) -> dict:
    """Per launch class: (busy ms, launches, summed ms) from the library's CUDA-event
    profile; busy = the union of the launches' intervals (the launches of concurrent shot
    lanes, and consecutive launches under programmatic dependent launch, overlap)."""
    import ctypes
    from paper_2506_20513_gb300 import _lib
    prof = {}
    for name, kind in (("fwd", _lib.GF_KERNEL_FWD), ("adj", _lib.GF_KERNEL_ADJ),
                       ("aux", _lib.GF_KERNEL_AUX)):
        tot, span, cnt = ctypes.c_double(), ctypes.c_double(), ctypes.c_longlong()
        lib.gf_profile_read_span(ctx, kind, ctypes.byref(tot), ctypes.byref(span),
                                 ctypes.byref(cnt))
        prof[name] = (span.value, cnt.value, tot.value)
    return prof


def blocks_per_pass(nt: int, K: int, checkpoint: int) -> int:
    """Launches of one pass of one lane: K-step blocks, the last of each segment shorter."""
    if checkpoint <= 0:
        return -(-nt // K)
    return sum(-(-min(checkpoint, nt - j) // K) for j in range(0, nt, checkpoint))


def tile_roofline(prof: dict, wl, steps: int, history_fwd: float, tiling: str, clk: dict,
                  sms: int, K: int = 7, checkpoint: int = 0) -> dict:
    """Roofline of the dominant tile kernel from its own launches' CUDA-event intervals: the
    algorithmic bytes of all its launches over the time they kept the GPU busy (the union
    of their intervals), i.e. bytes per launch over the effective launch duration."""
    g = wl.grid
    dom = max(("fwd", "adj"), key=lambda k: prof[k][0])
    tot_ms, cnt, sum_ms = prof[dom]
    # launches of K steps except the shorter last one of a segment: use the mean steps per
    # launch; under checkpointing the forward runs twice per gradient (checkpoints, then
    # recompute); the shots may be split into concurrent lanes, each launch one lane's shots
    passes = 2 if (dom == "fwd" and history_fwd < 1.0) else 1
    blocks = blocks_per_pass(g.nt, K, checkpoint)
    lanes = max(1, round(cnt / max(1, steps * passes * blocks)))
    per_launch_steps = g.nt / blocks
    shots = wl.nshots / lanes
    algo = algorithmic_bytes_per_launch(dom, wl, per_launch_steps, history_fwd, shots)
    avg_s = tot_ms / 1e3 / max(1, cnt)
    peak, peak_kind = hbm_peak()
    achieved = algo / avg_s / 1e9
    key = f"{dom}@{kernel_source_tag()}@{g.nx}x{g.ny}x{wl.nshots}@{tiling}"
    cell_steps = shots * g.ncells * per_launch_steps
    tpc = NCU_TRAFFIC_PER_CELL_STEP.get(key)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": tpc * cell_steps if tpc else None,
            "kernel": f"{dom}_tile_kernel", "peak_source": f"hbm_gbs of {peak_kind}",
            "algorithmic_bytes_per_launch": algo, "steps_per_launch": per_launch_steps,
            "shot_lanes": lanes, "shots_per_launch": shots,
            "avg_launch_us": avg_s * 1e6, "launches": cnt,
            "avg_launch_event_us": sum_ms / 1e3 / max(1, cnt) * 1e6,
            "phase_ms_per_step": {k: v[0] / steps for k, v in prof.items()}}
    ipc = NCU_WARP_INST_PER_CELL_STEP.get(key)
    if ipc:
        # the bound that holds the kernel: warp instructions issued per second against the
        # issue rate of all schedulers at the SM clock sampled during the timed region
        mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
        inst = ipc * cell_steps
        peak_issue = sms * ISSUE_SLOTS_PER_SM_CLK * mhz * 1e6
        roof["issue"] = {"achieved": inst / avg_s / 1e9, "peak": peak_issue / 1e9,
                         "unit": "G warp-instructions/s", "frac": inst / avg_s / peak_issue,
                         "warp_instructions_per_launch": inst,
                         "peak_source": "SMs x 4 schedulers x sampled SM clock"}
    return roof


def read_tile_span(lib, ctx) -> float:
    """Milliseconds during which forward or adjoint tile launches kept the GPU busy (the
    union of their intervals; the records stay for read_profile)."""
    import ctypes
    tot, span, cnt = ctypes.c_double(), ctypes.c_double(), ctypes.c_longlong()
    lib.gf_profile_read_span(ctx, 3, ctypes.byref(tot), ctypes.byref(span), ctypes.byref(cnt))
    return span.value


def lanes_used(fd, args) -> int:
    """Shot lanes of the run (the library runs one with the persistent variant or the
    reconstruction storage)."""
    t = fd.tiling()
    if t.variant == 3 or args.reconstruct:
        return 1
    return max(1, min(args.lanes, fd.nshots))


def path_roofline(span_ms: float, wl, steps: int, K: int, checkpoint: int,
                  tiling: str = "default") -> dict:
    """The forward and adjoint tile kernels together: the algorithmic bytes of all their
    launches over the time they kept the GPU busy (their launches overlap when the shots run
    in concurrent lanes)."""
    g = wl.grid
    blocks = blocks_per_pass(g.nt, K, checkpoint)
    k_avg = g.nt / blocks
    fwd = blocks * (algorithmic_bytes_per_launch("fwd", wl, k_avg, 1.0)
                    + (algorithmic_bytes_per_launch("fwd", wl, k_avg, 0.0) if checkpoint else 0))
    adj = blocks * algorithmic_bytes_per_launch("adj", wl, k_avg)
    total = steps * (fwd + adj)
    peak, peak_kind = hbm_peak()
    achieved = total / (span_ms / 1e3) / 1e9
    # ncu's DRAM bytes per cell-step of both kernels (same code), over the step's cell-steps
    tag = kernel_source_tag()
    key = lambda k: f"{k}@{tag}@{g.nx}x{g.ny}x{wl.nshots}@{tiling}"
    tf, ta = (NCU_TRAFFIC_PER_CELL_STEP.get(key(k)) for k in ("fwd", "adj"))
    cells = wl.nshots * g.ncells * g.nt
    traffic = (tf * cells * (2 if checkpoint else 1) + ta * cells) if tf and ta else None
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "traffic_unit": "bytes per step",
            "kernel": "fwd_tile_kernel + adj_tile_kernel (concurrent shot lanes)",
            "peak_source": f"hbm_gbs of {peak_kind}",
            "algorithmic_bytes_per_step": total / steps, "busy_ms_per_step": span_ms / steps,
            "meaning": "algorithmic bytes of every tile launch of the step over the time the "
                       "tile launches kept the GPU busy (union of their CUDA-event intervals)"}


def fwi_leg(args, fd, wl, eps_t, sig_t, eps0, sig0) -> dict:
    """The multishot workload's inversion as specified for it: L-BFGS over three Ricker bands
    (100, 200, 400 MHz peak) with TV regularisation on, ``args.fwi_iters`` iterations in all,
    from the smoothed starting model.  Reports seconds, FDTD evaluations and forward-equivalent
    passes per iteration, and the iteration's HBM fraction: the algorithmic bytes of all its
    FDTD time loops over its wall time."""
    import torch
    from paper_2506_20513_gb300.fdtd import ricker
    from paper_2506_20513_gb300.fwi import FWI, FWIConfig, interior_mask
    g = wl.grid
    dev = fd.device
    freqs = (100e6, 200e6, 400e6)
    n = args.fwi_iters
    iters = (n // 3, n // 3, n - 2 * (n // 3))
    wav = lambda f0: torch.tensor(np.broadcast_to(ricker(f0, g.dt, g.nt), (wl.nshots, 1, g.nt)),
                                  dtype=torch.float32, device=dev)
    observed = {f0: fd.forward_model(eps_t, sig_t, wav(f0)) for f0 in freqs}
    mask = interior_mask(g, rows_below_top=4)
    # an untimed two-iteration run first: the driver's first iterations otherwise include the
    # one-time loading of the PyTorch kernels its L-BFGS algebra uses
    FWI(fd, observed.get, mask, FWIConfig(bands=((freqs[0], 2),), tv=True)).run(eps0, sig0)
    cfg = FWIConfig(bands=tuple(zip(freqs, iters)), tv=True)
    drv = FWI(fd, observed.get, mask, cfg)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    eps, sig, hist = drv.run(eps0, sig0)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    its = len(hist.seconds)
    evals, passes = sum(hist.evaluations), sum(hist.passes)
    grads, misfits = passes - evals, 2 * evals - passes
    t = fd.tiling()
    nl = -(-g.nt // t.steps)
    k_eff = g.nt / nl
    b_mis = nl * algorithmic_bytes_per_launch("fwd", wl, k_eff, 0.0)
    b_grad = nl * (algorithmic_bytes_per_launch("fwd", wl, k_eff, 1.0)
                   + algorithmic_bytes_per_launch("adj", wl, k_eff))
    sec = sum(hist.seconds)
    peak, peak_kind = hbm_peak()
    achieved = (grads * b_grad + misfits * b_mis) / sec / 1e9
    err = lambda e: float(torch.linalg.vector_norm(e - eps_t) / torch.linalg.vector_norm(eps_t))
    return {"bands": [[f, i] for f, i in zip(freqs, iters)], "tv": True,
            "iterations": its, "s_per_iteration": sec / max(1, its), "wall_s": wall,
            "evaluations_per_iteration": evals / max(1, its),
            "forward_equivalent_passes_per_iteration": passes / max(1, its),
            "gradients": grads, "misfit_only_forwards": misfits,
            "misfit_first_last": [hist.misfit[0], hist.final_misfit] if hist.misfit else None,
            "eps_rel_error_start_end": [err(eps0), err(eps)],
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": f"hbm_gbs of {peak_kind}",
                         "meaning": "algorithmic bytes of every FDTD time loop of the "
                                    "iterations / their wall time (L-BFGS algebra, TV and "
                                    "line search included in the time)"}}


# TE forward, bytes per cell and step that a design with one H launch and one E launch per
# step must move: the H launch reads Ex, Ey, Hz and writes Hz (16 B), the E launch reads Hz,
# Ex, Ey and writes Ex, Ey (20 B); Ca, Cb (one plane pair for all shots) stay in L2, the
# CPML memories are touched in the strips only (not counted).
TE_BYTES_PER_CELL_STEP = 36.0
# TE gradient, per cell and step: the forward above plus its Ex, Ey history writes (8 B), and
# the adjoint's four launches: E reversed (reads aEx, aEy and Ex, Ey of two steps, writes
# aEx, aEy and two difference cotangents, updates two gradient planes: 56 B), Hz reversed
# (reads aHz and two cotangent planes, writes aHz and two: 24 B), gather (reads aEx, aEy and
# two cotangent planes, writes aEx, aEy: 24 B).
TE_GRAD_BYTES_PER_CELL_STEP = TE_BYTES_PER_CELL_STEP + 8.0 + 56.0 + 24.0 + 24.0


def te_leg(args, dev) -> dict:
    """The TE-mode forward model (x-directed sources: Ex, Ey, Hz at the receivers) on the
    benchmark's workload.  One warm-up call, three timed with CUDA events on the launching
    stream around whole calls (2 nt launches, the field clears and the coefficient kernel)."""
    import torch
    from paper_2506_20513_gb300 import FDTD
    from paper_2506_20513_gb300.fdtd import ricker
    wl = workload(0, args.nshots, args.nt, "multishot")
    g = wl.grid
    fd = FDTD(g, wl.src, wl.rec, device=dev)
    t32 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    wav = t32(np.broadcast_to(ricker(wl.f0, g.dt, g.nt), (wl.nshots, 1, g.nt)))
    e, s = t32(wl.eps_true), t32(wl.sig_true)
    fd.forward_model_te(e, s, wav, 0)
    torch.cuda.synchronize(dev)
    l0 = fd.lib.gf_kernel_launches(fd.ctx)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    ev0.record()
    for _ in range(reps):
        fd.forward_model_te(e, s, wav, 0)
    ev1.record()
    torch.cuda.synchronize(dev)
    ms = ev0.elapsed_time(ev1) / reps
    launches = (fd.lib.gf_kernel_launches(fd.ctx) - l0) // reps
    fd.status()
    cell_steps = wl.nshots * g.nt * (g.nx - 1) * (g.ny - 1)   # cells each step updates
    peak, kind = hbm_peak()
    achieved = TE_BYTES_PER_CELL_STEP * cell_steps / (ms / 1e3) / 1e9
    # the gradient at the smoothed start model for data of the true model (one warm-up call,
    # two timed); its E history is held by the context (nt x 2 planes per shot)
    grad = None
    try:
        obs = fd.forward_model_te(e, s, wav, 0)[..., 0].contiguous()
        e0, s0 = t32(wl.eps_init), t32(wl.sig_init)
        fd.misfit_and_gradient_te(e0, s0, wav, obs, 0)
        torch.cuda.synchronize(dev)
        ev0.record()
        for _ in range(2):
            J, _, _ = fd.misfit_and_gradient_te(e0, s0, wav, obs, 0)
        ev1.record()
        torch.cuda.synchronize(dev)
        gms = ev0.elapsed_time(ev1) / 2
        fd.status()
        ga = TE_GRAD_BYTES_PER_CELL_STEP * cell_steps / (gms / 1e3) / 1e9
        grad = {"s_per_gradient": gms / 1e3, "misfit": float(J.item()),
                "gcell_updates_per_s": 2 * wl.nshots * g.nt * g.ncells / gms / 1e6,
                "history_gb": 2 * g.nt * wl.nshots * g.ny * ((g.nx + 3) // 4 * 4) * 4 / 1e9,
                "roofline": {"bound": "hbm", "achieved": ga, "peak": peak, "unit": "GB/s",
                             "frac": ga / peak, "traffic": None,
                             "kernel": "TE forward with history + four adjoint launches per "
                                       "step (whole calls)",
                             "algorithmic_bytes_per_cell_step": TE_GRAD_BYTES_PER_CELL_STEP}}
    except Exception as ex:  # noqa: BLE001 -- reported in the record, not fatal to the bench
        grad = {"error": f"{type(ex).__name__}: {ex}"}
    fd.close()
    return {"workload": f"{wl.name}_te_x", "grid": f"{g.nx}x{g.ny}", "nshots": wl.nshots,
            "nt": g.nt, "nrec": wl.nrec, "polarisation": "x (traces of Ex, Ey, Hz)",
            "ms_per_forward": ms,
            "gcell_updates_per_s": wl.nshots * g.nt * g.ncells / ms / 1e6,
            "launches_per_forward": int(launches), "steps": reps, "warmup": 1,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "te_h_kernel + te_e_kernel (whole calls)",
                         "peak_source": f"hbm_gbs of {kind}",
                         "algorithmic_bytes_per_cell_step": TE_BYTES_PER_CELL_STEP},
            "gradient": grad}


def large_leg(args, dev, sms: int) -> dict:
    """The large-grid checkpointed gradient: 2108x1084 cells (30-cell CPML inside), 16 shots,
    nt 8000, 400 receivers, forward wavefield checkpointed every ``args.large_checkpoint``
    steps and recomputed per segment.  One warm-up gradient, two timed, one profiled."""
    import torch
    from paper_2506_20513_gb300 import FDTD
    from paper_2506_20513_gb300.fdtd import ricker
    wl = workload(0, 16, 8000, "large")
    g = wl.grid
    k = args.large_checkpoint
    fd = FDTD(g, wl.src, wl.rec, device=dev)
    fd.set_storage(k)
    t32 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    wav = t32(np.broadcast_to(ricker(wl.f0, g.dt, g.nt), (wl.nshots, 1, g.nt)))
    obs = fd.forward_model(t32(wl.eps_true), t32(wl.sig_true), wav)
    e0, s0 = t32(wl.eps_init), t32(wl.sig_init)
    fd.misfit_and_gradient(e0, s0, wav, obs)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 2
    ev0.record()
    for _ in range(reps):
        fd.misfit_and_gradient(e0, s0, wav, obs)
    ev1.record()
    torch.cuda.synchronize(dev)
    ms = ev0.elapsed_time(ev1) / reps
    fd.lib.gf_profile(fd.ctx, 1)
    fd.misfit_and_gradient(e0, s0, wav, obs)
    torch.cuda.synchronize(dev)
    span_all = read_tile_span(fd.lib, fd.ctx)
    prof = read_profile(fd.lib, fd.ctx)
    fd.lib.gf_profile(fd.ctx, 0)
    clk = clocks.stop()
    fd.status()
    t = fd.tiling()
    rec = {"workload": wl.name, "grid": f"{g.nx}x{g.ny}", "npml": g.npml, "nshots": wl.nshots,
           "nt": g.nt, "nrec": wl.nrec, "checkpoint_every": k,
           "s_per_gradient": ms / 1e3, "gcell_updates_per_s": wl.cell_updates() / ms / 1e6,
           "workspace_gb": fd.workspace_bytes() / 1e9,
           "tiling": f"{t.tile_w}x{t.tile_h}, K {t.steps}, variant {t.variant}",
           "steps": reps, "warmup": 1, "clocks": clk,
           "roofline": dict(path_roofline(span_all, wl, 1, t.steps, k),
                            phase_ms_per_step={kk: v[0] for kk, v in prof.items()})}
    fd.close()
    return rec


def ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    from paper_2506_20513_gb300 import FDTD, Tiling
    from paper_2506_20513_gb300.fdtd import ricker

    if args.workload == "large":
        if args.nt == 2000:
            args.nt = 8000
        if args.checkpoint <= 0:
            args.checkpoint = 100
        # the FP64 oracle would need ~146 GB of host memory per shot for this grid
        args.no_cpu_baseline = True
        args.no_large = True
    if args.workload in ("disc", "precond"):
        # the single-shot disc model (100 x 100 + 10-cell CPML, nt 600) and the learned
        # preconditioner's workload (256 x 128 + 20-cell CPML, 16 shots, nt 1500): working
        # sets that L2 holds, so latency, not HBM, is the binding roof
        if args.workload == "precond" and args.nt == 2000:
            args.nt = 1500
        args.no_large = True
        args.fwi_iters = 0
    wl = workload(rank, args.nshots, args.nt, args.workload, world)
    g = wl.grid
    tiling = Tiling(*[int(x) for x in args.tile.split(",")]) if args.tile else None
    fd = FDTD(g, wl.src, wl.rec, device=dev, tiling=tiling)
    fd.lib.gf_set_lanes(fd.ctx, args.lanes)
    if args.checkpoint > 0:
        fd.set_storage(args.checkpoint, reconstruct=args.reconstruct)
    t32 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    wav = t32(np.broadcast_to(ricker(wl.f0, g.dt, g.nt), (wl.nshots, 1, g.nt)))
    eps_t, sig_t = t32(wl.eps_true), t32(wl.sig_true)
    eps0, sig0 = t32(wl.eps_init), t32(wl.sig_init)
    obs = fd.forward_model(eps_t, sig_t, wav)
    fd.status()

    from paper_2506_20513_gb300.shard import allreduce_sum

    def step():
        # this rank's shots, then the sum over the ranks (the identity on one GPU)
        return allreduce_sum(*fd.misfit_and_gradient(eps0, sig0, wav, obs))

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
    span_all = read_tile_span(lib, ctx)
    prof = read_profile(lib, ctx)
    lib.gf_profile(ctx, 0)
    # the same again with the shots in one lane: the dominant kernel alone on the GPU
    prof1 = None
    if lanes_used(fd, args) > 1:
        lib.gf_set_lanes(ctx, 1)
        lib.gf_profile(ctx, 1)
        for _ in range(args.steps):
            step()
        barrier()
        prof1 = read_profile(lib, ctx)
        lib.gf_profile(ctx, 0)
        lib.gf_set_lanes(ctx, args.lanes)
    clk = clocks.stop()
    fd.status()
    ms = reduce_max(ms, dev)
    cells = wl.cell_updates() * args.steps * world
    value = job_value(wl.cell_updates() * args.steps, world, ms)
    t = fd.tiling()
    tiling_key = args.tile or "default"
    hist = 0.5 if args.checkpoint else 1.0
    kernel_roof = tile_roofline(prof1 or prof, wl, args.steps, hist, tiling_key, clk, sms,
                                t.steps, args.checkpoint)
    if prof1 is None:
        roof = kernel_roof
    else:
        # the lanes run the forward and adjoint kernels concurrently: the roofline of the two
        # together over the time they kept the GPU busy, and the dominant kernel alone (one
        # lane) beside it
        roof = path_roofline(span_all, wl, args.steps, t.steps, args.checkpoint, tiling_key)
        roof["phase_ms_per_step"] = {k: v[0] / args.steps for k, v in prof.items()}
        roof["dominant_kernel_one_lane"] = kernel_roof
    peak = roof["peak"]
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

        def e2e_step():
            if world == 1:
                return fd.misfit_and_gradient(he, hs, hw, ho)
            d = lambda x: x.to(dev, non_blocking=True)
            out = allreduce_sum(*fd.misfit_and_gradient(d(he), d(hs), d(hw), d(ho)))
            return tuple(x.cpu() for x in out)

        e2e_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            Jh, geh, gsh = e2e_step()
        barrier()
        te = reduce_max(time.perf_counter() - t0, dev)
        h2d = sum(x.numel() * x.element_size() for x in (he, hs, hw, ho))
        d2h = Jh.numel() * 8 + geh.numel() * 4 + gsh.numel() * 4
        e2e = {"value": cells / te / 1e9, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    # seconds per dual-parameter FWI iteration, and the large-grid checkpointed gradient
    # (on one GPU only: a multi-GPU run reports the scaling of the gradient step alone)
    fwi = None
    if args.fwi_iters > 0 and world == 1 and args.workload == "multishot":
        fwi = fwi_leg(args, fd, wl, eps_t, sig_t, eps0, sig0)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        shots = cpu_sample_shots(args.cpu_shots, wl.nshots)
        v, tcpu = run_oracle_sample(wl, shots)
        cpu = {"value": v, "unit": UNIT, "cores": shots, "nproc": host_cores(),
               "kind": "oracle", "sample": oracle_sample_text(wl, shots, tcpu)}
    workspace_gb = fd.workspace_bytes() / 1e9
    fd.close()
    large = None
    if not args.no_large and world == 1:
        large = large_leg(args, dev, sms)
    te_rec = None
    if not args.no_te and world == 1 and args.workload == "multishot" and not args.checkpoint:
        torch.cuda.empty_cache()   # the earlier legs' workspaces: room for the TE history
        te_rec = te_leg(args, dev)

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
                       "tiling": (f"{t.tile_w}x{t.tile_h}, K {t.steps}, variant {t.variant}"
                                  + (" (--tile)" if args.tile else " (default)")),
                       "l2": "inputs larger than L2: each step streams the "
                             f"{wl.nshots * g.nt * g.ncells * 4 / 1e9:.1f} GB wavefield "
                             "through HBM" if not args.checkpoint else
                             "inputs larger than L2: checkpoints and segment buffers of "
                             f"{workspace_gb:.1f} GB",
                       "storage": (f"checkpoint every {args.checkpoint} steps"
                                   + (", segments reconstructed backwards from a boundary ring"
                                      if args.reconstruct else "")
                                   if args.checkpoint else "full wavefield"),
                       "workspace_gb": workspace_gb,
                       "parallelism": (f"{wl.nshots * world} shots split round-robin over "
                                       f"{world} GPUs, (J, g_eps, g_sigma) summed by an NCCL "
                                       "all-reduce every step" if world > 1 else
                                       "one GPU, all shots"),
                       "fwi": fwi,
                       "binding_roof": ("L2 / latency: the working set fits in L2, HBM is "
                                        "not the binding roof"
                                        if args.workload in ("disc", "precond") else "HBM")},
            "roofline": roof, "large": large, "te": te_rec, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": gpu_launches, "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def uneven(args):
    """64 independent instances of uneven size (128-768 x 128-384 cells + 20-cell CPML, nt
    800-3000, 1-8 shots, checkpoints every 100 steps), each tuned by the autotuner, one
    gradient each per step: one after the other, concurrently as one replayed CUDA graph of
    per-instance streams, and as the persistent multi-instance schedule (the instances'
    persistent passes merged into single cooperative launches, replayed as one CUDA graph)."""
    import tempfile

    import torch
    from paper_2506_20513_gb300 import FDTD, FDTDBatch, Tiling, autotune, workloads as W
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
    cols = [list(x) for x in zip(*ins)]
    cells = sum(w.cell_updates() for w in insts)

    def timed(batch, mode):
        for _ in range(max(1, args.warmup)):
            batch.misfit_and_gradient(*cols, mode=mode)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            batch.misfit_and_gradient(*cols, mode=mode)
        e1.record()
        torch.cuda.synchronize(dev)
        for fd in fds:
            fd.status()
        return e0.elapsed_time(e1) / args.steps

    def tilings():
        out = {}
        for fd in fds:
            t = fd.tiling()
            key = f"{t.tile_w}x{t.tile_h}/K{t.steps}/v{t.variant}"
            out[key] = out.get(key, 0) + 1
        return out

    # the autotuned tilings: one instance after the other, and the graph of their streams
    batch = FDTDBatch(fds)
    out = {0: timed(batch, 0), 2: timed(batch, 2)}
    tuned = tilings()
    batch.close()
    # the persistent multi-instance schedule: every instance on the persistent variant with
    # its tuned time-block depth, the passes of all instances merged into single launches
    for fd in fds:
        fd.set_tiling(Tiling(0, 0, fd.tiling().steps, 3))
    batch = FDTDBatch(fds)
    flow_seq = timed(batch, 0)
    out[4] = timed(batch, 4)
    out[3] = timed(batch, 3)
    line = {"metric": METRIC + " (uneven-instance batch)", "value": cells / (out[4] / 1e3) / 1e9,
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": out[4], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{len(insts)} uneven instances (128-768 x 128-384 + CPML, "
                                   "nt 800-3000, 1-8 shots), checkpoint every 100 steps",
                       "cell_updates_per_step": cells,
                       "ms_sequential_tuned": out[0], "ms_stream_graph_tuned": out[2],
                       "ms_sequential_persistent_variant": flow_seq,
                       "ms_merged_persistent": out[3], "ms_merged_persistent_graph": out[4],
                       "speedup_vs_sequential_tuned": out[0] / out[4],
                       "speedup_stream_graph_vs_sequential": out[0] / out[2],
                       "autotune_s": t_tune, "tilings_chosen": tuned,
                       "tilings_persistent": tilings()}}
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
