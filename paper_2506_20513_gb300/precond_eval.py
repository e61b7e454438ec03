"""Train the learned preconditioner on seeded random models and evaluate it in FWI.

    python -m paper_2506_20513_gb300.precond_eval --train 10000 --eval 100

Workload: 256 x 128 physical cells (+20-cell CPML), dx 0.01 m, 400 MHz Ricker, 16 shots
on the surface, 64 receivers, nt 1500 (the preconditioner workload generator, seeds
``--seed`` ...).  For each training model the FDTD/adjoint kernels compute the observed data
of the true model, the misfit gradient at the smoothed starting model and that model's
illumination; the U-Net (4 levels, 32 base channels, 4 in / 2 out, BF16 kernels) learns the
normalised true-minus-start update.  Evaluation on held-out seeds: plain L-BFGS for
``--iters`` iterations gives a target misfit; the learned-preconditioned run (network
update tried first, plain step as fallback) counts the iterations, FDTD evaluations and
wall time it needs to reach that misfit.  Prints one JSON line.

With ``--stage2 N`` a second network, initialised from the first, is fine-tuned on N further
models at the model the first network's update reaches (:func:`generate_stage_pairs`) and
proposes the band's learned updates after the first kept one; the evaluation then also runs
the first network alone on the same held-out models.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import workloads as W
from .fdtd import FDTD, ricker
from .fwi import FWI, FWIConfig, interior_mask
from .precond import (LearnedPreconditioner, PreconditionerScales, generate_pairs,
                      generate_stage_pairs, pair_fractions, seeded_models, train,
                      validation_loss)
from .unet import UNet


def _fwi(fd, wl, obs, f0, iters, pre=None, stop=None, retry=0, scales=(1.0, 0.5), most=2):
    cfg = FWIConfig(bands=((f0, iters),), learned_retry=retry, learned_scales=tuple(scales),
                    learned_max=most)
    mask = interior_mask(wl.grid, rows_below_top=4)
    inv = FWI(fd, lambda f: obs, mask, cfg, preconditioner=pre)
    e0 = torch.tensor(wl.eps_init, dtype=torch.float32, device=fd.device)
    s0 = torch.tensor(wl.sig_init, dtype=torch.float32, device=fd.device)
    torch.cuda.synchronize(fd.device)
    t0 = time.perf_counter()
    _, _, hist = inv.run(e0, s0, stop_misfit=stop)
    torch.cuda.synchronize(fd.device)
    return hist, time.perf_counter() - t0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--train", type=int, default=10000)
    ap.add_argument("--val", type=int, default=200)
    ap.add_argument("--eval", type=int, default=100)
    ap.add_argument("--iters", type=int, default=50)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=100000)
    ap.add_argument("--nt", type=int, default=1500)
    ap.add_argument("--workers", type=int, default=12, help="host processes generating models")
    ap.add_argument("--save", default=None, help="write the trained parameters (.npy)")
    ap.add_argument("--out", default=None, help="write the summary and per-model rows (JSON)")
    ap.add_argument("--load", default=None,
                    help="trained parameters (.npy) to evaluate instead of generating and training")
    ap.add_argument("--retry", type=int, default=0,
                    help="L-BFGS iterations after a rejected learned update before the network "
                         "is consulted again (0 = not again)")
    ap.add_argument("--scales", default="1,0.5", help="scales of the learned update tried in turn")
    ap.add_argument("--plain-from", default=None,
                    help="JSON of an earlier evaluation of the same models: reuse its plain "
                         "L-BFGS rows (the plain runs are deterministic) instead of rerunning them")
    ap.add_argument("--stage2", type=int, default=0,
                    help="models for a second network, used after the first kept learned update")
    ap.add_argument("--stage2-val", type=int, default=100)
    ap.add_argument("--stage2-epochs", type=int, default=20)
    ap.add_argument("--stage2-lr", type=float, default=3e-4)
    ap.add_argument("--save2", default=None, help="write the second network's parameters (.npy)")
    ap.add_argument("--load2", default=None,
                    help="second network's parameters (.npy) to evaluate instead of training it")
    ap.add_argument("--learned-max", type=int, default=2,
                    help="most learned updates kept per band (0 = no limit)")
    args = ap.parse_args(argv)
    dev = torch.device("cuda:0")
    first = W.preconditioner_model(args.seed, nt=args.nt)
    g = first.grid
    fd = FDTD(g, first.src, first.rec, device=dev)
    wav = torch.tensor(ricker(first.f0, g.dt, g.nt), device=dev)
    scales = PreconditionerScales()
    gen = lambda s: W.preconditioner_model(s, nt=args.nt)  # noqa: E731
    H, Wd = g.ny - 2 * g.npml, g.nx - 2 * g.npml
    seeds_train = np.arange(args.seed, args.seed + args.train)
    seeds_val = np.arange(args.seed + args.train, args.seed + args.train + args.val)
    seeds_eval = np.arange(args.seed + 10 ** 6, args.seed + 10 ** 6 + args.eval)

    net = UNet(4, 32, 4, 2, H, Wd, max_batch=args.batch, device=dev)
    t_gen = gpu_gen = t_tr = 0.0
    losses = [float("nan")]
    val0 = val1 = float("nan")
    if args.load:
        net.set_params(torch.from_numpy(np.load(args.load).astype(np.float32)).to(dev))
        args.train = args.val = args.epochs = 0
    else:
        t_gen, gpu_gen, t_tr, losses, val0, val1 = _train(args, fd, wav, scales, g, net,
                                                          seeds_train, seeds_val)
        if args.save:
            np.save(args.save, net.get_params().cpu().numpy())
    pre = LearnedPreconditioner(net, g.npml, scales)
    stage2 = None
    if args.load2:
        net2 = UNet(4, 32, 4, 2, H, Wd, max_batch=args.batch, device=dev)
        net2.set_params(torch.from_numpy(np.load(args.load2).astype(np.float32)).to(dev))
        stage2 = dict(stage2_loaded_params=args.load2)
    elif args.stage2 > 0:
        net2, stage2 = _train_stage2(args, fd, wav, scales, g, net, pre, first)
    if stage2 is not None:
        if args.save2 and not args.load2:
            np.save(args.save2, net2.get_params().cpu().numpy())
        stage2["single"] = pre
        pre = LearnedPreconditioner([net, net2], g.npml, scales)
        stage2["nets"] = (net, net2)
    return _evaluate(args, fd, wav, pre, net, gen, g, seeds_eval, t_gen, gpu_gen, t_tr, losses,
                     val0, val1, stage2)


def _train_stage2(args, fd, wav, scales, g, net, pre, first):
    """Pairs at the first network's updated model on further seeded models; the second
    network starts from the first's parameters."""
    dev = fd.device
    mask = interior_mask(g, rows_below_top=4)
    base = args.seed + 2 * 10 ** 6
    seeds = np.arange(base, base + args.stage2)
    seeds_val = np.arange(base + args.stage2, base + args.stage2 + args.stage2_val)
    t = time.perf_counter()
    X, T, gpu_gen = generate_stage_pairs(fd, seeded_models(seeds, args.nt, args.workers),
                                         len(seeds), wav, scales, g.npml, pre, mask)
    Xv, Tv, _ = generate_stage_pairs(fd, seeded_models(seeds_val, args.nt, args.workers),
                                     len(seeds_val), wav, scales, g.npml, pre, mask)
    t_gen = time.perf_counter() - t
    H, Wd = g.ny - 2 * g.npml, g.nx - 2 * g.npml
    net2 = UNet(4, 32, 4, 2, H, Wd, max_batch=args.batch, device=dev)
    net2.set_params(net.get_params().clone())
    val0 = validation_loss(net2, Xv, Tv, args.batch)
    torch.cuda.synchronize(dev)
    t = time.perf_counter()
    losses = train(net2, X, T, args.stage2_epochs, args.batch, args.stage2_lr,
                   seed=args.seed + 1, decay_every=max(1, args.stage2_epochs // 3))
    torch.cuda.synchronize(dev)
    t_tr = time.perf_counter() - t
    val1 = validation_loss(net2, Xv, Tv, args.batch)
    del X, T, Xv, Tv
    return net2, dict(stage2_models=args.stage2, stage2_val_models=args.stage2_val,
                      stage2_epochs=args.stage2_epochs, stage2_lr=args.stage2_lr,
                      stage2_pair_generation_s=t_gen, stage2_pair_generation_gpu_s=gpu_gen,
                      stage2_training_s=t_tr, stage2_train_loss_first_epoch=losses[0],
                      stage2_train_loss_last_epoch=losses[-1],
                      stage2_val_loss_before=val0, stage2_val_loss_after=val1)


def _train(args, fd, wav, scales, g, net, seeds_train, seeds_val):
    dev = fd.device
    t_gen = time.perf_counter()
    X, T, gpu_gen = generate_pairs(fd, seeded_models(seeds_train, args.nt, args.workers),
                                   len(seeds_train), wav, scales, g.npml,
                                   fractions=pair_fractions(seeds_train))
    Xv, Tv, _ = generate_pairs(fd, seeded_models(seeds_val, args.nt, args.workers),
                               len(seeds_val), wav, scales, g.npml,
                               fractions=pair_fractions(seeds_val))
    t_gen = time.perf_counter() - t_gen
    net.init_params(args.seed)
    val0 = validation_loss(net, Xv, Tv, args.batch)
    torch.cuda.synchronize(dev)
    t_tr = time.perf_counter()
    losses = train(net, X, T, args.epochs, args.batch, args.lr, seed=args.seed,
                   decay_every=max(1, args.epochs // 3))
    torch.cuda.synchronize(dev)
    t_tr = time.perf_counter() - t_tr
    val1 = validation_loss(net, Xv, Tv, args.batch)
    return t_gen, gpu_gen, t_tr, losses, val0, val1


def _evaluate(args, fd, wav, pre, net, gen, g, seeds_eval, t_gen, gpu_gen, t_tr, losses, val0,
              val1, stage2=None):
    dev = fd.device
    rows = []
    plain = {}
    if args.plain_from:
        with open(args.plain_from) as f:
            plain = {r["seed"]: r for r in json.load(f)["rows"]}
    for s in seeds_eval:
        wl = gen(int(s))
        obs = fd.forward_model(torch.tensor(wl.eps_true, dtype=torch.float32, device=dev),
                               torch.tensor(wl.sig_true, dtype=torch.float32, device=dev), wav)
        if int(s) in plain:
            p = plain[int(s)]
        else:
            h_plain, t_plain = _fwi(fd, wl, obs, wl.f0, args.iters)
            p = dict(J0=h_plain.misfit[0] if h_plain.misfit else None,
                     J_plain=h_plain.final_misfit, it_plain=len(h_plain.misfit),
                     ev_plain=int(sum(h_plain.evaluations)),
                     passes_plain=int(sum(h_plain.passes)), s_plain=t_plain)
        target = p["J_plain"]
        h_l, t_l = _fwi(fd, wl, obs, wl.f0, args.iters, pre=pre, stop=target, retry=args.retry,
                        scales=[float(v) for v in args.scales.split(",")],
                        most=args.learned_max)
        one = {}
        if stage2 is not None:
            h_1, t_1 = _fwi(fd, wl, obs, wl.f0, args.iters, pre=stage2["single"], stop=target,
                            retry=args.retry, scales=[float(v) for v in args.scales.split(",")],
                            most=args.learned_max)
            one = dict(it_learned1=len(h_1.misfit), ev_learned1=int(sum(h_1.evaluations)),
                       passes_learned1=int(sum(h_1.passes)), s_learned1=t_1,
                       reached1=bool(h_1.final_misfit <= target),
                       learned_accepted1=int(sum(h_1.learned)))
        rows.append(dict(seed=int(s), J0=p["J0"], J_plain=target, it_plain=p["it_plain"],
                         ev_plain=p["ev_plain"], passes_plain=p.get("passes_plain"),
                         s_plain=p["s_plain"],
                         J_learned=h_l.final_misfit, it_learned=len(h_l.misfit),
                         ev_learned=int(sum(h_l.evaluations)),
                         passes_learned=int(sum(h_l.passes)), s_learned=t_l,
                         reached=bool(h_l.final_misfit <= target),
                         learned_accepted=int(sum(h_l.learned)), **one))
    reached = [r for r in rows if r["reached"]]
    out = {
        "workload": f"precond_{g.nx}x{g.ny}_16shots_nt{g.nt}",
        "train_models": args.train, "val_models": args.val, "eval_models": args.eval,
        "loaded_params": args.load, "learned_retry": args.retry, "learned_scales": args.scales,
        "learned_max": args.learned_max,
        "plain_rows_from": args.plain_from,
        "epochs": args.epochs, "batch": args.batch,
        "pair_generation_s": t_gen, "pair_generation_gpu_s": gpu_gen,
        "training_s": t_tr, "train_loss_first_epoch": losses[0], "train_loss_last_epoch": losses[-1],
        "val_loss_before": val0, "val_loss_after": val1,
        "reached_fraction": len(reached) / max(len(rows), 1),
        "median_iters_plain": float(np.median([r["it_plain"] for r in rows])),
        "median_iters_learned": float(np.median([r["it_learned"] for r in rows])),
        "median_evals_plain": float(np.median([r["ev_plain"] for r in rows])),
        "median_evals_learned": float(np.median([r["ev_learned"] for r in rows])),
        # forward-equivalent time loops: a misfit-only evaluation 1, a gradient 2
        "median_passes_plain": (float(np.median([r["passes_plain"] for r in rows]))
                                if all(r["passes_plain"] is not None for r in rows) else None),
        "median_passes_learned": float(np.median([r["passes_learned"] for r in rows])),
        "median_s_plain": float(np.median([r["s_plain"] for r in rows])),
        "median_s_learned": float(np.median([r["s_learned"] for r in rows])),
        "learned_steps_accepted": int(sum(r["learned_accepted"] for r in rows)),
        "unet_kernel_launches": net.kernel_launches,
    }
    if stage2 is not None:
        out.update({k: v for k, v in stage2.items() if k not in ("single", "nets")})
        out["unet_kernel_launches"] = sum(n.kernel_launches for n in stage2["nets"])
        out.update({
            "first_network_alone": {
                "reached_fraction": sum(r["reached1"] for r in rows) / max(len(rows), 1),
                "median_iters": float(np.median([r["it_learned1"] for r in rows])),
                "median_evals": float(np.median([r["ev_learned1"] for r in rows])),
                "median_passes": float(np.median([r["passes_learned1"] for r in rows])),
                "median_s": float(np.median([r["s_learned1"] for r in rows])),
                "learned_steps_accepted": int(sum(r["learned_accepted1"] for r in rows)),
            }})
    out["train_loss_per_epoch"] = losses
    print(json.dumps(out))
    if args.out:
        with open(args.out, "w") as f:
            json.dump({"summary": out, "rows": rows}, f, indent=1)
    return out, rows


if __name__ == "__main__":
    main()
