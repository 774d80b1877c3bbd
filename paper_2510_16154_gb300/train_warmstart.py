"""Train and evaluate the warm-start network on solves the method itself generates.

    python -m paper_2510_16154_gb300.train_warmstart [--n-train 1536] [--size 256]
        [--epochs 30] [--out FILE.npz] [--eval-n 8] [--eval-size 1024] [--json FILE]

1. Training set: n synthetic RGB images (Voronoi regions K ~ U{4..32}, linear ramp 0.1,
   noise sigma ~ U[0.02, 0.15]) of size x size, each solved to a relative residual of
   1e-4 by the batched solve (agents_solve_batch, CUDA graphs, autotuned tiles) from the
   cold start (mu = 0, eps = 57).  Targets: the converged dual field mu* and log eps*.
2. Training: Adam on the library's forward/backward kernels (loss: mean squared error on
   mu plus 0.1 x mean squared error on log eps).
3. Evaluation on unseen images of the same generator: the whole set as one batched
   solve (agents_solve_batch) to 1e-4, cold, warm-started from the network's mu, and from
   its mu and eps; a subset one by one through solve() with per-image multiplier steps,
   device time, the network's own time and the largest difference between the warm and
   the cold answer; and a few images at a higher resolution than the training set.
   The fallback to the cold start is taken on divergence.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np
import torch

from . import _lib as lib
from .warmstart import NetSpec, WarmStartNet, WEIGHTS_DIR

R, T = 5, 20
TOL = 1e-4
K_IN = 10


def image_spec(rng, size):
    from synth import ImageSpec
    return ImageSpec(size, size, 3, regions=int(rng.integers(4, 33)), ramp=0.1,
                     sigma=float(rng.uniform(0.02, 0.15)))


def make_images(n, size, seed, dev):
    from synth import make_image
    rng = np.random.default_rng(seed)
    out = torch.empty(n, size, size, 3, dtype=torch.float32, device=dev)
    for i in range(n):
        out[i] = torch.from_numpy(make_image(image_spec(rng, size), seed * 100003 + i)
                                  .astype(np.float32)).to(dev)
    return out


def solve_targets(imgs, k_out, chunk, stream, log):
    """Cold-start batched solves to TOL; returns mu* [n,H,W,6], log eps* [n,2T], infos."""
    n, H, W, C = imgs.shape
    mu_all = torch.empty(n, H, W, 2 * C, dtype=torch.float32, device=imgs.device)
    le_all = torch.empty(n, 2 * T, dtype=torch.float32, device=imgs.device)
    outer = []
    o = lib.agents_default_solve_opts()
    o.k_out, o.k_in, o.tol = k_out, K_IN, TOL
    for b in range(0, n, chunk):
        m = min(chunk, n - b)
        ctxs, eps, mus = [], [], []
        for i in range(b, b + m):
            p = lib.agents_default_params(H, W, C, R, T)
            ctxs.append(lib.Context(p, imgs[i].contiguous(), stream))
            eps.append(torch.full((T, 2), 57.0, dtype=torch.float64, device=imgs.device))
            mus.append(torch.zeros(H, W, 2, C, dtype=torch.float32, device=imgs.device))
        t0 = time.perf_counter()
        infos = lib.agents_solve_batch([c.handle for c in ctxs], o, eps, mus, None,
                                       autotune=True, use_graph=True)
        torch.cuda.synchronize()
        for k, i in enumerate(range(b, b + m)):
            mu_all[i] = mus[k].reshape(H, W, 2 * C)
            le_all[i] = torch.log(eps[k].reshape(-1)).float()
            outer.append(infos[k].outer_done)
        for c in ctxs:
            c.close()
        if log:
            log(f"solved {b + m}/{n} ({time.perf_counter() - t0:.1f} s for {m}; "
                f"multiplier steps mean {np.mean(outer[-m:]):.1f})")
    return mu_all, le_all, outer


def evaluate(net, n, size, seed, stream, log, k_out=150, per_image=True):
    from .warmstart import warm_solve
    dev = net.device
    imgs = make_images(n, size, seed, dev)
    o = lib.agents_default_solve_opts()
    o.k_out, o.k_in, o.tol = k_out, K_IN, TOL
    rows = []
    for i in range(n if per_image else 0):
        img = imgs[i].contiguous()
        p = lib.agents_default_params(size, size, 3, R, T)
        with lib.Context(p, img, stream) as ctx:
            res = {}
            for mode in ("cold", "warm", "warm_mu"):
                c_out = torch.empty(size, size, 3, dtype=torch.float32, device=dev)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                t_net = 0.0
                if mode == "cold":
                    eps = torch.full((T, 2), 57.0, dtype=torch.float64, device=dev)
                    mu = torch.zeros(size, size, 2, 3, dtype=torch.float32, device=dev)
                    info = lib.solve(ctx.handle, o, eps, mu, None, c_out)
                    fb = False
                else:
                    ts = time.perf_counter()
                    net.predict(img)                     # time of the network alone
                    torch.cuda.synchronize()
                    t_net = time.perf_counter() - ts
                    t0 = time.perf_counter()
                    info, eps, mu, fb = warm_solve(ctx.handle, net, img, o,
                                                   use_eps=(mode == "warm"), c_out=c_out)
                torch.cuda.synchronize()
                t = time.perf_counter() - t0
                res[mode] = {"outer": info.outer_done, "inner": info.inner_done,
                             "trials": info.trials, "seconds": t, "net_seconds": t_net,
                             "final_res": info.final_res, "final_obj": info.final_obj,
                             "fallback": fb, "c": c_out}
            for mode in ("warm", "warm_mu"):
                res[mode]["max_abs_dc_vs_cold"] = float((res[mode]["c"] - res["cold"]["c"])
                                                        .abs().max())
            for mode in res:
                del res[mode]["c"]
        rows.append(res)
        if log:
            log(f"eval {i + 1}/{n}: " + ", ".join(
                f"{m} {r['outer']} steps {r['seconds']:.2f}s" for m, r in res.items()))
    # the same images as one batched solve (CUDA graphs), cold and warm
    batch = {}
    ctxs = [lib.Context(lib.agents_default_params(size, size, 3, R, T), imgs[i].contiguous(),
                        stream) for i in range(n)]
    try:
        for mode in ("cold", "warm_mu", "warm"):
            eps = [torch.full((T, 2), 57.0, dtype=torch.float64, device=dev) for _ in range(n)]
            mus = [torch.zeros(size, size, 2, 3, device=dev) for _ in range(n)]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if mode != "cold":
                mu_p, eps_p = net.predict(imgs)
                if mode == "warm":
                    eps = [eps_p[i].contiguous() for i in range(n)]
                mus = [mu_p[i].reshape(size, size, 2, 3).contiguous() for i in range(n)]
            infos = lib.agents_solve_batch([c.handle for c in ctxs], o, eps, mus, None,
                                           autotune=True, use_graph=True)
            torch.cuda.synchronize()
            batch[mode] = {"seconds": time.perf_counter() - t0,
                           "outer_mean": float(np.mean([i.outer_done for i in infos])),
                           "outer": [i.outer_done for i in infos],
                           "reached_tol": int(sum(i.final_res < TOL for i in infos)),
                           "final_obj_mean": float(np.mean([i.final_obj for i in infos]))}
            if log:
                log(f"batched {mode}: {batch[mode]['seconds']:.2f} s, multiplier steps mean "
                    f"{batch[mode]['outer_mean']:.1f}, reached tol {batch[mode]['reached_tol']}"
                    f"/{n}, mean final L~ {batch[mode]['final_obj_mean']:.4f}")
    finally:
        for c in ctxs:
            c.close()
    summary = {"batched": batch}
    for mode in ("cold", "warm", "warm_mu") if rows else ():
        summary[mode] = {
            "outer_mean": float(np.mean([r[mode]["outer"] for r in rows])),
            "inner_mean": float(np.mean([r[mode]["inner"] for r in rows])),
            "seconds_mean": float(np.mean([r[mode]["seconds"] for r in rows])),
            "net_seconds_mean": float(np.mean([r[mode]["net_seconds"] for r in rows])),
            "reached_tol": int(sum(r[mode]["final_res"] < TOL for r in rows)),
            "final_obj_mean": float(np.mean([r[mode]["final_obj"] for r in rows])),
            "fallbacks": int(sum(r[mode]["fallback"] for r in rows))}
        if mode != "cold":
            summary[mode]["max_abs_dc_vs_cold"] = float(max(r[mode]["max_abs_dc_vs_cold"]
                                                            for r in rows))
    return {"images": n, "size": size, "per_image": rows, "summary": summary}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-train", type=int, default=1536)
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--k-out", type=int, default=40)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--base", type=int, default=32)
    ap.add_argument("--levels", type=int, default=4)
    ap.add_argument("--out", default=os.path.join(WEIGHTS_DIR, "warmstart_rgb_T20_R5.npz"))
    ap.add_argument("--init", default=None, help="start from these weights instead of a seed")
    ap.add_argument("--eval-n", type=int, default=64)
    ap.add_argument("--eval-size", type=int, default=256)
    ap.add_argument("--eval-per-image", type=int, default=16,
                    help="also solve this many of the eval images one by one (3 modes)")
    ap.add_argument("--xres-n", type=int, default=4, help="cross-resolution eval images")
    ap.add_argument("--xres-size", type=int, default=1024)
    ap.add_argument("--json", default=None)
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args(argv)

    def log(msg):
        print(msg, flush=True)

    from .build import build
    build()
    lib.load()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    report = {"R": R, "T": T, "tol": TOL, "k_in": K_IN}
    if args.n_train > 0:
        t0 = time.perf_counter()
        imgs = make_images(args.n_train, args.size, 1 + args.seed, dev)
        log(f"made {args.n_train} images in {time.perf_counter() - t0:.1f} s")
        t0 = time.perf_counter()
        mu_t, le_t, outer = solve_targets(imgs, args.k_out, 96, stream, log)
        t_solve = time.perf_counter() - t0
        zero_loss = float((mu_t.double() ** 2).mean() +
                          0.1 * ((le_t.double() - math.log(57.0)) ** 2).mean())
        log(f"loss of the cold start (mu = 0, eps = 57) on the targets: {zero_loss:.5f}")
        net = WarmStartNet(NetSpec(nsteps=T, base=args.base, levels=args.levels), dev, stream)
        if args.init:
            net.set_params(WarmStartNet.load(args.init, dev, stream).get_params())
        else:
            net.init_params(args.seed)
        t0 = time.perf_counter()
        hist = net.fit(imgs, mu_t, le_t, epochs=args.epochs, batch=args.batch, lr=args.lr,
                       seed=args.seed, log=log)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
        net.save(args.out)
        report["train"] = {"images": args.n_train, "size": args.size,
                           "solve_seconds": t_solve, "outer_mean": float(np.mean(outer)),
                           "reached_k_out": int(sum(x >= args.k_out for x in outer)),
                           "epochs": args.epochs, "batch": args.batch, "lr": args.lr,
                           "train_seconds": t_train, "loss_cold_start": zero_loss,
                           "loss_first": hist[0],
                           "loss_last": hist[-1], "weights": os.path.basename(args.out)}
        del imgs, mu_t, le_t
        torch.cuda.empty_cache()
    else:
        net = WarmStartNet.load(args.out, dev, stream)
    if args.eval_n > 0:
        report["eval"] = evaluate(net, args.eval_n, args.eval_size, 900 + args.seed, stream, log,
                                  k_out=args.k_out, per_image=False)
        log(json.dumps(report["eval"]["summary"]))
    if args.eval_per_image > 0:
        report["eval_per_image"] = evaluate(net, args.eval_per_image, args.eval_size,
                                            900 + args.seed, stream, log, k_out=args.k_out)
        log(json.dumps(report["eval_per_image"]["summary"]))
    if args.xres_n > 0:
        report["eval_xres"] = evaluate(net, args.xres_n, args.xres_size, 950 + args.seed, stream,
                                       log, k_out=150)
        log(json.dumps(report["eval_xres"]["summary"]))
    if args.json:
        with open(args.json, "w") as f:
            json.dump(report, f, indent=1)
    net.close()
    return 0


if __name__ == "__main__":
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    sys.exit(main())
