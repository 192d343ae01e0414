"""Learned warm start for OS-LALM: dataset generation, training and
evaluation on the fan-beam geometry.

* scans: seeded random ellipse phantoms (water body plus 9 inner ellipses,
  attenuation 0-0.04 /mm) on the 512^2 / 984-view / 888-channel fan beam,
  I0 uniform in [2e4, 2e5], W = counts;
* input: the FBP image (clipped at 0); target: the OS-LALM image after
  `target_iters` iterations from the FBP image (M = 24, continuation), both
  computed with the library (the targets with the batched persistent path);
* network: the U-Net of oslalm_cnn (BF16 tensor-core training kernels),
  Adam, mean-squared error in units of mu_water;
* evaluation on held-out scans: x* from a decreasing-M schedule ending with
  the convergent one-subset method; OS-LALM (M = 24, continuation, FP16
  storage) from the FBP image and from the network's image; RMS difference
  to x* in the field of view after every iteration; iterations and seconds
  (CUDA events, network inference included) to reach each HU threshold.
Host orchestration only: every arithmetic step runs in liboslalm.
"""
from __future__ import annotations

import concurrent.futures as cf
import dataclasses
import math
import multiprocessing as mp
import os
import time

import numpy as np

from . import synth, workloads as W

SCALE = 1.0 / synth.MU_WATER  # network units: water = 1
HU = synth.HU


def scan_workload(seed: int, geom=None) -> W.Workload:
    base = W.c1_fan()
    g = geom if geom is not None else base.geom
    rng = np.random.default_rng(10_000 + seed)
    I0 = float(rng.uniform(2e4, 2e5))
    return dataclasses.replace(base, name=f"warm_{seed}", geom=g, phantom="ellipses", phantom_seed=20_000 + seed,
                               noise_seed=30_000 + seed, n_ellipses=10, fov_radius=0.96 * g.nx * g.dx / 2,
                               I0=I0, sigma=0.0, w_dtype="f16", d_dtype="f16")


def _scan(wl):
    sc = wl.make_scan()
    return sc["y"], sc["w"]


def make_scans(wls, workers=None):
    """Sinograms of the workloads (numpy, in a spawn-context process pool:
    call before the process touches the GPU)."""
    workers = workers or min(16, os.cpu_count() or 1)
    if workers <= 1:
        return [_scan(w) for w in wls]
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_scan, wls, chunksize=4))


def fov_mask(g):
    ix = (np.arange(g.nx) - (g.nx - 1) / 2.0) * g.dx
    iy = (np.arange(g.ny) - (g.ny - 1) / 2.0) * g.dy
    Y, X = np.meshgrid(iy, ix, indexing="ij")
    R = g.dso * math.sin(g.ns * g.ds / 2.0 / g.dsd)
    return (np.sqrt(X * X + Y * Y) <= R)[None]


def targets(oslalm, torch, geom, wls, scans, x0s, iters, chunk=64):
    """OS-LALM images after `iters` iterations from x0, with the batched path."""
    out = []
    dev = x0s[0].device
    for k in range(0, len(wls), chunk):
        probs, xs = [], []
        for wl, (y, w), x0 in zip(wls[k:k + chunk], scans[k:k + chunk], x0s[k:k + chunk]):
            p = oslalm.Problem(geom, torch.as_tensor(y, device=dev), torch.as_tensor(w, device=dev), beta=wl.beta,
                               delta=wl.delta, nbr=wl.nbr, M=wl.M, w_dtype=wl.w_dtype, d_dtype=wl.d_dtype,
                               use_graph=False)
            x = x0.clone()
            p.init(x)
            probs.append(p)
            xs.append(x)
        b = oslalm.Batch(probs)
        b.iterate(xs, iters, use_graph=False)
        torch.cuda.synchronize()
        out += xs
        b.close()
        for p in probs:
            p.close()
    return out


def reference_image(oslalm, torch, geom, wl, y, w, x0, schedule=((24, 60), (8, 60), (2, 100), (1, 800))):
    x = x0.clone()
    for M, n in schedule:
        p = oslalm.Problem(geom, y, w, beta=wl.beta, delta=wl.delta, nbr=wl.nbr, M=M, use_graph=True)
        p.init(x)
        p.iterate(x, n)
        p.close()
    return x


def train(oslalm, torch, net, xs, ts, epochs, lr, batch, seed=0, log=None):
    n = len(xs)
    rng = np.random.default_rng(seed)
    X = torch.stack(xs)
    T = torch.stack(ts)
    hist = []
    steps = 0
    t0 = time.time()
    for ep in range(epochs):
        perm = rng.permutation(n)
        lr_e = lr * 0.5 * (1 + math.cos(math.pi * ep / epochs))
        losses = []
        for k in range(0, n - batch + 1, batch):
            idx = torch.as_tensor(perm[k:k + batch], device=X.device)
            xb = X.index_select(0, idx).contiguous()
            tb = T.index_select(0, idx).contiguous()
            losses.append(net.train_step(xb, tb, SCALE, lr_e, want_loss=(k == 0)))
            steps += 1
        hist.append(float(losses[0]))
        if log:
            log(f"epoch {ep}: loss {losses[0]:.4e} lr {lr_e:.2e}")
    torch.cuda.synchronize()
    return hist, steps, time.time() - t0


def evaluate(oslalm, torch, geom, wls, scans, x0s, xstars, mask_np, init_fn=None, n_iter=50,
             thresholds=(20.0, 10.0, 5.0, 2.0, 1.0)):
    """Per scan: RMSD curve (HU) of OS-LALM from x0 (or init_fn(x0)), and the
    iterations / seconds to reach each threshold."""
    dev = x0s[0].device
    mask = torch.as_tensor(mask_np.astype(np.uint8), device=dev)
    stream = torch.cuda.current_stream()
    rows = []
    for wl, (y, w), x0, xs in zip(wls, scans, x0s, xstars):
        p = oslalm.Problem(geom, torch.as_tensor(y, device=dev), torch.as_tensor(w, device=dev), beta=wl.beta,
                           delta=wl.delta, nbr=wl.nbr, M=wl.M, w_dtype=wl.w_dtype, d_dtype=wl.d_dtype,
                           use_graph=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        x = init_fn(x0) if init_fn else x0.clone()
        p.init(x)
        e1.record(stream)
        e1.synchronize()
        t = e0.elapsed_time(e1)
        curve = [oslalm.rmsd(x, xs, mask) / HU]
        reached = {}
        for k in range(1, n_iter + 1):
            e0.record(stream)
            p.iterate(x, 1)
            e1.record(stream)
            e1.synchronize()
            t += e0.elapsed_time(e1)
            r = oslalm.rmsd(x, xs, mask) / HU
            curve.append(r)
            for th in thresholds:
                if th not in reached and r <= th:
                    reached[th] = (k, t / 1000.0)
        for th in thresholds:
            if th not in reached and curve[0] <= th:
                reached[th] = (0, 0.0)
        rows.append(dict(curve=curve, reached=reached))
        p.close()
    return rows


def summarize(rows, thresholds=(20.0, 10.0, 5.0, 2.0, 1.0)):
    out = {"rmsd_hu_iter0": float(np.mean([r["curve"][0] for r in rows])),
           "rmsd_hu_last": float(np.mean([r["curve"][-1] for r in rows])), "thresholds": {}}
    for th in thresholds:
        hit = [r["reached"][th] for r in rows if th in r["reached"]]
        out["thresholds"][f"{th:g}"] = {
            "reached": f"{len(hit)}/{len(rows)}",
            "mean_iterations": float(np.mean([h[0] for h in hit])) if hit else None,
            "mean_seconds": float(np.mean([h[1] for h in hit])) if hit else None,
        }
    return out


def experiment(n_train=256, n_test=16, target_iters=200, epochs=30, batch=8, lr=1e-3, geom=None, n_eval_iter=50,
               log=print):
    """The whole warm-start experiment; returns a JSON-ready dict."""
    wls_tr = [scan_workload(s, geom) for s in range(n_train)]
    wls_te = [scan_workload(100_000 + s, geom) for s in range(n_test)]
    t0 = time.time()
    scans_tr = make_scans(wls_tr)
    scans_te = make_scans(wls_te)
    t_scan = time.time() - t0
    import torch
    from . import oslalm
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    g = wls_tr[0].geom
    geomh = oslalm.Geometry(g)
    x0_tr = [geomh.fbp(torch.as_tensor(y, device=dev), clip=True) for y, _ in scans_tr]
    x0_te = [geomh.fbp(torch.as_tensor(y, device=dev), clip=True) for y, _ in scans_te]
    t0 = time.time()
    tg = targets(oslalm, torch, geomh, wls_tr, scans_tr, x0_tr, target_iters)
    torch.cuda.synchronize()
    t_targets = time.time() - t0
    net = oslalm.WarmStartNet(batch, g.ny, g.nx, seed=0)
    hist, steps, t_train = train(oslalm, torch, net, x0_tr, tg, epochs, lr, batch, log=log)
    flops = 3.0 * oslalm.WarmStartNet.flops_per_image(g.ny, g.nx) * batch * steps
    # inference net for one image at a time
    inf = oslalm.WarmStartNet(1, g.ny, g.nx, seed=0)
    inf.set_params(net.get_params())

    def cnn_init(x0):
        return torch.clamp(inf.forward(x0.view(1, g.ny, g.nx).contiguous(), SCALE).view(1, g.ny, g.nx), min=0.0)

    t0 = time.time()
    xstars = [reference_image(oslalm, torch, geomh, wl, torch.as_tensor(y, device=dev),
                              torch.as_tensor(w, device=dev), x0)
              for wl, (y, w), x0 in zip(wls_te, scans_te, x0_te)]
    t_ref = time.time() - t0
    mask = fov_mask(g)
    fbp_rows = evaluate(oslalm, torch, geomh, wls_te, scans_te, x0_te, xstars, mask, None, n_eval_iter)
    cnn_rows = evaluate(oslalm, torch, geomh, wls_te, scans_te, x0_te, xstars, mask, cnn_init, n_eval_iter)
    return {
        "train": {"scans": n_train, "target_iterations": target_iters, "epochs": epochs, "batch": batch,
                  "steps": steps, "seconds": t_train, "tflops": flops / t_train / 1e12,
                  "loss_first_last": [hist[0], hist[-1]]},
        "fbp_init": summarize(fbp_rows), "cnn_init": summarize(cnn_rows),
        "held_out": n_test,
        "seconds": {"scan_generation_cpu": t_scan, "targets_gpu": t_targets, "references_gpu": t_ref},
    }
