"""Learned warm start for OS-LALM: dataset generation, training and
evaluation on a 2D fan-beam geometry.

* scans: seeded random ellipse phantoms (10 ellipses, attenuation
  0-0.04 /mm) on the fan beam (512^2 image, 984 views, 888 channels at full
  size), I0 uniform in [2e4, 2e5], W = counts;
* input: the FBP image (clipped at 0); target: the OS-LALM image after
  `target_iters` iterations from the FBP image (continuation, FP16 storage
  of W and D), both computed by the library, the targets with the batched
  persistent path;
* network: the U-Net of oslalm_cnn (BF16 tensor-core training kernels),
  Adam with a cosine learning-rate decay, mean-squared error in units of
  the attenuation of water;
* evaluation on held-out scans: x* from a decreasing-M schedule that ends
  with the convergent one-subset method; OS-LALM from the FBP image and
  from the network's image (clipped at 0); RMS difference to x* in the
  field of view after every iteration; iterations and seconds (CUDA events,
  network inference included) to reach each HU threshold.

The minimiser is unchanged: the network only supplies x0, and FBP stays the
fallback initial image.  Host orchestration only: every arithmetic step runs
in liboslalm.

Run: python -m paper_1402_4381_gb300.warmstart --train 2000 --test 100 --out result.json
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import dataclasses
import json
import math
import multiprocessing as mp
import os
import time

import numpy as np

from . import roi, synth, workloads as W

SCALE = 1.0 / synth.MU_WATER  # network units: water = 1
HU = synth.HU
THRESHOLDS = (20.0, 10.0, 5.0, 2.0, 1.0)
FULL_REF_SCHEDULE = ((24, 100), (8, 100), (2, 200))  # then the one-subset method to convergence
ROUTE_SCHEDULE = ((24, 100), (8, 100), (2, 300), (1, 2000))  # the subset-reduction route that reaches 1 HU


def base_workload(nx=512, nviews=984, ns=888, M=24) -> W.Workload:
    """The fan-beam scan family (full size by default, or scaled with the
    same field of view and fan angle)."""
    wl = W.c1_fan()
    if (nx, nviews, ns) != (wl.geom.nx, wl.geom.nviews, wl.geom.ns):
        wl = W.scaled(wl, nx, nviews, ns, M, name_suffix=f"{nx}_v{nviews}")
    return dataclasses.replace(wl, M=M)


def scan_workload(seed: int, base: W.Workload) -> W.Workload:
    g = base.geom
    rng = np.random.default_rng(10_000 + seed)
    I0 = float(rng.uniform(2e4, 2e5))
    return dataclasses.replace(base, name=f"warm_{seed}", phantom="ellipses", phantom_seed=20_000 + seed,
                               noise_seed=30_000 + seed, n_ellipses=10, fov_radius=0.96 * g.nx * g.dx / 2,
                               I0=I0, sigma=0.0, w_dtype="f16", d_dtype="f16")


def _scan(wl):
    sc = wl.make_scan()
    return sc["y"], sc["w"]


def make_scans(wls, workers=None):
    """Sinograms of the workloads (numpy, in a spawn-context process pool:
    call before the process touches the GPU)."""
    workers = workers or min(16, os.cpu_count() or 1)
    if workers <= 1 or len(wls) <= 2:
        return [_scan(w) for w in wls]
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_scan, wls, chunksize=4))


def _problem(oslalm, torch, geomh, wl, y, w, M=None, use_graph=True, storage=None):
    dev = torch.device("cuda", torch.cuda.current_device())
    wd, dd = storage or (wl.w_dtype, wl.d_dtype)
    return oslalm.Problem(geomh, torch.as_tensor(y, device=dev), torch.as_tensor(w, device=dev), beta=wl.beta,
                          delta=wl.delta, nbr=wl.nbr, M=M or wl.M, w_dtype=wd, d_dtype=dd, use_graph=use_graph)


def run_batched(oslalm, torch, geomh, wls, scans, xs, schedule, chunk=64, storage=None):
    """Advance the images xs (in place) through `schedule` = ((M, iters), ...)
    with the batched persistent path, `chunk` scans per batch; a new M
    restarts the method (init) from the current image."""
    for k in range(0, len(wls), chunk):
        for M, iters in schedule:
            probs = [_problem(oslalm, torch, geomh, wl, y, w, M=M, use_graph=False, storage=storage)
                     for wl, (y, w) in zip(wls[k:k + chunk], scans[k:k + chunk])]
            for p, x in zip(probs, xs[k:k + chunk]):
                p.init(x)
            b = oslalm.Batch(probs)
            b.iterate(xs[k:k + chunk], iters, use_graph=True)
            torch.cuda.synchronize()
            b.close()
            for p in probs:
                p.close()
    return xs


def converge_batched(oslalm, torch, geomh, wls, scans, xs, mask_np, pre_schedule, block=500, tol_hu=0.01,
                     max_iters=8000, chunk=64, storage=("f32", "f32")):
    """Converged images x* (in place): `pre_schedule` (subset reduction),
    then the one-subset method (Sec. III-A: it converges to the minimiser) in
    blocks of `block` iterations, each scan keeping its method state, until
    its image changes by less than tol_hu (RMS over the mask) in a block or
    max_iters.  Returns per scan {"iterations", "last_change_hu",
    "converged"}."""
    run_batched(oslalm, torch, geomh, wls, scans, xs, pre_schedule, chunk, storage)
    mask = torch.as_tensor(mask_np.astype(np.uint8), device=xs[0].device)
    info = [None] * len(wls)
    for k in range(0, len(wls), chunk):
        idx = list(range(k, min(k + chunk, len(wls))))
        probs = {i: _problem(oslalm, torch, geomh, wls[i], *scans[i], M=1, use_graph=False, storage=storage)
                 for i in idx}
        for i in idx:
            probs[i].init(xs[i])
        active, done = idx, 0
        while active and done < max_iters:
            before = {i: xs[i].clone() for i in active}
            b = oslalm.Batch([probs[i] for i in active])
            b.iterate([xs[i] for i in active], block, use_graph=True)
            torch.cuda.synchronize()
            b.close()
            done += block
            still = []
            for i in active:
                ch = oslalm.rmsd(xs[i], before[i], mask) / HU
                info[i] = {"iterations": done, "last_change_hu": round(ch, 5), "converged": ch < tol_hu}
                if ch >= tol_hu:
                    still.append(i)
            del before
            active = still
        for i in idx:
            probs[i].close()
    return info


def train(torch, net, xs, ts, epochs, lr, batch, seed=0, log=None):
    """Adam on shuffled mini-batches, cosine decay of the learning rate.
    Returns (first-batch loss per epoch, steps, seconds)."""
    n = len(xs)
    rng = np.random.default_rng(seed)
    X = torch.stack([x.reshape(x.shape[-2:]) for x in xs])
    T = torch.stack([t.reshape(t.shape[-2:]) for t in ts])
    hist, steps = [], 0
    torch.cuda.synchronize()
    t0 = time.time()
    for ep in range(epochs):
        perm = torch.as_tensor(rng.permutation(n), device=X.device)
        lr_e = lr * 0.5 * (1 + math.cos(math.pi * ep / epochs))
        first = None
        for k in range(0, n - batch + 1, batch):
            idx = perm[k:k + batch]
            xb = X.index_select(0, idx).contiguous()
            tb = T.index_select(0, idx).contiguous()
            l = net.train_step(xb, tb, SCALE, lr_e, want_loss=(k == 0))
            first = l if k == 0 else first
            steps += 1
        hist.append(float(first))
        if log:
            log(f"epoch {ep}: loss {first:.4e} lr {lr_e:.2e}")
    torch.cuda.synchronize()
    return hist, steps, time.time() - t0


def evaluate(oslalm, torch, geomh, wls, scans, x0s, xstars, mask_np, init_fn=None, n_iter=50,
             thresholds=THRESHOLDS):
    """Per scan: RMSD curve (HU) of OS-LALM from x0 (or init_fn(x0)), and the
    iterations / seconds to reach each threshold."""
    dev = x0s[0].device
    mask = torch.as_tensor(mask_np.astype(np.uint8), device=dev)
    stream = torch.cuda.current_stream()
    if init_fn is not None:  # one untimed call: first-launch costs stay out of the scans' times
        init_fn(x0s[0])
        torch.cuda.synchronize()
    rows = []
    for wl, (y, w), x0, xs in zip(wls, scans, x0s, xstars):
        p = _problem(oslalm, torch, geomh, wl, y, w)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        x = init_fn(x0) if init_fn else x0.clone()
        p.init(x)
        e1.record(stream)
        e1.synchronize()
        t = e0.elapsed_time(e1)
        curve = [oslalm.rmsd(x, xs, mask) / HU]
        reached = {th: (0, t / 1000.0) for th in thresholds if curve[0] <= th}
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
        rows.append(dict(curve=curve, reached=reached))
        p.close()
    return rows


def evaluate_route(oslalm, torch, geomh, wls, scans, x0s, xstars, mask_np, init_fn=None,
                   schedule=ROUTE_SCHEDULE, thresholds=THRESHOLDS, stop_hu=1.0):
    """Per scan: the subset-reduction route (OS-LALM with `schedule` =
    ((M, iterations), ...), each stage restarting the method from the
    current image; FP32 storage) from x0 (or init_fn(x0)), until the RMS
    difference to x* falls to stop_hu.  Timed with CUDA events: network
    inference, every stage's oslalm_init (D recomputed) and the iterations;
    the RMS differences after every iteration are not timed."""
    dev = x0s[0].device
    mask = torch.as_tensor(mask_np.astype(np.uint8), device=dev)
    stream = torch.cuda.current_stream()
    if init_fn is not None:
        init_fn(x0s[0])
        torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        return out, e0.elapsed_time(e1)

    rows = []
    for wl, (y, w), x0, xs in zip(wls, scans, x0s, xstars):
        torch.cuda.synchronize()
        x, t = timed(lambda: init_fn(x0) if init_fn else x0.clone())
        curve = [oslalm.rmsd(x, xs, mask) / HU]
        reached = {th: (0, t / 1000.0) for th in thresholds if curve[0] <= th}
        k, done = 0, curve[0] <= stop_hu
        for M, n in schedule:
            if done:
                break
            p = _problem(oslalm, torch, geomh, wl, y, w, M=M, storage=("f32", "f32"))
            t += timed(lambda: p.init(x))[1]
            for _ in range(n):
                t += timed(lambda: p.iterate(x, 1))[1]
                k += 1
                r = oslalm.rmsd(x, xs, mask) / HU
                curve.append(r)
                for th in thresholds:
                    if th not in reached and r <= th:
                        reached[th] = (k, t / 1000.0)
                if r <= stop_hu:
                    done = True
                    break
            p.close()
        rows.append(dict(curve=curve, reached=reached))
    return rows


def summarize_route(rows, thresholds=THRESHOLDS):
    out = {"thresholds": {}}
    for th in thresholds:
        hit = [r["reached"][th] for r in rows if th in r["reached"]]
        out["thresholds"][f"{th:g}"] = {
            "reached": len(hit), "of": len(rows),
            "mean_iterations": float(np.mean([h[0] for h in hit])) if hit else None,
            "mean_seconds": float(np.mean([h[1] for h in hit])) if hit else None,
            "median_seconds": float(np.median([h[1] for h in hit])) if hit else None,
        }
    return out


def summarize(rows, thresholds=THRESHOLDS):
    curves = np.array([r["curve"] for r in rows])
    out = {"rmsd_hu_mean_by_iteration": [round(float(v), 3) for v in curves.mean(axis=0)], "thresholds": {}}
    for th in thresholds:
        hit = [r["reached"][th] for r in rows if th in r["reached"]]
        out["thresholds"][f"{th:g}"] = {
            "reached": len(hit), "of": len(rows),
            "mean_iterations": float(np.mean([h[0] for h in hit])) if hit else None,
            "mean_seconds": float(np.mean([h[1] for h in hit])) if hit else None,
        }
    return out


def paired_gain(fbp_rows, cnn_rows, thresholds=THRESHOLDS):
    """Per threshold, over the scans where both starts reach it: mean
    iterations and seconds saved by the network's initial image."""
    out = {}
    for th in thresholds:
        both = [(f["reached"][th], c["reached"][th]) for f, c in zip(fbp_rows, cnn_rows)
                if th in f["reached"] and th in c["reached"]]
        only_cnn = sum(1 for f, c in zip(fbp_rows, cnn_rows) if th in c["reached"] and th not in f["reached"])
        out[f"{th:g}"] = {
            "scans_both": len(both), "scans_only_cnn": only_cnn,
            "iterations_fbp": float(np.mean([b[0][0] for b in both])) if both else None,
            "iterations_cnn": float(np.mean([b[1][0] for b in both])) if both else None,
            "seconds_fbp": float(np.mean([b[0][1] for b in both])) if both else None,
            "seconds_cnn": float(np.mean([b[1][1] for b in both])) if both else None,
        }
    return out


def experiment(n_train=2000, n_test=100, target_iters=200, epochs=30, batch=8, lr=1e-3, nx=512, nviews=984,
               ns=888, M=24, ref_schedule=FULL_REF_SCHEDULE, n_eval_iter=50, chunk=64, log=print,
               ref_block=500, ref_tol_hu=0.01, ref_max_iters=8000, params_out=None, params_in=None):
    """The whole warm-start experiment; returns a JSON-ready dict.  With
    `params_in` (parameters saved by an earlier run) the training part is
    skipped and the saved network is evaluated."""
    base = base_workload(nx, nviews, ns, M)
    if params_in:
        n_train = 0
    wls_tr = [scan_workload(s, base) for s in range(n_train)]
    wls_te = [scan_workload(1_000_000 + s, base) for s in range(n_test)]
    t0 = time.time()
    scans_tr = make_scans(wls_tr)
    scans_te = make_scans(wls_te)
    t_scan = time.time() - t0
    log(f"scans: {t_scan:.1f} s")
    import torch
    from . import oslalm
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    g = base.geom
    geomh = oslalm.Geometry(g)
    x0_tr = [geomh.fbp(torch.as_tensor(y, device=dev), clip=True) for y, _ in scans_tr]
    x0_te = [geomh.fbp(torch.as_tensor(y, device=dev), clip=True) for y, _ in scans_te]
    torch.cuda.synchronize()
    inf = oslalm.WarmStartNet(1, g.ny, g.nx, seed=0)
    if params_in:
        inf.set_params(np.load(params_in))
        hist, steps, t_train, t_targets, flops = [], 0, 0.0, 0.0, 0.0
    else:
        t0 = time.time()
        targets = run_batched(oslalm, torch, geomh, wls_tr, scans_tr, [x.clone() for x in x0_tr],
                              ((M, target_iters),), chunk)
        t_targets = time.time() - t0
        log(f"targets: {t_targets:.1f} s")
        net = oslalm.WarmStartNet(batch, g.ny, g.nx, seed=0)
        hist, steps, t_train = train(torch, net, x0_tr, targets, epochs, lr, batch, log=log)
        flops = 3.0 * oslalm.WarmStartNet.flops_per_image(g.ny, g.nx) * batch * steps
        del targets
        inf.set_params(net.get_params())
        if params_out:
            np.save(params_out, net.get_params())

    def cnn_init(x0):
        return torch.clamp(inf.forward(x0.view(1, g.ny, g.nx), SCALE), min=0.0).view(x0.shape)

    mask = roi.roi_mask(g)
    t0 = time.time()
    xstars = [x.clone() for x in x0_te]
    ref_info = converge_batched(oslalm, torch, geomh, wls_te, scans_te, xstars, mask, ref_schedule, ref_block,
                                ref_tol_hu, ref_max_iters, chunk)
    t_ref = time.time() - t0
    n_conv = sum(r["converged"] for r in ref_info)
    log(f"references: {t_ref:.1f} s; {n_conv} of {len(ref_info)} converged (change < {ref_tol_hu} HU per "
        f"{ref_block} iterations); iterations max {max(r['iterations'] for r in ref_info)}")
    fbp_rows = evaluate(oslalm, torch, geomh, wls_te, scans_te, x0_te, xstars, mask, None, n_eval_iter)
    cnn_rows = evaluate(oslalm, torch, geomh, wls_te, scans_te, x0_te, xstars, mask, cnn_init, n_eval_iter)
    t0 = time.time()
    fbp_route = evaluate_route(oslalm, torch, geomh, wls_te, scans_te, x0_te, xstars, mask, None)
    cnn_route = evaluate_route(oslalm, torch, geomh, wls_te, scans_te, x0_te, xstars, mask, cnn_init)
    log(f"route evaluation: {time.time() - t0:.1f} s")
    ok = [i for i, r in enumerate(ref_info) if r["converged"]]  # scans with a verified x*
    fbp_ok, cnn_ok = [fbp_route[i] for i in ok], [cnn_route[i] for i in ok]
    return {
        "geometry": {"image": [g.ny, g.nx], "views": g.nviews, "channels": g.ns, "M": M},
        "train": {"scans": n_train, "target_iterations": target_iters, "epochs": epochs, "batch": batch,
                  "steps": steps, "seconds": round(t_train, 2),
                  "tflops_bf16": round(flops / t_train / 1e12, 2) if t_train > 0 else None,
                  "params_in": params_in,
                  "loss_by_epoch": [round(v, 6) for v in hist]},
        "held_out": n_test, "reference_schedule": [list(s) for s in ref_schedule],
        "reference_storage": "f32",
        "reference": {"then": f"one subset in blocks of {ref_block} iterations until the RMS change in a block "
                              f"is below {ref_tol_hu} HU (at most {ref_max_iters})",
                      "converged": n_conv, "of": len(ref_info),
                      "iterations": [r["iterations"] for r in ref_info],
                      "last_change_hu": [r["last_change_hu"] for r in ref_info]},
        "configured": {"M": M, "iterations": n_eval_iter, "storage": [base.w_dtype, base.d_dtype],
                       "fbp_init": summarize(fbp_rows), "cnn_init": summarize(cnn_rows),
                       "paired": paired_gain(fbp_rows, cnn_rows)},
        "route": {"schedule": [list(s) for s in ROUTE_SCHEDULE], "stop_hu": 1.0, "storage": "f32",
                  "scans": "the held-out scans whose x* converged",
                  "fbp_init": summarize_route(fbp_ok), "cnn_init": summarize_route(cnn_ok),
                  "paired": paired_gain(fbp_ok, cnn_ok)},
        "seconds": {"scan_generation_cpu": round(t_scan, 1), "targets_gpu": round(t_targets, 1),
                    "references_gpu": round(t_ref, 1)},
    }


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--test", type=int, default=100)
    ap.add_argument("--target-iters", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--nx", type=int, default=512)
    ap.add_argument("--views", type=int, default=984)
    ap.add_argument("--channels", type=int, default=888)
    ap.add_argument("--M", type=int, default=24)
    ap.add_argument("--eval-iters", type=int, default=50)
    ap.add_argument("--out", default=None)
    ap.add_argument("--params-out", default=None, help="save the trained parameters (.npy)")
    ap.add_argument("--params-in", default=None, help="evaluate saved parameters (.npy) instead of training")
    a = ap.parse_args(argv)
    res = experiment(a.train, a.test, a.target_iters, a.epochs, a.batch, a.lr, a.nx, a.views, a.channels, a.M,
                     n_eval_iter=a.eval_iters, params_out=a.params_out, params_in=a.params_in)
    s = json.dumps(res, indent=1)
    if a.out:
        with open(a.out, "w") as f:
            f.write(s)
    print(s)


if __name__ == "__main__":
    main()
