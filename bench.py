#!/usr/bin/env python
"""Benchmark of the OS-LALM hot path on the 2D fan-beam PWLS workload
(512x512 image, 984 views x 888 channels, M = 24 subsets, 50 iterations,
FP16 storage of W and of the SQS denominator).

One step = one reconstruction: reset x to the initial image, oslalm_init
(first subset gradient, split gradient, rho = 1), then 50 iterations
(1200 subset-iterations).  The metric is subset-iterations per second (one
subset-iteration = one forward projection + exact-transpose back-projection
of a 41-view subset plus the fused update).  Also reported: time to reach
1 HU RMS difference from a converged image, the roofline of the dominant
kernel, an end-to-end figure through the C ABI with host buffers, and the
FP64 oracle timed on the host cores.

--impl reference times the FP64 oracle on the same workload (bounded sample:
one subset-iteration per step).  With torchrun (N > 1) every rank runs an
independent replica on its own GPU (the path has no exchange step).
"""
import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "A/A' subset-iters/s (OS-LALM, 2D fan beam 512^2, 984x888, M=24)"

UNIT = "subset-iters/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-time-to-hu", action="store_true")
    ap.add_argument("--workload", default="fan",
                    choices=["fan", "fan256", "cone", "helical", "parallel", "batch", "cnn"],
                    help="fan: the 512^2 fan-beam scan (default, the headline); fan256: the same scan family at "
                         "256^2, 492 views, M = 12; cone / parallel: the 512x512x128 cone-beam and 128^2 "
                         "parallel-beam scans; helical: 512x512x64, 2 turns of 984 views at pitch 0.5, M = 36; "
                         "batch: 64 fan-beam slices of mixed sizes advanced together; cnn: training steps of the "
                         "warm-start U-Net (batch 8 of 512^2 images)")
    ap.add_argument("--slices", type=int, default=64)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_noise_seed(seed, rank):
    """Independent replicas on N GPUs: rank r reconstructs its own noise
    realisation of the same scan (the path has no exchange step)."""
    return seed + 1000 * rank


def max_over_ranks(local_ms, dist, device):
    """The job's time: the slowest rank's (all ranks get it)."""
    import torch
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(local_ms)
    t = torch.tensor([float(local_ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world, steps, units_per_step, t_max_ms):
    """Units processed by all ranks per second of the slowest rank."""
    return world * steps * units_per_step / (t_max_ms / 1000.0)


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], [], set()
        for line in open(self.path):
            f = [t.strip() for t in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"], f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def intersections_per_subset(geom, M, max_views=24):
    """Number of (ray, pixel/voxel) pairs with a non-zero length, per subset
    on average, counted in closed form per ray: a ray clipped to the image box
    crosses 1 + (number of grid planes between its entry and exit points)
    cells.  Counted on up to max_views evenly spaced views and scaled."""
    from paper_1402_4381_gb300 import synth
    views = np.linspace(0, geom.nviews - 1, min(max_views, geom.nviews)).round().astype(int)
    org, d = synth.rays(geom, views)
    three = geom.kind == synth.CONE3D_FLAT
    nd = 3 if three else 2
    org, d = org[..., :nd].reshape(-1, nd), d[..., :nd].reshape(-1, nd)
    size = [geom.nx * geom.dx, geom.ny * geom.dy, geom.nz * geom.dz][:nd]
    lo = -np.array(size) / 2
    hi = -lo
    with np.errstate(divide="ignore", invalid="ignore"):
        t0 = np.full(len(org), -np.inf)
        t1 = np.full(len(org), np.inf)
        for k in range(nd):
            a = (lo[k] - org[:, k]) / d[:, k]
            b = (hi[k] - org[:, k]) / d[:, k]
            t0 = np.maximum(t0, np.where(d[:, k] != 0, np.minimum(a, b), -np.inf))
            t1 = np.minimum(t1, np.where(d[:, k] != 0, np.maximum(a, b), np.inf))
    ok = t1 > t0
    pe = org[ok] + t0[ok, None] * d[ok]
    px = org[ok] + t1[ok, None] * d[ok]
    pix = np.array([geom.dx, geom.dy, geom.dz][:nd])
    ie = np.floor((np.clip(pe, lo, hi - 1e-9) - lo) / pix)
    ix = np.floor((np.clip(px, lo, hi - 1e-9) - lo) / pix)
    n = np.sum(np.abs(ix - ie), axis=1) + 1
    return float(n.sum()) * geom.nviews / len(views) / M


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return None


# DRAM bytes (read + write) per launch of the fan-beam workload's kernels from
# one ncu capture, keyed by a hash of the 2D kernel sources it was taken on:
# when the sources change, the figure no longer describes the kernel and the
# bench reports traffic as null until a new capture is recorded here.
NCU_DRAM_FAN = {"sources": "5eadf27ed026415c",
                "bytes": {"bp2d_kernel": 3469824, "fp2d_kernel": 2443008, "update2d_kernel": 3679232}}
KERNEL_SOURCES_2D = ("kernels2d.cu", "proj2d.cuh", "kernels_common.cuh", "common.cuh")


def kernel_sources_hash(names=KERNEL_SOURCES_2D):
    import hashlib
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_1402_4381_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def roofline_record(torch, dev, wl, prof, graph_ms_sub, clocks, workload):
    """Roofline of the dominant kernel from the per-launch CUDA-event times.

    Work per launch (one subset): the projectors evaluate `inter` (ray,
    pixel) intersections, 3 FP32 operations each (crossing, length,
    multiply-add), against the FP32 issue peak (SMs x 128 lanes x the median
    SM clock sampled in the timed region); their algorithmic HBM bytes are
    the data a launch must read and write once: forward + residual reads x,
    y_m, w_m and writes r; back-projection + split gradient reads r and
    reads and writes zeta and g.  The update reads x, zeta, g, D and writes
    x+.  `achieved` uses the event times as measured; per_kernel_ms takes
    off each launch the same share of the gap between their sum and the
    graph-timed subset-iteration (launch and event overhead)."""
    g = wl.geom
    nl = prof["launches"][0]
    ev = {"update": prof["update"] / nl, "forward": prof["forward"] / nl, "backproject": prof["backproject"] / nl}
    overhead = max(0.0, (sum(ev.values()) - graph_ms_sub) / 3.0)
    per = {k: v - overhead for k, v in ev.items()}
    dom = max(ev, key=ev.get)
    pk = peaks() or {}
    hbm = pk.get("hbm_gbs", 6800.0) * 1e9
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    npix = g.nx * g.ny * g.nz
    rays = g.nviews / wl.M * g.nt * g.ns
    wb = 4 if wl.w_dtype == "f32" else 2
    db = 4 if wl.d_dtype == "f32" else 2
    nbytes = {"forward": 4 * npix + rays * (4 + wb + 4), "backproject": rays * 4 + 16 * npix,
              "update": (4 + 4 + 4 + db + 4) * npix}
    dim = "3d" if g.kind == 2 else "2d"
    names = {"forward": f"fp{dim}_kernel", "backproject": f"bp{dim}_kernel", "update": f"update{dim}_kernel"}
    t = ev[dom] / 1000.0
    traffic = None
    if workload == "fan" and NCU_DRAM_FAN["sources"] == kernel_sources_hash():
        traffic = NCU_DRAM_FAN["bytes"].get(names[dom])
    hbm_rec = {"achieved": nbytes[dom] / t / 1e9, "peak": hbm / 1e9, "unit": "GB/s", "frac": nbytes[dom] / t / hbm,
               "algorithmic_bytes": nbytes[dom], "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json)"}
    if dom in ("forward", "backproject"):
        inter = intersections_per_subset(g, wl.M)
        peak_ops = sms * 128 * sm_mhz * 1e6
        achieved = 3.0 * inter / t
        roof = {"kernel": names[dom], "bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                "unit": "TFLOP/s", "frac": achieved / peak_ops, "traffic": traffic,
                "work_per_launch": f"{inter:.4g} intersections x 3 FP32 ops",
                "peak_basis": f"{sms} SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz (median SM clock under load)",
                "hbm": hbm_rec, "intersections_per_s": inter / t}
    else:
        roof = {"kernel": names[dom], "bound": "hbm", "achieved": hbm_rec["achieved"], "peak": hbm / 1e9,
                "unit": "GB/s", "frac": hbm_rec["frac"], "traffic": traffic,
                "work_per_launch": f"{nbytes[dom] / 1e6:.2f} MB", "peak_basis": hbm_rec["peak_basis"]}
    roof["per_kernel_ms_events"] = {k: round(v, 5) for k, v in ev.items()}
    roof["per_kernel_ms"] = {k: round(v, 5) for k, v in per.items()}
    roof["graph_ms_per_subset_iteration"] = round(graph_ms_sub, 5)
    roof["launch_overhead_ms"] = round(overhead, 5)
    roof["kernel_sources"] = kernel_sources_hash()
    return roof


# ---------------------------------------------------------------------------- reference arm: the FP64 oracle

ORACLE_SAMPLE_NOTE = ("FP64 oracle subset-iterations (41 views x 888 rays each) of the same scan; for timing only, "
                      "its majorizer D is approximated from one subset (M A_0'W_0 A_0 1)")


def oracle_sample(wl, scan, x0, n_steps, threads=1):
    """Time the FP64 oracle's subset-iterations on the workload with
    `threads` host threads in its projector: seconds per subset-iteration."""
    from oracle import oslalm as O
    from oracle import siddon
    siddon.set_threads(threads)
    g = wl.geom
    data, _ = O.ct_subset_data(g, scan["y"].astype(np.float64), scan["w"].astype(np.float64), wl.M, siddon)
    # timing sample only: D approximated from one subset (M A_0' W_0 A_0 1)
    m0 = O.bit_reversal_order(wl.M)[0]
    D = wl.M * data.At_m(data.w[m0] * data.A_m(np.ones(g.image_shape), m0), m0)
    alg = O.OsLalm(data, D, wl.beta, wl.delta, wl.nbr)
    alg.init(x0.astype(np.float64))
    times = []
    for _ in range(n_steps):
        t = time.perf_counter()
        alg.step()
        times.append(time.perf_counter() - t)
    return times


def cpu_baseline(wl, scan, x0):
    """The oracle on all host cores (8 subset-iterations after one untimed)
    and on one core (2 after one untimed)."""
    cores = os.cpu_count() or 1
    times = oracle_sample(wl, scan, x0, 9, threads=cores)
    t = sum(times[1:])
    one = oracle_sample(wl, scan, x0, 3, threads=1)
    t1 = sum(one[1:])
    return {"value": 8 / t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"8 {ORACLE_SAMPLE_NOTE}, {cores} threads, after one untimed",
            "single_thread": {"value": 2 / t1, "unit": UNIT, "cores": 1,
                              "sample": "2 of the same subset-iterations, one thread, after one untimed"}}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    from paper_1402_4381_gb300 import workloads as W
    wl = {"fan": W.c1_fan, "fan256": W.c1_fan_256, "cone": W.c2_cone, "helical": W.c2_helical,
          "parallel": W.c0_parallel}[args.workload]()
    scan = wl.make_scan()
    from oracle import fbp as ofbp
    x0 = np.maximum(ofbp.fbp(wl.geom, scan["y"].astype(np.float64)), 0.0)
    cores = os.cpu_count() or 1
    times = oracle_sample(wl, scan, x0, args.warmup + args.steps, threads=cores)
    t = sum(times[args.warmup:])
    value = args.steps / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "step": "one subset-iteration of the FP64 oracle", "M": wl.M},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} timed {ORACLE_SAMPLE_NOTE}, {cores} threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_1402_4381_gb300 import oslalm, roi, workloads as W

    wl = {"fan": W.c1_fan, "fan256": W.c1_fan_256, "cone": W.c2_cone, "helical": W.c2_helical,
          "parallel": W.c0_parallel}[args.workload]()
    wl.noise_seed = replica_noise_seed(wl.noise_seed, rank)
    g = wl.geom
    scan = wl.make_scan()
    mask_np = roi.roi_mask(g)
    dev = torch.device("cuda", torch.cuda.current_device())
    y = torch.as_tensor(scan["y"], device=dev)
    w = torch.as_tensor(scan["w"], device=dev)
    geom = oslalm.Geometry(g)
    # initial image: FBP of the log sinogram, clipped to x >= 0 (set-up)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    if g.pitch != 0.0:  # no FDK for a helix: a water cylinder over the field of view
        x0 = torch.as_tensor(np.where(mask_np, 0.0192, 0.0).astype(np.float32), device=dev)
    else:
        x0 = geom.fbp(y, clip=True)
    e1.record()
    e1.synchronize()
    fbp_ms = e0.elapsed_time(e1)
    x0_np = x0.cpu().numpy()
    x = x0.clone()
    prob = oslalm.Problem(geom, y, w, beta=wl.beta, delta=wl.delta, nbr=wl.nbr, M=wl.M,
                          w_dtype=wl.w_dtype, d_dtype=wl.d_dtype, use_graph=True)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)

    def step():
        x.copy_(x0)
        prob.init(x)
        prob.iterate(x, wl.n_iter)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    total_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()  # L2 flush between timed steps (outside the events)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    t_max = max_over_ranks(total_ms, torch.distributed if world > 1 else None, dev)
    units_per_step = wl.n_iter * wl.M
    value = whole_job_value(world, args.steps, units_per_step, t_max)

    # ---- end to end through the C ABI with host buffers
    y_h = torch.as_tensor(scan["y"]).pin_memory()
    w_h = torch.as_tensor(scan["w"]).pin_memory()
    x0_h = torch.as_tensor(x0_np).pin_memory()
    x_out = torch.empty_like(x0_h).pin_memory()
    y_d, w_d = torch.empty_like(y), torch.empty_like(w)

    def e2e_step():
        y_d.copy_(y_h, non_blocking=True)
        w_d.copy_(w_h, non_blocking=True)
        x.copy_(x0_h, non_blocking=True)
        prob.set_data(y_d, w_d)
        prob.init(x)
        prob.iterate(x, wl.n_iter)
        x_out.copy_(x, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    e2e_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_step()
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    e2e_value = whole_job_value(world, args.steps, units_per_step,
                                max_over_ranks(e2e_ms, torch.distributed if world > 1 else None, dev))
    h2d = y_h.numel() * 4 + w_h.numel() * 4 + x0_h.numel() * 4
    d2h = x_out.numel() * 4

    # ---- per-kernel device time (CUDA events around each launch kind)
    x.copy_(x0)
    prob.init(x)
    prof = prob.profile_iterate(x, 4 if g.kind != 2 else 1)
    graph_ms_sub = t_max / args.steps / units_per_step  # graph replay, per subset-iteration
    roof = roofline_record(torch, dev, wl, prof, graph_ms_sub, clocks, args.workload)

    # ---- time to 1 HU against a converged image (M = 1 continuation, long run)
    ttu = None
    if not args.no_time_to_hu and g.kind != 2 and rank == 0:  # a study of one scan: rank 0 alone
        ttu = time_to_hu(torch, oslalm, wl, geom, y, w, x0, mask_np, dev, stream)
        ttu["fbp_setup_ms"] = fbp_ms

    line = {
        "metric": METRIC if args.workload == "fan" else f"A/A' subset-iters/s (OS-LALM, {wl.name})", "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name, "image": [g.nx, g.ny], "views": g.nviews, "channels": g.ns, "M": wl.M,
                   "iterations_per_step": wl.n_iter, "storage": {"W": wl.w_dtype, "D": wl.d_dtype},
                   "parallelism": f"replicas{world}", "l2": "flushed between timed steps (256 MB write)",
                   "system_matrix": "evaluated in every launch"},
        "gpu_launches": args.steps * (wl.n_iter * wl.M * 3 + 3),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "roofline": roof, "clocks": clocks,
    }
    if ttu:
        line["time_to_1hu"] = ttu
    if rank == 0 and world == 1 and not args.no_cpu_baseline and g.kind != 2:  # the oracle: rank 0 at N = 1
        line["cpu_baseline"] = cpu_baseline(wl, scan, x0_np)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


XSTAR_TOL_HU = 0.1  # the two limits of x* must agree to a tenth of the 1 HU target


def verify_converged(torch, oslalm, wl, geom, y, w, xs, xs_b, mask, HU):
    """Checks of the converged image x* (Sec. III-A: the one-subset method
    converges to the minimiser of Eq. ct_recon over x >= 0):
    * KKT: the gradient A'W(Ax - y) + grad R(x) (oslalm_gradient), projected
      on the constraint (at x = 0 only its negative part), relative to
      |A'Wy|_inf (the gradient at x = 0), max over the field of view;
    * the projected SQS step x - max(0, x - grad / D) in HU (RMS and max
      over the field of view): what one more rho = 1, M = 1 step would move;
    * the cost (FP64 reductions) and the RMS difference to the limit of the
      same schedule from another initial image; x* is accepted when that
      difference is below XSTAR_TOL_HU."""
    pk = oslalm.Problem(geom, y, w, beta=wl.beta, delta=wl.delta, nbr=wl.nbr, M=1, use_graph=False)
    pk.init(xs)
    D = pk.denominator()
    m = mask.bool()
    scale = float(pk.gradient(torch.zeros_like(xs)).abs().max())
    out = {}
    for name, x in (("x_star", xs), ("second_limit", xs_b)):
        gr = pk.gradient(x)
        pg = torch.where(x > 0, gr, torch.clamp(gr, max=0.0))
        step = x - torch.clamp(x - gr / D, min=0.0)
        out[name] = {"kkt_rel": float(pg[m].abs().max()) / scale,
                     "sqs_step_hu_rms": float(step[m].square().mean().sqrt()) / HU,
                     "sqs_step_hu_max": float(step[m].abs().max()) / HU,
                     "cost": pk.cost(x)}
    pk.close()
    diff = oslalm.rmsd(xs, xs_b, mask) / HU
    out["limits_rmsd_hu"] = round(diff, 4)
    out["tolerance_hu"] = XSTAR_TOL_HU
    out["accepted"] = bool(diff <= XSTAR_TOL_HU)
    return out


def time_to_hu(torch, oslalm, wl, geom, y, w, x0, mask_np, dev, stream,
               thresholds=(20.0, 10.0, 5.0, 2.0, 1.0), max_iter=300,
               schedule=((24, 100), (8, 100), (2, 200)), m1_block=1000, m1_max=12000, m1_tol_hu=2e-3,
               snap_every=10, inner_iters=100):
    """Time to reach HU thresholds of RMS difference (field of view) from a
    converged image x*, from the FBP image.

    x*: OS-LALM with a decreasing number of subsets (fast early progress),
    then the convergent one-subset method (Sec. III-A) until its image
    changes by less than m1_tol_hu over m1_block iterations.  That run is
    itself timed (CUDA events per stage, set-up of each stage included) and
    snapshotted every snap_every iterations, so its own time to each
    threshold is reported too ("subset_reduction").  Then the benchmark
    configuration (M subsets, storage types of the workload) from the same
    FBP image for up to max_iter iterations, timing each iteration with CUDA
    events ("configured"); OS-LALM with M > 1 does not converge to x*
    (Sec. III-A), so its RMS difference levels off, reported as "plateau".
    The same run with Barzilai-Borwein scaling of the majorizer, and with
    n = 2 and 5 inner FISTA steps for inner_iters iterations ("inner_sweep":
    per-iteration device time, one graph launch and synchronisation each)."""
    HU = 0.0192 / 1000.0
    mask = torch.as_tensor(mask_np.astype(np.uint8), device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    # ---- x* by subset reduction, timed and snapshotted
    def converge(x_start, record):
        """Subset reduction, then the one-subset method until the image
        changes by less than m1_tol_hu over m1_block iterations."""
        xc = x_start.clone()
        snaps, t_ms, it, stages, change = [], 0.0, 0, [], None
        for M, n in list(schedule) + [(1, m1_max)]:
            p = oslalm.Problem(geom, y, w, beta=wl.beta, delta=wl.delta, nbr=wl.nbr, M=M, use_graph=True)
            t_ms += timed(lambda: p.init(xc))
            done = 0
            prev = xc.clone()
            while done < n:
                k = min(snap_every, n - done)
                t_ms += timed(lambda: p.iterate(xc, k))
                done += k
                it += k
                if record:
                    snaps.append((it, t_ms / 1000.0, xc.clone()))
                if M == 1 and done % m1_block == 0:
                    change = oslalm.rmsd(xc, prev, mask) / HU
                    prev = xc.clone()
                    if change < m1_tol_hu:
                        break
            stages.append(f"M={M} x {done}")
            p.close()
        return xc, snaps, stages, change

    xs, snaps, stages, change = converge(x0, True)
    # the same from a second start (water over the field of view): the two
    # limits bound how far either is from the minimiser
    xs_b, _, stages_b, _ = converge(torch.where(mask.bool(), 0.0192, 0.0).to(torch.float32), False)
    xstar = verify_converged(torch, oslalm, wl, geom, y, w, xs, xs_b, mask, HU)
    xstar["second_start"] = {"x0": "water (0.0192 /mm) over the field of view", "schedule": ", ".join(stages_b)}
    del xs_b
    sub = {}
    for k, t, im in snaps:
        r = oslalm.rmsd(im, xs, mask) / HU
        for th in thresholds:
            if th not in sub and r <= th:
                sub[th] = {"iterations": k, "seconds": round(t, 4)}
    del snaps

    # ---- the configured OS-LALM from the same FBP image, without and with
    # Barzilai-Borwein scaling of the majorizer (supplement Sec. II-A)
    keep_at = (5, 20, 50)

    def configured(bb, n_inner=1, iters=max_iter, storage=(wl.w_dtype, wl.d_dtype), keep=None):
        prob = oslalm.Problem(geom, y, w, beta=wl.beta, delta=wl.delta, nbr=wl.nbr, M=wl.M,
                              w_dtype=storage[0], d_dtype=storage[1], use_graph=True, bb=bb, n_inner=n_inner)
        x = x0.clone()
        t_ms = timed(lambda: prob.init(x))
        t_iter = 0.0
        curve, reached = [], {}
        for k in range(1, iters + 1):
            dt = timed(lambda: prob.iterate(x, 1))
            t_ms += dt
            t_iter += dt
            r = oslalm.rmsd(x, xs, mask) / HU
            curve.append(round(r, 3))
            for th in thresholds:
                if th not in reached and r <= th:
                    reached[th] = {"iterations": k, "seconds": round(t_ms / 1000.0, 5)}
            if keep is not None and k in keep_at:
                keep[k] = x.clone()
        prob.close()
        return curve, reached, t_iter / iters

    kept16, kept32 = {}, {}
    curve, reached, ms_it = configured(False, keep=kept16)
    configured(False, iters=max(keep_at), storage=("f32", "f32"), keep=kept32)
    storage_err = {str(k): round(oslalm.rmsd(kept16[k], kept32[k], mask) / HU, 4) for k in keep_at}
    del kept16, kept32
    curve_bb, reached_bb, _ = configured(True)
    # number n of inner FISTA steps of the constrained denoising (Sec. III-A):
    # more steps per outer iteration against their cost
    sweep = {}
    for n_inner in (1, 2, 5):
        c, r, m = (curve, reached, ms_it) if n_inner == 1 else configured(False, n_inner, inner_iters)
        sweep[str(n_inner)] = {"ms_per_iteration": round(m, 4),
                               "thresholds": {f"{th:g}": r.get(th) for th in thresholds},
                               "rmsd_hu_every_10": c[9:inner_iters:10]}
    one = reached.get(1.0)
    sub_one = sub.get(1.0)
    routes = [(n, r) for n, r in (("configured", one), ("configured_bb", reached_bb.get(1.0)),
                                  ("subset_reduction", sub_one)) if r]
    best = min(routes, key=lambda t: t[1]["seconds"]) if routes else (None, None)
    return {"target_hu": 1.0,
            "route": best[0],
            "iterations": best[1]["iterations"] if best[1] else None,
            "seconds": best[1]["seconds"] if best[1] else None,
            "configured": {"M": wl.M, "thresholds": {f"{th:g}": reached.get(th) for th in thresholds},
                           "plateau_hu": round(float(np.mean(curve[-20:])), 3), "iterations_run": max_iter,
                           "rmsd_hu_every_10": curve[9::10],
                           "includes": "oslalm_init (first subset gradient; D cached) and the iterations; x0 = FBP"},
            "configured_bb": {"M": wl.M, "thresholds": {f"{th:g}": reached_bb.get(th) for th in thresholds},
                              "plateau_hu": round(float(np.mean(curve_bb[-20:])), 3),
                              "rmsd_hu_every_10": curve_bb[9::10],
                              "note": "the configured run with Barzilai-Borwein scaling of the majorizer"},
            "inner_sweep": {"iterations_run": inner_iters, "M": wl.M, "n": sweep,
                            "note": "n inner FISTA steps per subset-iteration (n = 1: the SQS step)"},
            "subset_reduction": {"schedule": ", ".join(stages),
                                 "thresholds": {f"{th:g}": sub.get(th) for th in thresholds},
                                 "seconds_to_1hu": sub_one["seconds"] if sub_one else None,
                                 "iterations_to_1hu": sub_one["iterations"] if sub_one else None,
                                 "includes": "every stage's oslalm_init (D recomputed) and iterations, FP32 storage; "
                                             "x0 = FBP; resolution 10 iterations"},
            "storage_error_hu": {"iterations": storage_err,
                                 "note": f"RMS difference (field of view) between the configured run with "
                                         f"{wl.w_dtype} W and {wl.d_dtype} D and the same run with FP32 storage"},
            "xstar": xstar,
            "reference": f"x*: end of the subset-reduction run; change over its last {m1_block} one-subset "
                         f"iterations {change:.4f} HU" if change is not None else "x*: end of the subset-reduction run"}


def _make_scan(wl):
    sc = wl.make_scan()
    return sc["y"], sc["w"]


def run_batch(args):
    """64 fan-beam slices (mixed image sizes / view counts / subsets), one
    step = the whole batch reconstructed (init + 30 iterations of every
    slice) by the batched persistent kernels under a CUDA graph."""
    import concurrent.futures as cf
    import multiprocessing as mp
    from paper_1402_4381_gb300 import workloads as W
    wls = W.c3_batch(args.slices)
    with cf.ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 1),
                                mp_context=mp.get_context("spawn")) as ex:
        scans = list(ex.map(_make_scan, wls))
    import torch
    torch.cuda.set_device(0)
    from paper_1402_4381_gb300 import oslalm
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    geoms, probs, x0s, xs = [], [], [], []
    for wl, (y, w) in zip(wls, scans):
        geom = oslalm.Geometry(wl.geom)
        yt, wt = torch.as_tensor(y, device=dev), torch.as_tensor(w, device=dev)
        x0 = geom.fbp(yt, clip=True)
        p = oslalm.Problem(geom, yt, wt, beta=wl.beta, delta=wl.delta, nbr=wl.nbr, M=wl.M, use_graph=False)
        x = x0.clone()
        p.init(x)
        geoms.append(geom); probs.append(p); x0s.append(x0); xs.append(x)
    batch = oslalm.Batch(probs)
    tune = batch.autotune(xs, probe_iters=1)
    shape, bps = batch.get_shape()
    n_iter = wls[0].n_iter
    units = sum(n_iter * wl.M for wl in wls)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        for x, x0, p in zip(xs, x0s, probs):
            x.copy_(x0)
            p.init(x)
        batch.iterate(xs, n_iter, use_graph=True)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    total = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    clocks = sampler.stop()
    # the same slices one at a time (single-problem path, graphs on) for comparison
    single_ms = 0.0
    singles = []
    for wl, (y, w), geom, x0 in zip(wls, scans, geoms, x0s):
        p = oslalm.Problem(geom, torch.as_tensor(y, device=dev), torch.as_tensor(w, device=dev), beta=wl.beta,
                           delta=wl.delta, nbr=wl.nbr, M=wl.M, use_graph=True)
        x = x0.clone()
        p.init(x)
        p.iterate(x, 1)
        singles.append((p, x, x0))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for p, x, x0 in singles:
        x.copy_(x0)
        p.init(x)
        p.iterate(x, n_iter)
    e1.record(stream)
    e1.synchronize()
    single_ms = e0.elapsed_time(e1)
    sizes = sorted({wl.geom.nx for wl in wls})
    line = {
        "metric": f"A/A' subset-iters/s (OS-LALM, batch of {len(wls)} fan-beam slices)",
        "value": args.steps * units / (total / 1000.0), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batch{len(wls)}_fan_mixed", "slices": len(wls), "image_sizes": sizes,
                   "views": sorted({wl.geom.nviews for wl in wls}), "subset_iters_per_step": units,
                   "iterations": n_iter, "shape": {**oslalm.Batch.shapes()[shape], "blocks_per_sm": bps},
                   "autotune_ms": tune, "l2": "flushed between timed steps (256 MB write)"},
        "gpu_launches": args.steps * (3 * len(wls) + 4 * max(n_iter * wl.M for wl in wls)),
        "one_at_a_time": {"value": units / (single_ms / 1000.0), "unit": UNIT,
                          "note": "the same slices reconstructed sequentially by the single-problem path"},
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_cnn(args):
    """Training steps (forward, backward, Adam) of the warm-start U-Net on
    batches of 8 images of 512^2 pixels: TFLOP/s against the BF16 tensor-core
    peak, plus the forward pass alone (inference)."""
    import torch
    torch.cuda.set_device(0)
    from paper_1402_4381_gb300 import oslalm
    B, H, Wd = 8, 512, 512
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    gen = torch.Generator(device=dev).manual_seed(0)
    x = torch.rand((B, H, Wd), device=dev, generator=gen) * 0.04
    t = x + 0.002 * torch.randn((B, H, Wd), device=dev, generator=gen)
    scale = 1.0 / 0.0192
    net = oslalm.WarmStartNet(B, H, Wd, seed=0)
    fpi = oslalm.WarmStartNet.flops_per_image(H, Wd)

    def timed(fn, n):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / n

    # the network's own kernels in one training step (the timed steps repeat it)
    n0 = oslalm.WarmStartNet.launch_count()
    net.train_step(x, t, scale, 1e-4, want_loss=False)
    launches_per_step = oslalm.WarmStartNet.launch_count() - n0
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    ms_train = timed(lambda: net.train_step(x, t, scale, 1e-4, want_loss=False), args.steps)
    ms_fwd = timed(lambda: net.forward(x, scale), args.steps)
    clocks = sampler.stop()
    tf_train = 3.0 * fpi * B / (ms_train / 1000.0) / 1e12
    tf_fwd = fpi * B / (ms_fwd / 1000.0) / 1e12
    pk = peaks() or {}
    peak = pk.get("bf16_tflops_sustained", 1700.0)
    line = {
        "metric": "warm-start U-Net training throughput (BF16 tensor cores, FP32 accumulation)",
        "value": tf_train, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_train, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic", "config": {"workload": "unet4_c32_batch8_512x512", "batch": B, "image": [H, Wd],
                                        "flop_per_image_forward": fpi,
                                        "l2": "activations of one step (~1 GB) exceed the L2"},
        "forward_only": {"value": tf_fwd, "unit": "TFLOP/s", "ms_per_batch": ms_fwd},
        "roofline": {"kernel": "conv3x3_tma_kernel + wgrad3x3_tma_kernel (tcgen05, TMA)", "bound": "tensor",
                     "achieved": tf_train, "peak": peak, "unit": "TFLOP/s", "frac": tf_train / peak,
                     "traffic": None, "peak_basis": "measured cuBLAS BF16, sustained"},
        "gpu_launches": launches_per_step * args.steps, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    net.close()
    return 0


def main():
    args = parse()
    if args.workload == "cnn":
        return run_cnn(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
