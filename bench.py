#!/usr/bin/env python
"""Benchmark of the polarized ray-tracing hot path on GB300.

Metric: Stokes-IQUV pixels/s for one 1024x1024 image of the GRMHD-shaped torus grid
(FMKS 288x128x128 FP32 primitives, R_high = 40, i = 20 deg, 230 GHz) in the chosen form
(RT_MIXED: FP64 geodesic, FP32 transfer), with the plain FP64 form timed beside it. One step
is one rt_render of the whole image (backward geodesics, path arena, forward transfer)
plus rt_image_stats, with inputs resident in HBM. The grid (151 MB) and the path arena
(tens of GB) are both larger than L2, so nothing is flushed between steps.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun (N > 1) every rank renders its own replica image (the method has no data
exchange between images); value = pixels of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Stokes-IQUV pixels/s at 1024^2, chosen form (FP64 geodesic + FP32 transfer) vs plain FP64 form"
# Algorithmic work per unit (derivation in the design notes): FP64 flops of one RK4 step of
# the geodesic (4 right-hand sides of the contracted Kerr-Schild connection + stage algebra),
# counting an FMA as 2 and sin, cos, a division or a square root as 1 each.
GEO_FLOP_PER_STEP = 612
XFER_FLOP_PER_POINT = {"fp64": 1450, "mixed": 1450}
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12   # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
# DRAM bytes (read + write) per RK4 step of geodesic_kernel: ncu dram__bytes_read.sum +
# dram__bytes_write.sum = 0.003515 + 1.424256 GB over 22,982,083 steps (torus, 256^2, one launch,
# the kernel as built now). The kernel's traffic is the path arena it writes (64 B per state), so
# it scales with the steps.
GEO_DRAM_BYTES_PER_STEP = (0.003515e9 + 1.424256e9) / 22982083


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--size", type=int, default=1024)
    ap.add_argument("--no-compare", action="store_true", help="skip the FP64-form comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-form (96-image library) leg")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the kappa/surrogate leg")
    ap.add_argument("--no-highres", action="store_true", help="skip the ADAF 4096^2 leg")
    ap.add_argument("--batch-images", type=int, default=96,
                    help="images of the library in the batched leg (the first ones of the 96)")
    ap.add_argument("--batch-mode", default="auto", choices=["auto", "persistent"],
                    help="persistent: mode 0 at a fixed balanced shape, no autotuner, no mode-1 or "
                         "unpolarized batches (a small device footprint, for profiling the persistent kernel)")
    ap.add_argument("--fetch", default="auto", choices=["auto", "gather", "staged"],
                    help="grid fetch of the FP32 transfer (rt_set_grid_fetch)")
    return ap.parse_args()


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str | None):
        self.idx = gpu_index
        self.proc = None

    def __enter__(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.idx is not None:
            cmd += ["-i", self.idx]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = [r.split(",") for r in (self.out or "").strip().splitlines() if r.strip()]
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower().startswith("active"):
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        load = [v for v in sm if v > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(v, device="cpu"):
    """The largest v over the ranks of the process group (v itself outside one)."""
    import torch

    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return v
    t = torch.tensor([v], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(ws, npix, seconds):
    """Whole-job throughput: every rank renders its own npix-pixel image (replicas), so the
    job does ws * npix pixels in the slowest rank's time."""
    return ws * npix / seconds


def workload(size):
    from paper_2302_02733_gb300 import synth

    cam = synth.Camera(incl_deg=20.0, nx=size, ny=size)
    prims, g = synth.fm_torus_grid(1)
    return cam, prims, g


def oracle_sample(cam, prims, g, npix, seed=0, nthreads=0):
    """Time the CPU oracle (as it stands; all host cores, or nthreads) on npix strided pixels."""
    import numpy as np

    import oracle

    stride = max(1, int(round((cam.nx * cam.ny / npix) ** 0.5)))
    iy, ix = np.meshgrid(np.arange(stride // 2, cam.ny, stride), np.arange(stride // 2, cam.nx, stride),
                         indexing="ij")
    ix, iy = ix.ravel()[:npix], iy.ravel()[:npix]
    ocam, om = oracle.camera(cam), oracle.grid_model(prims, g)
    t = time.perf_counter()
    ref = oracle.render_pixels(ocam, om, ix, iy, nthreads=nthreads)[0]
    dt = time.perf_counter() - t
    oracle_sample.last = (ix, iy, ref)
    return ix.size / dt, ix.size, stride, dt


def vs_oracle(img, ix, iy, ref):
    """Per-pixel error max_S |S - S_oracle| / max(I_oracle, 1e-8 max I_oracle) over the sampled
    pixels (p50, p99, max) and the error of their summed intensity."""
    import numpy as np

    g = img[iy, ix].double().cpu().numpy()
    scale = np.maximum(ref[:, 0], 1e-8 * ref[:, 0].max())
    err = np.abs(g - ref).max(axis=-1) / scale
    return {"pixels": int(ix.size), "pixel_rel_err_p50": float(np.median(err)),
            "pixel_rel_err_p99": float(np.percentile(err, 99)), "pixel_rel_err_max": float(err.max()),
            "sampled_flux_rel_err": float(abs(g[:, 0].sum() / ref[:, 0].sum() - 1))}


def run_reference(args):
    """The reference arm: the plain FP64 CPU oracle on a bounded sample per step."""
    ws, rank, _ = dist_env()
    if ws > 1 and rank != 0:
        return
    import oracle

    oracle.build()
    cam, prims, g = workload(args.size)
    npix = 1024
    for _ in range(args.warmup):
        oracle_sample(cam, prims, g, npix)
    rates, walls = [], []
    for _ in range(args.steps):
        r, n, stride, dt = oracle_sample(cam, prims, g, npix)
        rates.append(r)
        walls.append(dt)
    value = args.steps * n / sum(walls)
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pixels/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(walls) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded FM torus on an FMKS grid)",
            "config": {"workload": f"grmhd-torus-{args.size}x{args.size}", "grid": "288x128x128x8 f32",
                       "inclination_deg": 20, "freq_ghz": 230, "sample": f"{n} pixels, stride {stride}"},
            "cpu_baseline": {"value": value, "unit": "pixels/s", "cores": cores, "kind": "oracle",
                             "sample": f"{n} strided pixels of the {args.size}^2 image per step"},
            "e2e": {"value": value, "unit": "pixels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def batch_leg(polrt, ctx, prims_dev, g, dev, torch, nimg=96, mode="auto"):
    """rt_render_batch of the image library: 96 images, N in {128, 256, 512}, inclination
    10-170 deg, R_high 1-160, M_unit 1e17-1e20 g, mixed form; autotuned shape, graph replay.
    nimg < 96 takes the first nimg images; mode "persistent" runs mode 0 alone at a fixed shape."""
    from paper_2302_02733_gb300 import synth

    table = synth.batch_jobs(7, nimg)
    cams = [synth.Camera(incl_deg=j.incl_deg, nx=j.n, ny=j.n) for j in table]
    outs = [torch.empty((j.n, j.n, 4), dtype=torch.float32, device=dev) for j in table]
    jobs = polrt.make_jobs((c, j.M_unit, j.R_high, o, None, None) for c, j, o in zip(cams, table, outs))
    polrt.rt_load_model(ctx, polrt.grid_model(prims_dev, g))
    npix = sum(j.n * j.n for j in table)
    workload = f"image library: {nimg} images, N in {{128,256,512}}, torus grid, mixed form"
    if mode == "persistent":  # 3 and 4 geodesic warps in alternate 8-warp blocks, 2 blocks per SM
        polrt.rt_set_batch_config(ctx, polrt.RT_MIXED, 3, 1, 2, polrt.RT_BATCH_PERSISTENT, 4)
    polrt.rt_render_batch(ctx, polrt.RT_MIXED, jobs)  # autotune (mode auto), capture
    polrt.rt_render_batch(ctx, polrt.RT_MIXED, jobs)  # warm replay
    ms, steps = [], 0
    for _ in range(2):
        polrt.rt_render_batch(ctx, polrt.RT_MIXED, jobs)
        c = polrt.rt_last_counters(ctx)
        ms.append(c["ms_total"])
        steps = c["steps"]
    m = statistics.mean(ms)
    fp64 = steps * GEO_FLOP_PER_STEP / (m / 1e3) / 1e12
    shape = polrt.rt_get_batch_config(ctx, polrt.RT_MIXED)
    launch = {polrt.RT_BATCH_PERSISTENT: "one persistent kernel per batch, replayed from a CUDA graph",
              polrt.RT_BATCH_CHUNKS: "the images' rays as one ray space, in the overlapped two-kernel shape of rt_render"}
    res = {"workload": workload, "images": nimg,
           "pixels": npix, "value": npix / (m / 1e3), "unit": "pixels/s", "ms_per_batch": m,
           "launch": launch[shape["mode"]], "shape": shape,
           "geodesic_fp64_tflops": fp64, "geodesic_fp64_frac": fp64 / FP64_PEAK_TFLOPS}
    if mode == "persistent":
        return res
    # the other mode at the autotuner's best shape for it, for comparison
    other = polrt.RT_BATCH_PERSISTENT if shape["mode"] == polrt.RT_BATCH_CHUNKS else polrt.RT_BATCH_CHUNKS
    g, t, b = (shape["geo_warps"] or 4), (shape["step_tile"] or 1), (shape["blocks_per_sm"] or 2)
    go = shape.get("geo_warps_odd", 0)
    polrt.rt_set_batch_config(ctx, polrt.RT_MIXED, g, t, b, other, go)
    polrt.rt_render_batch(ctx, polrt.RT_MIXED, jobs)
    polrt.rt_render_batch(ctx, polrt.RT_MIXED, jobs)
    mo = polrt.rt_last_counters(ctx)["ms_total"]
    res["other_mode"] = {"launch": launch[other], "value": npix / (mo / 1e3), "ms_per_batch": mo}
    if polrt.RT_BATCH_PERSISTENT in (shape["mode"], other):
        if other != polrt.RT_BATCH_PERSISTENT:  # the last batch ran mode 1: run mode 0 once more
            polrt.rt_set_batch_config(ctx, polrt.RT_MIXED, g, t, b, polrt.RT_BATCH_PERSISTENT, go)
            polrt.rt_render_batch(ctx, polrt.RT_MIXED, jobs)
        st = polrt.rt_get_batch_stats(ctx)
        res["persistent_flow"] = {
            "geo_sleep_frac": st["geo_sleeps"] / max(st["geo_iters"], 1),
            "xfer_sleep_frac": st["xfer_sleeps"] / max(st["xfer_iters"], 1),
            "empty_polls_per_ticket": st["ticket_polls"] / max(st["tickets"], 1),
            "ready_polls_per_ray": st["ready_polls"] / npix, "free_spins": st["free_spins"], "raw": st}
    # the same library unpolarized (the fitting loop's form; always mode 1)
    uouts = [torch.empty((j.n, j.n), dtype=torch.float32, device=dev) for j in table]
    ujobs = polrt.make_jobs((c, j.M_unit, j.R_high, o, None, None) for c, j, o in zip(cams, table, uouts))
    polrt.rt_render_batch(ctx, polrt.RT_UNPOL, ujobs)
    polrt.rt_render_batch(ctx, polrt.RT_UNPOL, ujobs)
    mu = polrt.rt_last_counters(ctx)["ms_total"]
    res["unpolarized"] = {"launch": launch[polrt.RT_BATCH_CHUNKS], "value": npix / (mu / 1e3), "ms_per_batch": mu}
    return res


def highres_leg(polrt, ctx, dev, torch):
    """The 64^2 ADAF camera at 4096^2 in the mixed form: time the second render (rays longest
    first, as for any repeated camera), and check a 64 x 64 strided subsample of pixel centres
    against the CPU oracle."""
    import numpy as np

    import oracle
    from paper_2302_02733_gb300 import synth

    n = 4096
    cam = synth.Camera(incl_deg=60.0, nx=n, ny=n)
    par = synth.adaf_params(1)
    polrt.rt_set_camera(ctx, cam)
    polrt.rt_load_model(ctx, polrt.adaf_model(par))
    img = torch.empty((n, n, 4), dtype=torch.float32, device=dev)
    polrt.rt_render(ctx, polrt.RT_MIXED, img)
    polrt.rt_render(ctx, polrt.RT_MIXED, img)
    c = polrt.rt_last_counters(ctx)
    q = np.arange(64) * 64 + 32
    sub = img[q][:, q].double().cpu().numpy()
    iy, ix = np.meshgrid(q, q, indexing="ij")
    oracle.build()
    ref = oracle.render_pixels(oracle.camera(cam), oracle.adaf_model(par), ix.ravel(), iy.ravel())[0]
    ref = ref.reshape(64, 64, 4)
    scale = np.maximum(ref[..., 0], 1e-8 * ref[..., 0].max())
    err = np.abs(sub - ref).max(axis=-1) / scale
    del img
    return {"workload": "ADAF (seed 1), i = 60 deg, 4096^2, mixed form", "value": n * n / (c["ms_total"] / 1e3),
            "unit": "pixels/s", "ms_per_image": c["ms_total"], "chunks": c["chunks"],
            "shape": {0: "one pass", 1: "overlapped halves", 2: "streamed"}[c["shape"]],
            "geodesic_launches": c["geodesic_launches"], "transfer_launches": c["transfer_launches"],
            "vs_oracle_64x64": {"pixel_rel_err_p99": float(np.percentile(err, 99)), "pixel_rel_err_max": float(err.max()),
                                "flux_rel_err": float(abs(sub[..., 0].sum() / ref[..., 0].sum() - 1))}}


def surrogate_leg(polrt, ctx, prims_dev, g, dev, torch, size):
    """Kappa electrons (kappa drawn from U(3, 8) with a fixed seed) on the torus grid: train the
    surrogate on 2^20 quadrature points in the box of the image's features (below), time the
    RT_SURROGATE image at size^2, check it against the quadrature image at 128^2, and time both
    forms at 256^2."""
    import math

    import numpy as np
    from paper_2302_02733_gb300 import synth

    kappa = 3.0 + 5.0 * float(synth.uniform(2302, [0])[0])
    polrt.rt_load_model(ctx, polrt.grid_model(prims_dev, g, kappa=kappa))
    cam128 = synth.Camera(incl_deg=20.0, nx=128, ny=128)
    polrt.rt_set_camera(ctx, cam128)
    feat = torch.zeros((1 << 22, 4), dtype=torch.float32, device=dev)
    cnt = polrt.rt_render_features(ctx, feat)
    f = feat[: min(cnt, feat.shape[0])]
    f = f[torch.isfinite(f).all(dim=1)]
    sub = f[torch.randperm(len(f), device=dev, generator=torch.Generator(device=dev).manual_seed(2302))[: 1 << 20]]
    # the box: the 128^2 image's 0.001-99.999 percentiles widened by 5% of their range, so that
    # few points of the full-size image fall back to the quadrature
    qlo = torch.quantile(sub[:, :3], 1e-5, dim=0)
    qhi = torch.quantile(sub[:, :3], 1.0 - 1e-5, dim=0)
    lo, hi = (qlo - 0.05 * (qhi - qlo)).tolist(), (qhi + 0.05 * (qhi - qlo)).tolist()
    box_lo, box_hi = [lo[0], max(lo[1], 1e-3), lo[2], 3.2], [hi[0], min(hi[1], math.pi / 2), hi[2], 8.0]
    t0 = time.perf_counter()
    n = 1 << 20
    xs = torch.empty((n, 4), dtype=torch.float32, device=dev)
    ys = torch.empty((n, 8), dtype=torch.float32, device=dev)
    vs = torch.empty((n,), dtype=torch.int32, device=dev)
    polrt.rt_surrogate_dataset(ctx, box_lo + box_hi, n, 2302, xs, ys, vs)
    tn = torch.empty_like(ys)
    norm = polrt.rt_surrogate_fit(ctx, xs, ys, vs, tn, box_lo, box_hi)
    rng = np.random.default_rng(2302)
    shapes = [(64, 4), (64, 64), (64, 64), (8, 64)]
    theta = np.concatenate([np.concatenate([rng.uniform(-math.sqrt(3 / i), math.sqrt(3 / i), (o, i)),
                                            np.zeros((o, 1))], axis=1).ravel() for o, i in shapes])
    polrt.rt_mlp_set_params(ctx, theta.astype(np.float32), norm)
    keep = vs.bool()
    steps = 40000
    curve = np.zeros(steps, dtype=np.float32)
    polrt.rt_mlp_train(ctx, xs[keep].contiguous(), tn[keep].contiguous(), steps, 8192, 2e-3, 2302, curve)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0

    def img(cam, form):
        polrt.rt_set_camera(ctx, cam)
        o = torch.empty((cam.ny, cam.nx, 4), dtype=torch.float32, device=dev)
        polrt.rt_render(ctx, form, o)
        return o

    def pol(o):
        s_ = o.double().sum(dim=(0, 1)).cpu().numpy()
        return s_[0], math.hypot(s_[1], s_[2]) / s_[0], s_[3] / s_[0]

    (fq, lq, cq), (fs, ls, cs) = pol(img(cam128, polrt.RT_MIXED)), pol(img(cam128, polrt.RT_SURROGATE))
    cam256 = synth.Camera(incl_deg=20.0, nx=256, ny=256)
    t256 = {}
    for name, form in (("quadrature", polrt.RT_MIXED), ("surrogate", polrt.RT_SURROGATE)):
        img(cam256, form)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        img(cam256, form)
        torch.cuda.synchronize()
        t256[name] = time.perf_counter() - t1
    camN = synth.Camera(incl_deg=20.0, nx=size, ny=size)
    img(camN, polrt.RT_SURROGATE)
    reps, ms = 2, []
    for _ in range(reps):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        img(camN, polrt.RT_SURROGATE)
        torch.cuda.synchronize()
        ms.append((time.perf_counter() - t1) * 1e3)
    m = statistics.mean(ms)
    return {"workload": f"kappa electrons (kappa {kappa:.2f}) on the torus grid, {size}^2, RT_SURROGATE",
            "value": size * size / (m / 1e3), "unit": "pixels/s", "ms_per_image": m,
            "training": {"samples": n, "steps": steps, "batch": 8192, "seconds": train_s,
                         "final_loss": float(curve[-100:].mean())},
            "vs_quadrature_128": {"flux_rel_err": abs(fs / fq - 1), "lp": [lq, ls], "cp": [cq, cs]},
            "speedup_256_vs_quadrature": t256["quadrature"] / t256["surrogate"]}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2302_02733_gb300 import build, polrt, synth

    build.build()
    dev = f"cuda:{local}"
    stream = torch.cuda.current_stream()
    cam, prims, g = workload(args.size)
    npix = cam.nx * cam.ny
    form = polrt.RT_MIXED if args.form == "mixed" else polrt.RT_FP64
    odt = torch.float32 if form == polrt.RT_MIXED else torch.float64
    ctx = polrt.rt_create(local, stream.cuda_stream)
    polrt.rt_set_grid_fetch(ctx, {"auto": polrt.RT_FETCH_AUTO, "gather": polrt.RT_FETCH_GATHER,
                                  "staged": polrt.RT_FETCH_STAGED}[args.fetch])
    polrt.rt_set_camera(ctx, cam)
    prims_dev = torch.from_numpy(prims).to(dev)
    polrt.rt_load_model(ctx, polrt.grid_model(prims_dev, g))
    out = torch.empty((cam.ny, cam.nx, 4), dtype=odt, device=dev)

    def step(f=form, o=out):
        polrt.rt_render(ctx, f, o)
        polrt.rt_image_stats(ctx, o, f)

    for _ in range(max(args.warmup, 3)):
        step()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local] if ws == 1 else None
    kt_geo, kt_xf, counters, launches = [], [], None, 0
    barrier()
    torch.cuda.synchronize()
    with Clocks(gpu_index) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
            counters = polrt.rt_last_counters(ctx)
            kt_geo.append(counters["ms_geodesic"])
            kt_xf.append(counters["ms_transfer"])
            # the geodesic and transfer launches, and the two image-sum kernels
            launches += counters["geodesic_launches"] + counters["transfer_launches"] + 2
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = max_over_ranks(ms, dev)
    value = job_rate(ws, npix, ms_max / 1e3)

    # per-kernel roofline of the dominant kernel (measured live with CUDA events in the library).
    # In the overlapped launch shapes the geodesic shares the SMs with the transfers, so its
    # durations include that sharing; the kernel alone (one pass of each kernel, the shape used
    # below 2^19 rays) is timed once after the timed region.
    geo_ms, xf_ms = statistics.mean(kt_geo), statistics.mean(kt_xf)
    steps_per_launch = counters["steps"]
    pts_per_launch = counters["points"]
    geo_launches = max(counters["geodesic_launches"], 1)
    shape_note = {0: "one launch per image",
                  1: "overlapped in two workspace halves: each geodesic launch shares the SMs with the "
                     "transfer of the previous chunk",
                  2: "streamed: one geodesic launch per image beside the transfers of its completed chunks "
                     f"({counters['transfer_launches']} transfer launches)"}[counters["shape"]]
    polrt.rt_set_render_config(ctx, 0, 0, 1)
    step()
    alone = polrt.rt_last_counters(ctx)
    polrt.rt_set_render_config(ctx, 0, 0, 0)
    if geo_ms >= xf_ms:
        achieved = steps_per_launch * GEO_FLOP_PER_STEP / (geo_ms / 1e3) / 1e12
        achieved_alone = steps_per_launch * GEO_FLOP_PER_STEP / (alone["ms_geodesic"] / 1e3) / 1e12
        dom = "geodesic_kernel (FP64 RK4)"
    else:
        achieved = pts_per_launch * XFER_FLOP_PER_POINT[args.form] / (xf_ms / 1e3) / 1e12
        achieved_alone = pts_per_launch * XFER_FLOP_PER_POINT[args.form] / (alone["ms_transfer"] / 1e3) / 1e12
        dom = f"transfer_kernel ({args.form})"
    traffic = GEO_DRAM_BYTES_PER_STEP * steps_per_launch / geo_launches if geo_ms >= xf_ms else None
    try:
        probe = polrt.rt_fp64_fma_peak(local)  # measured FP64 FMA rate of this device
    except polrt.PolrtError:
        probe = None
    roof = {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
            "traffic_source": "bytes per launch, scaled by steps from the ncu capture of the 256^2 case",
            "peak_source": "FP64 pipe: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (nominal 1.25 TFLOP/s)",
            "launches_per_image": geo_launches,
            "note": shape_note,
            "measured_fp64_fma_peak": probe,
            "frac_of_measured_fma_peak": (achieved / probe) if probe else None,
            "alone": {"achieved": achieved_alone, "frac": achieved_alone / FP64_PEAK_TFLOPS,
                      "frac_of_measured_fma_peak": (achieved_alone / probe) if probe else None,
                      "ms_geodesic": alone["ms_geodesic"], "ms_transfer": alone["ms_transfer"],
                      "ms_total": alone["ms_total"]}}

    extra = {"kernel_ms": {"geodesic": geo_ms, "transfer": xf_ms}, "steps_per_image": steps_per_launch,
             "points_per_image": pts_per_launch, "mean_steps_per_ray": steps_per_launch / npix}

    # the plain FP64 form on the same image
    o64 = None
    if not args.no_compare and form != polrt.RT_FP64:
        o64 = torch.empty((cam.ny, cam.nx, 4), dtype=torch.float64, device=dev)
        step(polrt.RT_FP64, o64)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = 2
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(reps):
            step(polrt.RT_FP64, o64)
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1) / reps
        c64 = polrt.rt_last_counters(ctx)
        ref = o64.cpu().numpy()
        mix = out.double().cpu().numpy()
        scale = np.maximum(ref[..., 0], 1e-8 * ref[..., 0].max())
        err = np.abs(mix - ref).max(axis=-1) / scale
        extra["fp64_form"] = {"value": npix / (ms64 / 1e3), "unit": "pixels/s", "ms_per_step": ms64,
                              "kernel_ms": {"geodesic": c64["ms_geodesic"], "transfer": c64["ms_transfer"]}}
        extra["chosen_vs_fp64"] = {"speedup": ms64 / ms, "pixel_rel_err_p50": float(np.median(err)),
                                   "pixel_rel_err_p99": float(np.percentile(err, 99)),
                                   "pixel_rel_err_max": float(err.max()),
                                   "flux_rel_err": float(abs(mix[..., 0].sum() / ref[..., 0].sum() - 1))}

    # end to end through the C ABI with host buffers: prims H2D from pinned memory, image D2H
    e2e = None
    if not args.no_e2e:
        host_prims = torch.from_numpy(prims).pin_memory()
        host_out = torch.empty((cam.ny, cam.nx, 4), dtype=odt).pin_memory()
        model_h = polrt.grid_model(host_prims, g)
        polrt.rt_load_model(ctx, model_h)
        polrt.rt_render(ctx, form, host_out)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            polrt.rt_load_model(ctx, model_h)
            polrt.rt_render(ctx, form, host_out)
            polrt.rt_image_stats(ctx, host_out, form)
        torch.cuda.synchronize()
        dt = max_over_ranks((time.perf_counter() - t0) / args.steps, dev)
        e2e = {"value": job_rate(ws, npix, dt), "unit": "pixels/s", "h2d_bytes_per_step": int(prims.nbytes),
               "d2h_bytes_per_step": int(host_out.numel() * host_out.element_size()), "ms_per_step": dt * 1e3}

    # batched form: the 96-image library in one persistent launch per batch (graph replay)
    if not args.no_batch and ws == 1:
        extra["batched_form"] = batch_leg(polrt, ctx, prims_dev, g, dev, torch, args.batch_images, args.batch_mode)
    # the high-resolution ADAF image
    if not args.no_highres and ws == 1:
        extra["highres_form"] = highres_leg(polrt, ctx, dev, torch)
    # surrogate form: kappa electrons through the trained network
    if not args.no_surrogate and ws == 1:
        extra["surrogate_form"] = surrogate_leg(polrt, ctx, prims_dev, g, dev, torch, args.size)

    cpu = None
    if rank == 0 and not args.no_cpu:
        import oracle

        oracle.build()
        rate, n, stride, dt = oracle_sample(cam, prims, g, 8192)
        sample = oracle_sample.last
        rate1, n1, stride1, dt1 = oracle_sample(cam, prims, g, 512, nthreads=1)
        # the benchmark image (and the FP64 form's) against the oracle on the timed sample
        extra["vs_oracle_sample"] = {"chosen_form": vs_oracle(out, *sample)}
        if o64 is not None:
            extra["vs_oracle_sample"]["fp64_form"] = vs_oracle(o64, *sample)
        cpu = {"value": rate, "unit": "pixels/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{n} pixels (stride {stride}) of the {cam.nx}^2 image, {dt:.1f} s",
               "single_thread": {"value": rate1, "unit": "pixels/s", "cores": 1,
                                 "sample": f"{n1} pixels (stride {stride1}) of the {cam.nx}^2 image, {dt1:.1f} s"}}

    polrt.rt_destroy(ctx)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "pixels/s", "n_gpus": ws, "steps": args.steps,
                "warmup": max(args.warmup, 3), "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64 geodesic + f32 transfer" if form == polrt.RT_MIXED else "f64",
                "data": "synthetic (seeded FM torus on an FMKS grid, log-normal perturbations)",
                "config": {"workload": f"grmhd-torus-{cam.nx}x{cam.ny}", "grid": "288x128x128x8 f32",
                           "inclination_deg": 20, "freq_ghz": 230, "form": args.form, "grid_fetch": args.fetch,
                           "beta_min": synth.TorusParams().beta_min,
                           "perturbation_sigma": synth.TorusParams().sigma_pert,
                           "R_high": 40, "M_unit_g": 1e19,
                           "parallelism": f"replicas x{ws}",
                           "l2": "inputs larger than L2 (151 MB grid, multi-GB path arena); no flush"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk.summary(),
                "gpu_launches": launches, **extra}
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
