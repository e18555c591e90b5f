"""Images with kappa electrons on the torus grid: the quadrature path against the oracle, and
the surrogate form against the quadrature path (its reference) and against the oracle.

- FP64 form (coefficients by the exact-grade quadrature at every emitting point) against the
  oracle as the FP64 form of thermal images is held: per pixel within 1e-9 outside the oracle's
  sensitivity mask, total flux within 1e-10, on a 32x32 image and on 545 pixels of the 1024x1024
  image (the lattice of every 64th pixel and the centres between, traced by rt_render_adaptive
  with an unreachable tolerance, so through the same kernels in a full-size camera); the mixed form (the
  tabulated quadrature, FP32 transfer) p99 within 3e-4 and flux within 1e-5 at 32x32.
- Surrogate: trained on 2^20 quadrature points drawn in the box that covers the 0.1-99.9
  percentiles of the image's emitting points; the 128^2 surrogate image against the
  quadrature image: flux within 1%, net LP and CP within 0.5 percentage points; a 32x32
  strided subsample of the 1024^2 surrogate image against the oracle, to the same bounds; and
  the speed-up of the surrogate form over the quadrature form at 256^2.
"""
import math
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

KAPPA = 4.5


@pytest.fixture(scope="module")
def rt():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2302_02733_gb300 import polrt

    torch.cuda.set_device(0)
    ctx = polrt.rt_create(0, torch.cuda.current_stream().cuda_stream)
    yield polrt, ctx
    polrt.rt_destroy(ctx)


def render(polrt, ctx, cam, form):
    polrt.rt_set_camera(ctx, cam)
    dt = torch.float64 if form == polrt.RT_FP64 else torch.float32
    out = torch.zeros((cam.ny, cam.nx, 4), dtype=dt, device="cuda")
    polrt.rt_render(ctx, form, out)
    return out.double().cpu().numpy(), polrt.rt_last_counters(ctx)


def rel_err(a, b):
    scale = np.maximum(b[..., 0], 1e-8 * b[..., 0].max())
    return np.abs(a - b).max(axis=-1) / scale


def pol(img):
    s = img.reshape(-1, 4).sum(axis=0)
    return s[0], math.hypot(s[1], s[2]) / s[0], s[3] / s[0]


def _mask(ora, ocam, om, ref, nsteps, ix, iy):
    from test_gpu_parity import oracle_mask

    return oracle_mask(ora, ocam, om, ref, nsteps, ix, iy)


def test_kappa_image_matches_oracle(rt, ora, synth, torus_grid):
    polrt, ctx = rt
    prims, g = torus_grid
    polrt.rt_load_model(ctx, polrt.grid_model(torch.from_numpy(prims).cuda(), g, kappa=KAPPA))
    polrt.rt_set_integrator(ctx, 0.05, 20000)
    n = 32
    cam = synth.Camera(incl_deg=20.0, nx=n, ny=n)
    ocam, om = ora.camera(cam), ora.grid_model(prims, g, kappa=KAPPA)
    iy, ix = np.mgrid[0:n, 0:n]
    ix, iy = ix.ravel(), iy.ravel()
    ref, nsteps, _, _ = ora.render_pixels(ocam, om, ix, iy)
    mask = _mask(ora, ocam, om, ref, nsteps, ix, iy).reshape(n, n)
    ref = ref.reshape(n, n, 4)
    g64, _ = render(polrt, ctx, cam, polrt.RT_FP64)
    g32, _ = render(polrt, ctx, cam, polrt.RT_MIXED)
    e64, e32 = rel_err(g64, ref), rel_err(g32, ref)
    f64, f32 = abs(g64[..., 0].sum() / ref[..., 0].sum() - 1), abs(g32[..., 0].sum() / ref[..., 0].sum() - 1)
    print(f"kappa 32x32: FP64 max {e64[~mask].max():.2e} (mask {mask.sum()}) flux {f64:.2e}; "
          f"mixed p99 {np.percentile(e32, 99):.2e} flux {f32:.2e}")
    assert ref[..., 0].max() > 0 and mask.mean() < 1e-2
    assert e64[~mask].max() <= 1e-9 and f64 <= 1e-10
    if mask.any():
        assert e64[mask].max() <= 1e-6
    assert np.percentile(e32, 99) <= 3e-4 and f32 <= 1e-5  # measured 4.6e-5 and 4.5e-7


def test_kappa_fp64_sampled_at_full_size(rt, ora, synth, torus_grid):
    polrt, ctx = rt
    prims, g = torus_grid
    polrt.rt_load_model(ctx, polrt.grid_model(torch.from_numpy(prims).cuda(), g, kappa=KAPPA))
    polrt.rt_set_integrator(ctx, 0.05, 20000)
    n = 1024
    cam = synth.Camera(incl_deg=20.0, nx=n, ny=n)
    polrt.rt_set_camera(ctx, cam)
    out = torch.zeros((n, n, 4), dtype=torch.float64, device="cuda")
    st = torch.zeros((n, n), dtype=torch.uint8, device="cuda")
    # the lattice (every 64th pixel and the last) and the first level's centres; blocks whose
    # rays end differently (across the shadow's edge) refine further, and are not compared. Those
    # refinement lists are made of long rays near the photon ring, which may outgrow the path
    # arena's per-ray budget (RT_ERR_WORKSPACE, the rays marked RT_RAY_OVERFLOW)
    rc = polrt.rt_render_adaptive(ctx, polrt.RT_FP64, out, st, 64, 1e300, check=False)
    assert rc in (polrt.RT_OK, polrt.RT_ERR_WORKSPACE)
    traced = polrt.rt_last_counters(ctx)["rays"]
    lat = list(range(0, n, 64)) + [n - 1]
    cen = list(range(32, n - 1, 64))
    pix = [(i, j) for j in lat for i in lat] + [(i, j) for j in cen for i in cen]
    ix, iy = np.array([p[0] for p in pix]), np.array([p[1] for p in pix])
    stc = st.cpu().numpy()[iy, ix]
    assert traced >= ix.size == 17 * 17 + 16 * 16 and (stc > 0).all() and (stc != polrt.RT_RAY_OVERFLOW).all()
    gpu = out.cpu().numpy()[iy, ix]
    ocam, om = ora.camera(cam), ora.grid_model(prims, g, kappa=KAPPA)
    ref, nsteps, _, _ = ora.render_pixels(ocam, om, ix, iy)
    mask = _mask(ora, ocam, om, ref, nsteps, ix, iy)
    e = rel_err(gpu, ref)
    print(f"kappa 1024^2, {ix.size} pixels: FP64 max {e[~mask].max():.2e} (mask {mask.sum()})")
    assert ref[:, 0].max() > 0 and mask.mean() < 1e-2
    assert e[~mask].max() <= 1e-9
    if mask.any():
        assert e[mask].max() <= 1e-6


def test_surrogate_image_against_quadrature(rt, ora, synth, torus_grid):
    polrt, ctx = rt
    prims, g = torus_grid
    polrt.rt_load_model(ctx, polrt.grid_model(torch.from_numpy(prims).cuda(), g, kappa=KAPPA))
    polrt.rt_set_integrator(ctx, 0.05, 20000)
    cam = synth.Camera(incl_deg=20.0, nx=128, ny=128)
    polrt.rt_set_camera(ctx, cam)
    # the training box: 0.1-99.9 percentiles of the image's emitting points; kappa over (3.2, 8)
    feat = torch.zeros((1 << 23, 4), dtype=torch.float32, device="cuda")
    cnt = polrt.rt_render_features(ctx, feat)
    f = feat[: min(cnt, feat.shape[0])]
    f = f[torch.isfinite(f).all(dim=1)]  # B along k or B = 0 has nu_c = 0: outside any box
    sub = f[torch.randperm(len(f), device="cuda")[: 1 << 20]]
    lo = torch.quantile(sub[:, :3], 0.001, dim=0).tolist()
    hi = torch.quantile(sub[:, :3], 0.999, dim=0).tolist()
    box_lo = [lo[0], max(lo[1], 1e-3), lo[2], 3.2]
    box_hi = [hi[0], min(hi[1], math.pi / 2), hi[2], 8.0]
    print(f"emitting points {cnt}; box lo {np.round(box_lo, 3)} hi {np.round(box_hi, 3)}")
    n = 1 << 20
    xs = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    ys = torch.empty((n, 8), dtype=torch.float32, device="cuda")
    vs = torch.empty((n,), dtype=torch.int32, device="cuda")
    polrt.rt_surrogate_dataset(ctx, box_lo + box_hi, n, 31, xs, ys, vs)
    assert vs.float().mean() > 0.99
    tn = torch.empty_like(ys)
    norm = polrt.rt_surrogate_fit(ctx, xs, ys, vs, tn, box_lo, box_hi)
    import oracle.mlp as M  # only for the initial weights' shapes

    rng = np.random.default_rng(32)
    theta = np.concatenate([np.concatenate([rng.uniform(-math.sqrt(3 / i), math.sqrt(3 / i), (o, i)),
                                            np.zeros((o, 1))], axis=1).ravel() for o, i in M.SHAPES])
    polrt.rt_mlp_set_params(ctx, theta.astype(np.float32), norm)
    keep = vs.bool()
    xs, tn = xs[keep].contiguous(), tn[keep].contiguous()
    curve = np.zeros(20000, dtype=np.float32)
    polrt.rt_mlp_train(ctx, xs, tn, 20000, 8192, 2e-3, 33, curve)
    print(f"training loss {curve[:10].mean():.3e} -> {curve[-100:].mean():.3e}")
    # the reference: quadrature image (mixed form) against the surrogate image
    q, cq = render(polrt, ctx, cam, polrt.RT_MIXED)
    s, cs = render(polrt, ctx, cam, polrt.RT_SURROGATE)
    e = rel_err(s, q)
    (fq, lpq, cpq), (fs, lps, cps) = pol(q), pol(s)
    print(f"surrogate vs quadrature 128^2: pixel p50 {np.median(e):.2e} p99 {np.percentile(e, 99):.2e}; "
          f"flux {abs(fs / fq - 1):.2e}; LP {lpq:.4f} vs {lps:.4f}; CP {cpq:.4f} vs {cps:.4f}")
    assert abs(fs / fq - 1) <= 1e-2 and abs(lps - lpq) <= 5e-3 and abs(cps - cpq) <= 5e-3
    # the surrogate form at full size against the oracle (quadrature), on every 32nd pixel
    camN = synth.Camera(incl_deg=20.0, nx=1024, ny=1024)
    sN, _ = render(polrt, ctx, camN, polrt.RT_SURROGATE)
    q = np.arange(32) * 32 + 16
    iy, ix = np.meshgrid(q, q, indexing="ij")
    ref = ora.render_pixels(ora.camera(camN), ora.grid_model(prims, g, kappa=KAPPA), ix.ravel(), iy.ravel())[0]
    sub = sN[iy, ix].reshape(-1, 4)
    (fo, lpo, cpo), (fs2, lps2, cps2) = pol(ref), pol(sub)
    print(f"surrogate 1024^2 (32x32 subsample) vs oracle: flux {abs(fs2 / fo - 1):.2e}; LP {lpo:.4f} vs {lps2:.4f}; "
          f"CP {cpo:.4f} vs {cps2:.4f}")
    assert abs(fs2 / fo - 1) <= 1e-2 and abs(lps2 - lpo) <= 5e-3 and abs(cps2 - cpo) <= 5e-3
    # what the network gains: the same image at 256^2 by quadrature and by the surrogate
    cam2 = synth.Camera(incl_deg=20.0, nx=256, ny=256)
    times = {}
    for name, form in (("quadrature", polrt.RT_MIXED), ("surrogate", polrt.RT_SURROGATE)):
        render(polrt, ctx, cam2, form)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        render(polrt, ctx, cam2, form)
        times[name] = time.perf_counter() - t0
    print(f"256^2 kappa image: quadrature {times['quadrature']:.2f} s, surrogate {times['surrogate']:.3f} s, "
          f"speed-up {times['quadrature'] / times['surrogate']:.1f}x")
    assert times["surrogate"] * 3 < times["quadrature"]
