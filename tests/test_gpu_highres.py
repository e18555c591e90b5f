"""High resolution: the ADAF (a = 0.9375, i = 60 deg, 230 GHz, 40 M field of view) at 4096^2 in
the mixed form, against the FP64 oracle on the 256^2 subsample of pixel centres
(16p + 8, 16q + 8). Tolerances are those of the mixed form at 64^2 (per-pixel p99 <= 5e-6,
flux and net LP/CP of the subsample within 1e-6), with the per-pixel maximum at 1e-4: the
subsample reaches 16x deeper into the photon ring, where one-ulp changes of the initial
direction move the oracle itself."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_adaf_4096_mixed_against_subsample(ora, synth):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2302_02733_gb300 import polrt

    torch.cuda.set_device(0)
    ctx = polrt.rt_create(0, torch.cuda.current_stream().cuda_stream)
    try:
        cam = synth.Camera(incl_deg=60.0, nx=4096, ny=4096)
        par = synth.adaf_params(1)
        polrt.rt_set_camera(ctx, cam)
        polrt.rt_load_model(ctx, polrt.adaf_model(par))
        img = torch.zeros((4096, 4096, 4), dtype=torch.float32, device="cuda")
        st = torch.zeros((4096, 4096), dtype=torch.uint8, device="cuda")
        t0 = time.perf_counter()
        polrt.rt_render(ctx, polrt.RT_MIXED, img, st)
        wall = time.perf_counter() - t0
        cnt = polrt.rt_last_counters(ctx)
        f_full, lp_full, cp_full = polrt.rt_image_stats(ctx, img, polrt.RT_MIXED)
        q = np.arange(256) * 16 + 8
        sub = img[q][:, q].double().cpu().numpy()
        sst = st[q][:, q].cpu().numpy()
    finally:
        polrt.rt_destroy(ctx)
    iy, ix = np.meshgrid(q, q, indexing="ij")
    ref, nsteps, status, _ = ora.render_pixels(ora.camera(cam), ora.adaf_model(par), ix.ravel(), iy.ravel())
    ref = ref.reshape(256, 256, 4)
    assert np.array_equal(sst.astype(np.int64).ravel(), status.astype(np.int64))
    scale = np.maximum(ref[..., 0], 1e-8 * ref[..., 0].max())
    err = np.abs(sub - ref).max(axis=-1) / scale
    f_err = abs(sub[..., 0].sum() / ref[..., 0].sum() - 1)

    def pol(x):
        s = x.reshape(-1, 4).sum(axis=0)
        return np.hypot(s[1], s[2]) / s[0], s[3] / s[0]

    dlp, dcp = (abs(a - b) for a, b in zip(pol(sub), pol(ref)))
    print(f"adaf4096 mixed: {16.7772e6 / wall:.3e} px/s wall ({cnt['ms_geodesic']:.0f} + {cnt['ms_transfer']:.0f} ms "
          f"first chunk), full flux {f_full:.4e} Jy LP {lp_full:.4f} CP {cp_full:.2e}; subsample p50 "
          f"{np.median(err):.2e} p99 {np.percentile(err, 99):.2e} max {err.max():.2e} flux {f_err:.2e} "
          f"dLP {dlp:.1e} dCP {dcp:.1e}")
    assert cnt["n_overflow"] == 0 and cnt["rays"] == 4096 * 4096
    assert np.percentile(err, 99) <= 5e-6 and err.max() <= 1e-4
    assert f_err <= 1e-6 and dlp <= 1e-6 and dcp <= 1e-6
