"""The overlapped launch shape (geodesic of one ray chunk beside the transfer of the previous
chunk, on two streams and two halves of the workspace) against one pass of each kernel: every
ray takes the same arithmetic, so images, depth maps, status codes and step and point counts
are identical, for every form and for chunk counts that do and do not divide the rays. Also the
shape's argument checks and the automatic choice (one pass below 2^19 rays)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


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


def render(polrt, ctx, form, cam, cfg, depth=False):
    polrt.rt_set_render_config(ctx, *cfg)
    dt = torch.float64 if form == polrt.RT_FP64 else torch.float32
    shape = (cam.ny, cam.nx) if form == polrt.RT_UNPOL else (cam.ny, cam.nx, 4)
    out = torch.full(shape, float("nan"), dtype=dt, device="cuda")
    st = torch.zeros((cam.ny, cam.nx), dtype=torch.uint8, device="cuda")
    dep = None
    if depth:
        dep = torch.full((cam.ny, cam.nx, 2), float("nan"), dtype=dt, device="cuda")
        polrt.rt_render_depths(ctx, form, out, dep, st)
    else:
        polrt.rt_render(ctx, form, out, st)
    return out, st, dep, polrt.rt_last_counters(ctx)


def test_overlapped_render_is_identical(rt, synth, torus_grid):
    polrt, ctx = rt
    prims, g = torus_grid
    cam = synth.Camera(incl_deg=20.0, nx=200, ny=160)
    polrt.rt_set_integrator(ctx, 0.05, 20000)
    polrt.rt_set_camera(ctx, cam)
    polrt.rt_load_model(ctx, polrt.grid_model(torch.from_numpy(prims).cuda(), g))
    try:
        for form, depth in ((polrt.RT_MIXED, True), (polrt.RT_FP64, False), (polrt.RT_UNPOL, False)):
            ref, st0, d0, c0 = render(polrt, ctx, form, cam, (0, 0, 1), depth)
            assert c0["chunks"] == 1 and torch.isfinite(ref).all()
            for cfg in ((1, 0, 4), (2, 2, 3), (0, 0, 2), (1, 1, 7)):
                out, st, dep, c = render(polrt, ctx, form, cam, cfg, depth)
                assert c["chunks"] == cfg[2], (form, cfg)
                assert torch.equal(out, ref), (form, cfg)
                assert torch.equal(st, st0), (form, cfg)
                if depth:
                    assert torch.equal(dep, d0), (form, cfg)
                for k in ("rays", "steps", "points", "emitting_points", "n_horizon", "n_escape", "n_nmax"):
                    assert c[k] == c0[k], (form, cfg, k)
                assert c["n_overflow"] == 0 and c["ms_geodesic"] > 0 and c["ms_transfer"] > 0
        # automatic shape: one pass of each kernel for an image this small
        render(polrt, ctx, polrt.RT_MIXED, cam, (0, 0, 0))
        assert polrt.rt_last_counters(ctx)["chunks"] == 1
    finally:
        polrt.rt_set_render_config(ctx, 0, 0, 0)


def test_render_config_checks(rt):
    polrt, ctx = rt
    for bad in ((0, 0, 257), (0, 0, -1), (99, 0, 0), (0, 99, 0), (-1, 0, 0)):
        with pytest.raises(polrt.PolrtError):
            polrt.rt_set_render_config(ctx, *bad)
    polrt.rt_set_render_config(ctx, 1, 2, 8)
    assert polrt.rt_get_render_config(ctx) == {"geo_blocks_per_sm": 1, "xfer_blocks_per_sm": 2, "chunks": 8}
    polrt.rt_set_render_config(ctx, 0, 0, 0)
    assert polrt.rt_get_render_config(ctx) == {"geo_blocks_per_sm": 0, "xfer_blocks_per_sm": 0, "chunks": 0}


def test_overlapped_surrogate_is_identical(rt, synth, torus_grid):
    """The surrogate form through the overlapped shape: per chunk the features pass, the
    tensor-core network pass (its row count read on the device) and the transfer, in each
    workspace half. A fixed random network is enough: the check is that the shape does not
    change the image."""
    polrt, ctx = rt
    prims, g = torus_grid
    cam = synth.Camera(incl_deg=20.0, nx=160, ny=128)
    polrt.rt_set_integrator(ctx, 0.05, 20000)
    polrt.rt_set_camera(ctx, cam)
    polrt.rt_load_model(ctx, polrt.grid_model(torch.from_numpy(prims).cuda(), g, kappa=4.5))
    rng = np.random.default_rng(5)
    theta = (0.05 * rng.standard_normal(polrt.RT_MLP_PARAMS)).astype(np.float32)
    # targets near -30 (coefficients about e^-30 of their prefactors, as for cool electrons),
    # so the FP32 image stays finite
    norm = polrt.mlp_norm([-5.0, 1e-3, -6.0, 3.2], [40.0, 1.5707963, 4.0, 8.0], [-30.0] * 8, [0.01] * 8)
    polrt.rt_mlp_set_params(ctx, theta, norm)
    try:
        ref, st0, _, c0 = render(polrt, ctx, polrt.RT_SURROGATE, cam, (0, 0, 1))
        assert c0["chunks"] == 1 and torch.isfinite(ref).all() and ref[..., 0].max() > 0
        for cfg in ((1, 0, 4), (0, 0, 3)):
            out, st, _, c = render(polrt, ctx, polrt.RT_SURROGATE, cam, cfg)
            assert c["chunks"] == cfg[2]
            assert torch.equal(out, ref) and torch.equal(st, st0), cfg
            assert c["points"] == c0["points"] and c["steps"] == c0["steps"]
    finally:
        polrt.rt_set_render_config(ctx, 0, 0, 0)


def test_small_caller_workspace_falls_back_to_one_pass(rt, synth, torus_grid):
    """An overlapped shape that a caller's workspace cannot hold in at most 256 chunks renders
    in one pass of each kernel per chunk instead, with the same image."""
    polrt, ctx = rt
    prims, g = torus_grid
    cam = synth.Camera(incl_deg=20.0, nx=160, ny=128)
    polrt.rt_set_integrator(ctx, 0.05, 20000)
    polrt.rt_set_camera(ctx, cam)
    polrt.rt_load_model(ctx, polrt.grid_model(torch.from_numpy(prims).cuda(), g))
    ref, st0, _, _ = render(polrt, ctx, polrt.RT_MIXED, cam, (0, 0, 1))
    # about 1/400 of the image's rays: 400 sequential chunks, or 800 overlapped ones (over 256)
    ws = torch.empty(polrt.rt_workspace_hint(ctx) // 400, dtype=torch.uint8, device="cuda")
    polrt.rt_set_workspace(ctx, ws)
    try:
        out, st, _, c = render(polrt, ctx, polrt.RT_MIXED, cam, (1, 0, 8))
        assert c["chunks"] >= 256 and c["n_overflow"] == 0
        assert torch.equal(out, ref) and torch.equal(st, st0)
    finally:
        polrt.rt_set_workspace(ctx, None)
        polrt.rt_set_render_config(ctx, 0, 0, 0)


def test_probe_order_for_a_new_camera(rt, synth, torus_grid):
    """A new camera of 2^18 rays or more is first probed (one ray per 8 x 8 block) to predict
    the longest-first order; the image equals that of the next render, which uses the exact
    step counts the first one recorded."""
    polrt, ctx = rt
    prims, g = torus_grid
    cam = synth.Camera(incl_deg=33.0, nx=512, ny=512)  # a camera no other test renders
    polrt.rt_set_integrator(ctx, 0.05, 20000)
    polrt.rt_set_camera(ctx, cam)
    polrt.rt_load_model(ctx, polrt.grid_model(torch.from_numpy(prims).cuda(), g))
    first, st1, _, c1 = render(polrt, ctx, polrt.RT_MIXED, cam, (0, 0, 0))
    second, st2, _, c2 = render(polrt, ctx, polrt.RT_MIXED, cam, (0, 0, 0))
    assert torch.isfinite(first).all() and torch.equal(first, second) and torch.equal(st1, st2)
    assert c1["steps"] == c2["steps"] and c1["rays"] == 512 * 512 and c1["n_overflow"] == 0
