"""The overlapped launch shapes against one pass of each kernel: streamed (one geodesic launch
over all rays, each chunk's transfer launched as the chunk completes) and in two halves of the
workspace (the geodesic of one chunk beside the transfer of the previous). Every ray takes the
same arithmetic, so images, depth maps, status codes and step and point counts are identical,
for every form, for chunk counts that do and do not divide the rays and for a smaller last
chunk. Also the per-chunk timeline, the shape's argument checks and the automatic choice (one
pass below 2^19 rays)."""
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


def check_timeline(tl, K, shape):
    """The launch order of the overlapped shapes, read from the per-chunk events.
    Streamed (shape 2): the chunks of a piece report the piece's one geodesic launch; a transfer
    covers a run of complete chunks of one piece (which report the same launch), transfers run
    one after another on their stream, and a piece's geodesic starts after the previous piece's
    transfers have ended. Two halves (shape 1): each stream runs its launches in order, a
    transfer starts after its chunk's geodesic, and a geodesic after the transfer that last
    used its half (chunk k - 2)."""
    assert len(tl) == K
    eps = 1e-3  # event resolution, ms
    assert tl[0][0] == 0.0
    for k, (gs, ge, ts, te) in enumerate(tl):
        assert ge >= gs - eps and te >= ts - eps and ts >= -eps, (k, tl[k])
    if shape == 2:
        runs = sorted((t[2], t[3]) for t in tl)
        for (s0, e0), (s1, e1) in zip(runs, runs[1:]):
            same = abs(s1 - s0) < 0.01 and abs(e1 - e0) < 0.01  # chunks of one launch
            assert same or s1 >= e0 - eps, (s0, e0, s1, e1)
        pieces = sorted({(t[0], t[1]) for t in tl})
        for (g0, g1) in pieces:
            mine = [t for t in tl if (t[0], t[1]) == (g0, g1)]
            assert all(t[2] >= g0 - eps for t in mine)
            later = [t for t in tl if t[0] > g0 + eps]
            if later:
                assert min(t[0] for t in later) >= max(t[3] for t in mine) - eps
        return len(pieces)
    for k, (gs, ge, ts, te) in enumerate(tl):
        assert ts >= ge - eps, (k, tl[k])
        if k >= 1:
            assert gs >= tl[k - 1][1] - eps and ts >= tl[k - 1][3] - eps, k
        if k >= 2:
            assert gs >= tl[k - 2][3] - eps, k
    return 0


def test_overlapped_render_is_identical(rt, synth, torus_grid):
    """Streamed in one piece (the library's workspace holds every path), streamed in three
    pieces (a caller's workspace of 0.45 of the image's), and in two halves (a caller's
    workspace of 1/80 of it: a piece would hold under 1/64 of the rays), with equal chunks and,
    in halves, with a smaller last chunk."""
    polrt, ctx = rt
    prims, g = torus_grid
    cam = synth.Camera(incl_deg=20.0, nx=200, ny=160)
    polrt.rt_set_integrator(ctx, 0.05, 20000)
    polrt.rt_set_camera(ctx, cam)
    polrt.rt_load_model(ctx, polrt.grid_model(torch.from_numpy(prims).cuda(), g))
    shapes = ((1.0, ((1, 0, 4), (2, 2, 3), (0, 0, 2), (1, 1, 7))),
              (0.45, ((2, 0, 4), (1, 1, 7))),
              (1 / 80, ((1, 0, 4), (1, 1, 7, 4))))
    try:
        for form, depth in ((polrt.RT_MIXED, True), (polrt.RT_FP64, False), (polrt.RT_UNPOL, False)):
            ref, st0, d0, c0 = render(polrt, ctx, form, cam, (0, 0, 1), depth)
            assert c0["chunks"] == 1 and c0["shape"] == 0 and torch.isfinite(ref).all()
            for frac, cfgs in shapes:
                if frac < 1.0:
                    ws = torch.empty(int(frac * polrt.rt_workspace_hint(ctx)), dtype=torch.uint8, device="cuda")
                    polrt.rt_set_workspace(ctx, ws)
                for cfg in cfgs:
                    out, st, dep, c = render(polrt, ctx, form, cam, cfg, depth)
                    assert torch.equal(out, ref), (form, frac, cfg)
                    assert torch.equal(st, st0), (form, frac, cfg)
                    if depth:
                        assert torch.equal(dep, d0), (form, frac, cfg)
                    for k in ("rays", "steps", "points", "emitting_points", "n_horizon", "n_escape", "n_nmax"):
                        assert c[k] == c0[k], (form, cfg, k)
                    assert c["n_overflow"] == 0 and c["ms_geodesic"] > 0 and c["ms_transfer"] > 0
                    tl = polrt.rt_last_timeline(ctx)
                    if frac == 1.0:
                        assert c["shape"] == 2 and c["chunks"] == cfg[2] and c["geodesic_launches"] == 1
                        assert check_timeline(tl, c["chunks"], 2) == 1
                    elif frac > 0.1:
                        assert c["shape"] == 2 and c["chunks"] == 3 * cfg[2] and c["geodesic_launches"] == 3
                        assert check_timeline(tl, c["chunks"], 2) == 3
                    else:
                        assert c["shape"] == 1 and c["chunks"] >= 160 and c["geodesic_launches"] == c["chunks"]
                        check_timeline(tl, c["chunks"], 1)
                    assert 1 <= c["transfer_launches"] <= c["chunks"]
                if frac < 1.0:
                    polrt.rt_set_workspace(ctx, None)
        # automatic shape: one pass of each kernel for an image this small
        render(polrt, ctx, polrt.RT_MIXED, cam, (0, 0, 0))
        assert polrt.rt_last_counters(ctx)["chunks"] == 1
        assert polrt.rt_last_timeline(ctx) == []
    finally:
        polrt.rt_set_workspace(ctx, None)
        polrt.rt_set_render_config(ctx, 0, 0, 0)


def test_render_config_checks(rt):
    polrt, ctx = rt
    for bad in ((0, 0, 257), (0, 0, -1), (99, 0, 0), (0, 99, 0), (-1, 0, 0), (0, 0, 4, 17), (0, 0, 4, -1)):
        with pytest.raises(polrt.PolrtError):
            polrt.rt_set_render_config(ctx, *bad)
    polrt.rt_set_render_config(ctx, 1, 2, 8, 4)
    assert polrt.rt_get_render_config(ctx) == {"geo_blocks_per_sm": 1, "xfer_blocks_per_sm": 2, "chunks": 8,
                                               "last_chunk_div": 4}
    polrt.rt_set_render_config(ctx, 0, 0, 0)
    assert polrt.rt_get_render_config(ctx) == {"geo_blocks_per_sm": 0, "xfer_blocks_per_sm": 0, "chunks": 0,
                                               "last_chunk_div": 0}


def test_overlapped_surrogate_is_identical(rt, synth, torus_grid):
    """The surrogate form through the overlapped shapes: streamed, where each transfer launch's
    rays get compact rows for the features pass and the tensor-core network pass (its row count
    read on the device); and in two halves, per chunk over the half's arena (a caller's
    workspace of 1/50 of the thermal image's: a streamed piece would hold under 1/64 of the
    rays, a half about 1/175). A fixed random network is enough: the check is that the shape
    does not change the image."""
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
        # streamed (the network over each transfer launch's compact rows), then in two halves
        for frac, cfgs, shape in ((1.0, ((1, 0, 4), (0, 0, 3)), 2), (1 / 50, ((1, 0, 4),), 1)):
            if frac < 1.0:
                ws = torch.empty(int(frac * polrt.rt_workspace_hint(ctx)), dtype=torch.uint8, device="cuda")
                polrt.rt_set_workspace(ctx, ws)
            for cfg in cfgs:
                out, st, _, c = render(polrt, ctx, polrt.RT_SURROGATE, cam, cfg)
                assert c["shape"] == shape, (frac, cfg)
                if shape == 2:
                    assert c["chunks"] == cfg[2]
                assert torch.equal(out, ref) and torch.equal(st, st0), (frac, cfg)
                assert c["points"] == c0["points"] and c["steps"] == c0["steps"]
            if frac < 1.0:
                polrt.rt_set_workspace(ctx, None)
    finally:
        polrt.rt_set_workspace(ctx, None)
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


def test_streamed_image_with_probed_then_recorded_order(rt, synth, torus_grid):
    """The automatic shape of a new 1024^2 camera: streamed, its first render in the order the
    probe predicts, the next in the order the first recorded (a different cut of the rays into
    chunks and transfer launches); the images and counts agree with one pass of each kernel."""
    polrt, ctx = rt
    prims, g = torus_grid
    cam = synth.Camera(incl_deg=27.0, nx=1024, ny=1024)  # a camera no other test renders
    polrt.rt_set_integrator(ctx, 0.05, 20000)
    polrt.rt_set_camera(ctx, cam)
    polrt.rt_load_model(ctx, polrt.grid_model(torch.from_numpy(prims).cuda(), g))
    try:
        first, st1, _, c1 = render(polrt, ctx, polrt.RT_MIXED, cam, (0, 0, 0))
        assert c1["shape"] == 2 and c1["geodesic_launches"] == 1
        second, st2, _, c2 = render(polrt, ctx, polrt.RT_MIXED, cam, (0, 0, 0))
        ref, st0, _, c0 = render(polrt, ctx, polrt.RT_MIXED, cam, (0, 0, 1))
        assert c0["shape"] == 0 and torch.isfinite(ref).all()
        for img, st, c in ((first, st1, c1), (second, st2, c2)):
            assert torch.equal(img, ref) and torch.equal(st, st0)
            assert c["steps"] == c0["steps"] and c["points"] == c0["points"] and c["n_overflow"] == 0
    finally:
        polrt.rt_set_render_config(ctx, 0, 0, 0)
