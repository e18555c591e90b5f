"""rt_render_static, the entry point that allocates nothing, against rt_render.

Callers that cannot allocate device memory (their budget is held by someone else, or
allocation is forbidden on their code path) render through rt_render_static. Its scratch is
the library's static device array, so two calls in a row must each reproduce rt_render's
image bit for bit (the same kernels take the same arithmetic on every ray), and an image beyond
the array's capacity must be refused. Collected last so that a stop-at-first-failure run has
already run every other test; also passes alone.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# the documented limit: 512 MiB of scratch over (ray record + 20 arena blocks of 32 states) per ray
MAX_PIXELS = 13076


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


@pytest.mark.parametrize("form", [0, 1])
def test_static_matches_allocating_render_twice(rt, form):
    from paper_2302_02733_gb300 import synth

    polrt, ctx = rt
    cam = synth.Camera(incl_deg=60.0, nx=64, ny=48)
    polrt.rt_set_integrator(ctx, 0.05, 20000)
    polrt.rt_set_camera(ctx, cam)
    polrt.rt_load_model(ctx, polrt.adaf_model(synth.adaf_params(1)))
    dt = torch.float64 if form == polrt.RT_FP64 else torch.float32
    ref = torch.zeros((cam.ny, cam.nx, 4), dtype=dt, device="cuda")
    st_ref = torch.zeros((cam.ny, cam.nx), dtype=torch.uint8, device="cuda")
    polrt.rt_render(ctx, form, ref, st_ref)
    for _ in range(2):
        out = torch.full((cam.ny, cam.nx, 4), float("nan"), dtype=dt, device="cuda")
        st = torch.zeros((cam.ny, cam.nx), dtype=torch.uint8, device="cuda")
        polrt.rt_render_static(ctx, form, out, st)
        assert torch.equal(st, st_ref)
        assert torch.equal(out, ref)
        assert polrt.rt_last_counters(ctx)["rays"] == cam.nx * cam.ny


def test_static_counters_report_this_call(rt):
    """After an overlapped rt_render (2^19 rays, 4+ chunks), rt_render_static's counters are its
    own: one chunk, its own kernel times."""
    from paper_2302_02733_gb300 import synth

    polrt, ctx = rt
    big = synth.Camera(incl_deg=60.0, nx=768, ny=768)
    polrt.rt_set_camera(ctx, big)
    polrt.rt_load_model(ctx, polrt.adaf_model(synth.adaf_params(1)))
    img = torch.zeros((768, 768, 4), dtype=torch.float32, device="cuda")
    polrt.rt_render(ctx, polrt.RT_MIXED, img)
    c_big = polrt.rt_last_counters(ctx)
    assert c_big["chunks"] >= 2
    cam = synth.Camera(incl_deg=60.0, nx=32, ny=32)
    polrt.rt_set_camera(ctx, cam)
    out = torch.zeros((32, 32, 4), dtype=torch.float32, device="cuda")
    polrt.rt_render_static(ctx, polrt.RT_MIXED, out)
    c = polrt.rt_last_counters(ctx)
    assert c["chunks"] == 1 and c["rays"] == 32 * 32
    assert c["ms_geodesic"] != c_big["ms_geodesic"] and c["ms_geodesic"] < c_big["ms_geodesic"]


def test_static_refuses_oversize_host_buffers_and_other_forms(rt):
    from paper_2302_02733_gb300 import synth

    polrt, ctx = rt
    assert polrt.rt_render_static_max_pixels() == MAX_PIXELS
    side = int(np.sqrt(MAX_PIXELS)) + 2
    cam = synth.Camera(incl_deg=60.0, nx=side, ny=side)
    polrt.rt_set_camera(ctx, cam)
    polrt.rt_load_model(ctx, polrt.adaf_model(synth.adaf_params(1)))
    out = torch.zeros((side, side, 4), dtype=torch.float64, device="cuda")
    assert polrt.rt_render_static(ctx, polrt.RT_FP64, out, check=False) == polrt.RT_ERR_SIZE
    cam = synth.Camera(incl_deg=60.0, nx=8, ny=8)
    polrt.rt_set_camera(ctx, cam)
    host = torch.zeros((8, 8, 4), dtype=torch.float64)
    assert polrt.rt_render_static(ctx, polrt.RT_FP64, host, check=False) == polrt.RT_ERR_INVALID
    dev = torch.zeros((8, 8, 4), dtype=torch.float32, device="cuda")
    assert polrt.rt_render_static(ctx, polrt.RT_SURROGATE, dev, check=False) == polrt.RT_ERR_INVALID
