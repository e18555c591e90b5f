"""The grid fetch staged through shared memory by TMA (RT_FETCH_STAGED) against the gathering
fetch (RT_FETCH_GATHER): the same image bit for bit, in one pass (64x48 torus, the seam in phi
crossed by many rays at i = 20 deg) and in the overlapped shape (768x768, 4+ chunks), with the
status codes and the depth maps. Both fetches take the same cells and interpolate them in the
same order; only where the cells come from differs."""
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


@pytest.mark.parametrize("nx,ny", [(64, 48), (768, 768)])
def test_staged_fetch_equals_gather(rt, synth, torus_grid, nx, ny):
    polrt, ctx = rt
    prims, g = torus_grid
    polrt.rt_set_integrator(ctx, 0.05, 20000)
    polrt.rt_set_camera(ctx, synth.Camera(incl_deg=20.0, nx=nx, ny=ny))
    polrt.rt_load_model(ctx, polrt.grid_model(torch.from_numpy(prims).cuda(), g))
    res = {}
    for mode in (polrt.RT_FETCH_GATHER, polrt.RT_FETCH_STAGED):
        polrt.rt_set_grid_fetch(ctx, mode)
        out = torch.full((ny, nx, 4), float("nan"), dtype=torch.float32, device="cuda")
        st = torch.zeros((ny, nx), dtype=torch.uint8, device="cuda")
        dep = torch.full((ny, nx, 2), float("nan"), dtype=torch.float32, device="cuda")
        polrt.rt_render_depths(ctx, polrt.RT_MIXED, out, dep, st)
        c = polrt.rt_last_counters(ctx)
        res[mode] = (out, st, dep, c)
    polrt.rt_set_grid_fetch(ctx, polrt.RT_FETCH_AUTO)
    (a, sa, da, ca), (b, sb, db, cb) = res[polrt.RT_FETCH_GATHER], res[polrt.RT_FETCH_STAGED]
    assert torch.equal(sa, sb) and torch.equal(a, b) and torch.equal(da, db)
    assert ca["emitting_points"] == cb["emitting_points"] > 0
    if nx * ny >= 1 << 19:
        assert cb["chunks"] >= 2
    print(f"{nx}x{ny}: gather {ca['ms_transfer']:.2f} ms, staged {cb['ms_transfer']:.2f} ms (transfer span)")


def test_fetch_mode_argument_checks(rt):
    polrt, ctx = rt
    assert polrt.rt_get_grid_fetch(ctx) == polrt.RT_FETCH_AUTO
    assert polrt.lib().rt_set_grid_fetch(ctx, 3) == polrt.RT_ERR_INVALID
    assert polrt.lib().rt_set_grid_fetch(ctx, -1) == polrt.RT_ERR_INVALID
