"""Visibilities on the GPU (cuFFT plus the phase and centring kernels) against the oracle's
direct sums of the same image: FP64 within 1e-12 of max |V|, float within 1e-5; host and
device buffers; every Stokes plane; a non-square image and the I-only layout."""
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


@pytest.mark.parametrize("nx,ny", [(64, 64), (48, 32)])
def test_visibilities_match_direct_sums(rt, ora, synth, nx, ny):
    polrt, ctx = rt
    cam = synth.Camera(incl_deg=60.0, nx=nx, ny=ny)
    polrt.rt_set_camera(ctx, cam)
    polrt.rt_load_model(ctx, polrt.adaf_model(synth.adaf_params(1)))
    ocam = ora.camera(cam)
    for form, dt, ct, tol in ((polrt.RT_FP64, torch.float64, torch.complex128, 1e-12),
                              (polrt.RT_MIXED, torch.float32, torch.complex64, 1e-5)):
        img = torch.zeros((ny, nx, 4), dtype=dt, device="cuda")
        polrt.rt_render(ctx, form, img)
        h = img.double().cpu().numpy()
        for stokes in range(4):
            vis = torch.zeros((ny, nx), dtype=ct, device="cuda")
            polrt.rt_image_visibilities(ctx, img, form, stokes, vis)
            ref = ora.visibilities(ocam, h[..., stokes])
            err = np.abs(vis.cpu().numpy() - ref).max() / np.abs(ref).max()
            assert err <= tol, (form, stokes, err)
        # host buffers
        vh = np.zeros((ny, nx), dtype=np.complex128 if form == polrt.RT_FP64 else np.complex64)
        polrt.rt_image_visibilities(ctx, img.cpu().numpy(), form, 0, vh)
        ref = ora.visibilities(ocam, h[..., 0])
        assert np.abs(vh - ref).max() / np.abs(ref).max() <= tol
        flux = polrt.rt_image_stats(ctx, img, form)[0]
        assert abs(ref[ny // 2, nx // 2].real / flux - 1) < 10 * tol
    # the I-only layout
    i1 = torch.zeros((ny, nx), dtype=torch.float32, device="cuda")
    polrt.rt_render(ctx, polrt.RT_UNPOL, i1)
    vis = torch.zeros((ny, nx), dtype=torch.complex64, device="cuda")
    polrt.rt_image_visibilities(ctx, i1, polrt.RT_UNPOL, 0, vis)
    ref = ora.visibilities(ocam, i1.double().cpu().numpy())
    assert np.abs(vis.cpu().numpy() - ref).max() / np.abs(ref).max() <= 1e-5
