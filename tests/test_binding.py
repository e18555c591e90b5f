"""CPU checks of the Python binding's buffer checks. The C calls take bare pointers, and the
binding refuses buffers that are smaller than the call's output, or that hold elements of
another size, before any pointer reaches the library. Without such a check the library would
write past the end of the buffer."""
import numpy as np
import pytest

import __graft_entry__  # noqa: F401  (puts the repo root on sys.path)

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def polrt():
    from paper_2302_02733_gb300 import build, polrt as p

    build.build()
    return p


def cam(polrt, nx, ny):
    from paper_2302_02733_gb300 import synth

    return polrt._camera(synth.Camera(nx=nx, ny=ny))


def test_need(polrt):
    polrt._need(None, 10, 8, "none passes")
    polrt._need(np.zeros(10), 10, 8, "exact")
    polrt._need(torch.zeros(12, dtype=torch.float32), 12, 4, "torch")
    with pytest.raises(ValueError):
        polrt._need(np.zeros(9), 10, 8, "short")
    with pytest.raises(ValueError):
        polrt._need(np.zeros(20, dtype=np.float32), 10, 8, "float32 where float64 is written")


@pytest.mark.parametrize("form,dtype,shape", [
    ("RT_FP64", np.float64, (6, 5, 4)), ("RT_MIXED", np.float32, (6, 5, 4)),
    ("RT_SURROGATE", np.float32, (6, 5, 4)), ("RT_UNPOL", np.float32, (6, 5))])
def test_image_buffers_per_form(polrt, form, dtype, shape):
    f = getattr(polrt, form)
    c = cam(polrt, 5, 6)
    polrt._check_images(None, f, np.zeros(shape, dtype), np.zeros((6, 5), np.uint8), cam=c)
    wrong = np.float32 if dtype == np.float64 else np.float64
    with pytest.raises(ValueError):  # the other precision, even with enough bytes
        polrt._check_images(None, f, np.zeros(shape, wrong), cam=c)
    per_pixel = shape[2] if len(shape) == 3 else 1
    with pytest.raises(ValueError):  # one pixel short
        polrt._check_images(None, f, np.zeros(6 * 5 * per_pixel - per_pixel, dtype), cam=c)
    with pytest.raises(ValueError):
        polrt._check_images(None, f, np.zeros(shape, dtype), np.zeros((6, 4), np.uint8), cam=c)
    if f != polrt.RT_UNPOL:
        esz = np.dtype(dtype).itemsize
        polrt._check_images(None, f, np.zeros(shape, dtype), depth=np.zeros((6, 5, 2), dtype), cam=c)
        with pytest.raises(ValueError):
            polrt._check_images(None, f, np.zeros(shape, dtype), depth=np.zeros((6, 5, 1), dtype), cam=c)
        vis_t = np.complex128 if esz == 8 else np.complex64
        polrt._check_images(None, f, np.zeros(shape, dtype), vis=np.zeros((6, 5), vis_t), cam=c)
        with pytest.raises(ValueError):
            polrt._check_images(None, f, np.zeros(shape, dtype), vis=np.zeros((6, 5), dtype), cam=c)


def test_unknown_form_is_left_to_the_library(polrt):
    polrt._check_images(None, 7, np.zeros(1), cam=cam(polrt, 5, 6))


def test_batch_jobs_are_checked_against_their_own_cameras(polrt):
    from paper_2302_02733_gb300 import synth

    good = polrt.make_jobs([(synth.Camera(nx=8, ny=4), 0.0, 0.0, np.zeros((4, 8, 4), np.float32), None, None),
                            (synth.Camera(nx=3, ny=3), 0.0, 0.0, np.zeros((3, 3, 4), np.float32), None, None)])
    polrt._check_jobs(None, polrt.RT_MIXED, good)
    with pytest.raises(ValueError):  # float32 images for the FP64 form
        polrt._check_jobs(None, polrt.RT_FP64, good)
    short = polrt.make_jobs([(synth.Camera(nx=8, ny=4), 0.0, 0.0, np.zeros((3, 8, 4), np.float32), None, None)])
    with pytest.raises(ValueError):
        polrt.rt_render_batch(None, polrt.RT_MIXED, short)
    with pytest.raises(ValueError):
        polrt.rt_batch_autotune(None, polrt.RT_MIXED, short)


def test_row_buffers(polrt):
    x = np.zeros((10, 4), np.float32)
    with pytest.raises(ValueError):
        polrt.rt_mlp_forward(None, x, np.zeros((9, 8), np.float32))
    with pytest.raises(ValueError):
        polrt.rt_kappa_coeffs(None, np.zeros((10, 6)), np.zeros((10, 8), np.float32))
    with pytest.raises(ValueError):
        polrt.rt_surrogate_coeffs(None, np.zeros((10, 6)), np.zeros((10, 8)), np.zeros(9, np.uint8))
    with pytest.raises(ValueError):
        polrt.rt_mlp_set_params(None, np.zeros(polrt.RT_MLP_PARAMS, np.float64), polrt.mlp_norm([0] * 4, [1] * 4))
    with pytest.raises(ValueError):
        polrt.rt_mlp_train(None, x, np.zeros((10, 8), np.float32), 100, 128, 1e-3, 1, np.zeros(99, np.float32))
    with pytest.raises(ValueError):
        polrt.rt_surrogate_dataset(None, [0.0] * 8, 10, 1, x, np.zeros((10, 8), np.float32), np.zeros(10, np.uint8))


def test_grid_and_workspace(polrt):
    from paper_2302_02733_gb300 import synth

    g = synth.GridParams(n1=4, n2=3, n3=2)
    polrt.grid_model(np.zeros((4, 3, 2, 8), np.float32), g)
    with pytest.raises(ValueError):
        polrt.grid_model(np.zeros((4, 3, 2, 8), np.float64), g)
    with pytest.raises(ValueError):
        polrt.rt_set_workspace(None, np.zeros(100, np.uint8), 101)
