"""Thin Python binding of the polrt C ABI (include/polrt.h): argument marshalling only.

Every function keeps the C name. Buffers may be torch tensors (on the GPU or the host) or
numpy arrays; their data pointers are passed through unchanged, once the buffer is known to
hold what the call reads or writes (the C calls take bare pointers; the sizes follow from the
camera or the row count). The CUDA library must have
been built in-tree (``paper_2302_02733_gb300.build.build()``). Without it this module raises:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

RT_OK, RT_ERR_INVALID, RT_ERR_CUDA, RT_ERR_NOMEM, RT_ERR_NOT_READY, RT_ERR_WORKSPACE, RT_ERR_SIZE = 0, -1, -2, -3, -4, -5, -6
RT_ERR_STALL = -7
RT_MODEL_ADAF, RT_MODEL_GRID = 1, 2
RT_FP64, RT_MIXED, RT_SURROGATE, RT_UNPOL = 0, 1, 2, 3
RT_EDF_THERMAL, RT_EDF_KAPPA = 0, 1
RT_RAY_HORIZON, RT_RAY_ESCAPE, RT_RAY_NMAX, RT_RAY_NAN, RT_RAY_OVERFLOW = 1, 2, 3, 4, 5


class rt_adaf_params(C.Structure):
    _fields_ = [("n0", C.c_double), ("T0", C.c_double), ("beta", C.c_double), ("f_kep", C.c_double),
                ("Ti_over_Te", C.c_double), ("r_out", C.c_double)]


class rt_grid_params(C.Structure):
    _fields_ = [("n1", C.c_int), ("n2", C.c_int), ("n3", C.c_int), ("r_in", C.c_double), ("r_out", C.c_double),
                ("hslope", C.c_double), ("poly_xt", C.c_double), ("poly_alpha", C.c_double),
                ("mks_smooth", C.c_double), ("prims", C.c_void_p), ("M_unit", C.c_double), ("R_high", C.c_double),
                ("R_low", C.c_double), ("sigma_cut", C.c_double), ("gamma_ad", C.c_double)]


class rt_model_params(C.Structure):
    _fields_ = [("kind", C.c_int), ("adaf", rt_adaf_params), ("grid", rt_grid_params), ("edf", C.c_int),
                ("kappa", C.c_double)]


class rt_camera(C.Structure):
    _fields_ = [("a", C.c_double), ("incl_deg", C.c_double), ("r_cam", C.c_double), ("freq_hz", C.c_double),
                ("fov_M", C.c_double), ("nx", C.c_int), ("ny", C.c_int), ("M_bh_g", C.c_double),
                ("dist_cm", C.c_double)]


class rt_counters(C.Structure):
    _fields_ = [("rays", C.c_uint64), ("steps", C.c_uint64), ("points", C.c_uint64),
                ("emitting_points", C.c_uint64), ("arena_blocks_used", C.c_uint64),
                ("arena_blocks_total", C.c_uint64), ("n_horizon", C.c_uint32), ("n_escape", C.c_uint32),
                ("n_nmax", C.c_uint32), ("n_nan", C.c_uint32), ("n_overflow", C.c_uint32),
                ("ms_geodesic", C.c_float), ("ms_transfer", C.c_float), ("ms_total", C.c_float),
                ("chunks", C.c_uint32), ("shape", C.c_uint32), ("geodesic_launches", C.c_uint32),
                ("transfer_launches", C.c_uint32)]


class rt_mlp_norm(C.Structure):
    _fields_ = [("lo", C.c_float * 4), ("hi", C.c_float * 4), ("y_mean", C.c_float * 8), ("y_std", C.c_float * 8),
                ("base", (C.c_float * 35) * 8)]


RT_MLP_PARAMS = 9160


class rt_job(C.Structure):
    _fields_ = [("cam", rt_camera), ("M_unit", C.c_double), ("R_high", C.c_double), ("out_iquv", C.c_void_p),
                ("status", C.c_void_p), ("out_depth", C.c_void_p)]


class rt_batch_config(C.Structure):
    _fields_ = [("geo_warps", C.c_int), ("step_tile", C.c_int), ("blocks_per_sm", C.c_int), ("ms", C.c_float),
                ("mode", C.c_int), ("geo_warps_odd", C.c_int)]


RT_BATCH_PERSISTENT, RT_BATCH_CHUNKS = 0, 1
RT_FETCH_AUTO, RT_FETCH_GATHER, RT_FETCH_STAGED = 0, 1, 2


_lib = None
_VP = C.c_void_p


class rt_render_config(C.Structure):
    _fields_ = [("geo_blocks_per_sm", C.c_int), ("xfer_blocks_per_sm", C.c_int), ("chunks", C.c_int),
                ("last_chunk_div", C.c_int)]


def lib():
    """Load libpolrt.so; raises if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"polrt CUDA library missing at {_build.LIB}: run build() first")
        L = C.CDLL(_build.LIB)
        L.rt_create.argtypes = [C.POINTER(_VP), C.c_int, _VP]
        L.rt_destroy.argtypes = [_VP]
        L.rt_set_stream.argtypes = [_VP, _VP]
        L.rt_load_model.argtypes = [_VP, C.POINTER(rt_model_params)]
        L.rt_set_camera.argtypes = [_VP, C.POINTER(rt_camera)]
        L.rt_get_camera.argtypes = [_VP, C.POINTER(rt_camera)]
        L.rt_set_integrator.argtypes = [_VP, C.c_double, C.c_int]
        L.rt_set_workspace.argtypes = [_VP, _VP, C.c_size_t]
        L.rt_workspace_min_bytes.argtypes = []
        L.rt_workspace_min_bytes.restype = C.c_size_t
        L.rt_workspace_hint.argtypes = [_VP, C.POINTER(C.c_size_t)]
        L.rt_render.argtypes = [_VP, C.c_int, _VP, _VP]
        L.rt_image_stats.argtypes = [_VP, _VP, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                     C.POINTER(C.c_double)]
        L.rt_last_counters.argtypes = [_VP, C.POINTER(rt_counters)]
        L.rt_last_timeline.argtypes = [_VP, _VP, C.c_int, C.POINTER(C.c_int)]
        L.rt_render_static.argtypes = [_VP, C.c_int, _VP, _VP]
        L.rt_render_depths.argtypes = [_VP, C.c_int, _VP, _VP, _VP]
        L.rt_kappa_coeffs.argtypes = [_VP, _VP, C.c_longlong, _VP]
        L.rt_mlp_set_params.argtypes = [_VP, _VP, C.POINTER(rt_mlp_norm)]
        L.rt_mlp_get_params.argtypes = [_VP, _VP, C.POINTER(rt_mlp_norm)]
        L.rt_mlp_forward.argtypes = [_VP, _VP, C.c_longlong, _VP]
        L.rt_mlp_grad.argtypes = [_VP, _VP, _VP, C.c_longlong, _VP, C.POINTER(C.c_float)]
        L.rt_mlp_train.argtypes = [_VP, _VP, _VP, C.c_longlong, C.c_int, C.c_int, C.c_float, C.c_uint64, _VP]
        L.rt_surrogate_dataset.argtypes = [_VP, _VP, C.c_longlong, C.c_uint64, _VP, _VP, _VP]
        L.rt_surrogate_coeffs.argtypes = [_VP, _VP, C.c_longlong, _VP, _VP]
        L.rt_render_adaptive.argtypes = [_VP, C.c_int, _VP, _VP, C.c_int, C.c_double, C.POINTER(C.c_longlong)]
        L.rt_image_visibilities.argtypes = [_VP, _VP, C.c_int, C.c_int, _VP]
        L.rt_render_features.argtypes = [_VP, _VP, C.c_longlong, C.POINTER(C.c_longlong)]
        L.rt_surrogate_fit.argtypes = [_VP, _VP, _VP, _VP, C.c_longlong, _VP, C.POINTER(rt_mlp_norm)]
        L.rt_render_batch.argtypes = [_VP, C.c_int, C.POINTER(rt_job), C.c_int]
        L.rt_batch_autotune.argtypes = [_VP, C.c_int, C.POINTER(rt_job), C.c_int, C.POINTER(rt_batch_config)]
        L.rt_set_batch_config.argtypes = [_VP, C.c_int, C.POINTER(rt_batch_config)]
        L.rt_get_batch_config.argtypes = [_VP, C.c_int, C.POINTER(rt_batch_config)]
        L.rt_set_render_config.argtypes = [_VP, C.POINTER(rt_render_config)]
        L.rt_get_render_config.argtypes = [_VP, C.POINTER(rt_render_config)]
        L.rt_set_grid_fetch.argtypes = [_VP, C.c_int]
        L.rt_fp64_fma_peak.argtypes = [C.c_int, C.POINTER(C.c_double)]
        L.rt_get_batch_stats.argtypes = [_VP, C.c_void_p]
        L.rt_get_grid_fetch.argtypes = [_VP, C.POINTER(C.c_int)]
        L.rt_render_static_max_pixels.argtypes = []
        L.rt_render_static_max_pixels.restype = C.c_longlong
        L.rt_error_string.argtypes = [C.c_int]
        L.rt_error_string.restype = C.c_char_p
        _lib = L
    return _lib


class PolrtError(RuntimeError):
    def __init__(self, code: int, call: str):
        super().__init__(f"{call}: {lib().rt_error_string(code).decode()} ({code})")
        self.code = code


def _check(code: int, call: str):
    if code != RT_OK:
        raise PolrtError(code, call)


def _ptr(buf):
    """Data pointer of a torch tensor or numpy array (None -> NULL)."""
    if buf is None:
        return None
    if hasattr(buf, "data_ptr"):
        if not buf.is_contiguous():
            raise ValueError("buffer must be contiguous")
        return buf.data_ptr()
    if isinstance(buf, np.ndarray):
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("buffer must be C-contiguous")
        return buf.ctypes.data
    raise TypeError(f"unsupported buffer type {type(buf)}")


def _bytes_of(buf):
    """(total bytes, bytes per element) of a torch tensor or numpy array."""
    if hasattr(buf, "element_size"):
        return buf.numel() * buf.element_size(), buf.element_size()
    return buf.nbytes, buf.itemsize


def _need(buf, count: int, itemsize: int, what: str):
    """Refuse a buffer (None passes) with elements of another size than itemsize, or fewer
    than count of them: the library would read or write past its end."""
    if buf is None:
        return
    have, isz = _bytes_of(buf)
    if isz != itemsize or have < count * itemsize:
        raise ValueError(f"{what}: needs {count} elements of {itemsize} bytes, has {have // max(isz, 1)} of {isz}")


def _image_layout(form: int):
    """(values per pixel, bytes per value) of an image of this form; None for a form the
    library rejects itself."""
    return {RT_FP64: (4, 8), RT_MIXED: (4, 4), RT_SURROGATE: (4, 4), RT_UNPOL: (1, 4)}.get(form)


def _check_images(ctx, form: int, out, status=None, depth=None, vis=None, cam=None):
    """The image-sized buffers of a call on the current camera (or cam) hold one image."""
    lay = _image_layout(form)
    if lay is None:
        return
    if cam is None:
        cam = rt_camera()
        if lib().rt_get_camera(ctx, C.byref(cam)) != RT_OK:
            return  # no camera yet: the call reports that itself
    npix = cam.nx * cam.ny
    ncomp, esz = lay
    _need(out, npix * ncomp, esz, "image buffer")
    _need(status, npix, 1, "status buffer")
    _need(depth, npix * 2, esz, "depth buffer")
    _need(vis, npix, 2 * esz, "visibility buffer")


def rt_create(device: int = 0, stream=None) -> int:
    h = _VP()
    _check(lib().rt_create(C.byref(h), device, stream), "rt_create")
    return h.value


def rt_destroy(ctx):
    _check(lib().rt_destroy(ctx), "rt_destroy")


def rt_set_stream(ctx, stream):
    _check(lib().rt_set_stream(ctx, stream), "rt_set_stream")


def _camera(cam) -> rt_camera:
    if isinstance(cam, rt_camera):
        return cam
    return rt_camera(cam.a, cam.incl_deg, cam.r_cam, cam.freq_hz, cam.fov_M, cam.nx, cam.ny, cam.M_bh_g, cam.dist_cm)


def rt_set_camera(ctx, cam):
    """cam: an rt_camera, or any object with the same field names (e.g. synth.Camera)."""
    _check(lib().rt_set_camera(ctx, C.byref(_camera(cam))), "rt_set_camera")


def rt_get_camera(ctx) -> rt_camera:
    cam = rt_camera()
    _check(lib().rt_get_camera(ctx, C.byref(cam)), "rt_get_camera")
    return cam


def rt_set_integrator(ctx, eps: float = 0.05, nmax: int = 20000):
    _check(lib().rt_set_integrator(ctx, eps, nmax), "rt_set_integrator")


def rt_load_model(ctx, params: rt_model_params, keepalive=None):
    _check(lib().rt_load_model(ctx, C.byref(params)), "rt_load_model")


def adaf_model(p, kappa: float = 0.0) -> rt_model_params:
    """kappa > 3 selects kappa electrons, else thermal."""
    m = rt_model_params()
    m.kind = RT_MODEL_ADAF
    m.adaf = rt_adaf_params(p.n0, p.T0, p.beta, p.f_kep, p.Ti_over_Te, p.r_out)
    m.edf, m.kappa = (RT_EDF_KAPPA, kappa) if kappa > 3.0 else (RT_EDF_THERMAL, 0.0)
    return m


def grid_model(prims, g, kappa: float = 0.0) -> rt_model_params:
    """prims: float32 [n1][n2][n3][8] (torch tensor on any device, or numpy); kappa > 3 selects
    kappa electrons, else thermal."""
    shape = tuple(prims.shape)
    if len(shape) != 4 or shape[3] != 8:
        raise ValueError("prims must be [n1][n2][n3][8]")
    _need(prims, shape[0] * shape[1] * shape[2] * 8, 4, "prims (float32)")
    m = rt_model_params()
    m.kind = RT_MODEL_GRID
    m.grid = rt_grid_params(shape[0], shape[1], shape[2], g.r_in, g.r_out, g.hslope, g.poly_xt, g.poly_alpha,
                            g.mks_smooth, _ptr(prims), g.M_unit, g.R_high, g.R_low, g.sigma_cut, g.gamma_ad)
    m.edf, m.kappa = (RT_EDF_KAPPA, kappa) if kappa > 3.0 else (RT_EDF_THERMAL, 0.0)
    return m


def rt_set_workspace(ctx, buf, nbytes: int | None = None):
    if buf is None:
        _check(lib().rt_set_workspace(ctx, None, 0), "rt_set_workspace")
        return
    have = _bytes_of(buf)[0]
    if nbytes is None:
        nbytes = have
    elif nbytes > have:
        raise ValueError(f"workspace: {nbytes} bytes declared, buffer holds {have}")
    _check(lib().rt_set_workspace(ctx, _ptr(buf), nbytes), "rt_set_workspace")


def rt_workspace_min_bytes() -> int:
    return lib().rt_workspace_min_bytes()


def rt_workspace_hint(ctx) -> int:
    b = C.c_size_t(0)
    _check(lib().rt_workspace_hint(ctx, C.byref(b)), "rt_workspace_hint")
    return b.value


def rt_render(ctx, form: int, out_iquv, status=None, check: bool = True) -> int:
    _check_images(ctx, form, out_iquv, status)
    rc = lib().rt_render(ctx, form, _ptr(out_iquv), _ptr(status))
    if check:
        _check(rc, "rt_render")
    return rc


def rt_render_depths(ctx, form: int, out_iquv, out_depth, status=None, check: bool = True) -> int:
    """rt_render plus the per-pixel optical and Faraday depths [ny][nx][2]."""
    _check_images(ctx, form, out_iquv, status, out_depth)
    rc = lib().rt_render_depths(ctx, form, _ptr(out_iquv), _ptr(status), _ptr(out_depth))
    if check:
        _check(rc, "rt_render_depths")
    return rc


def rt_kappa_coeffs(ctx, inp, out):
    """inp: [n, 6] float64 (ne, Theta_e, B, nu, theta_B, kappa); out: [n, 8] float64."""
    n = int(inp.shape[0])
    _need(inp, 6 * n, 8, "inp")
    _need(out, 8 * n, 8, "out")
    _check(lib().rt_kappa_coeffs(ctx, _ptr(inp), int(inp.shape[0]), _ptr(out)), "rt_kappa_coeffs")


def mlp_norm(lo, hi, y_mean=None, y_std=None) -> rt_mlp_norm:
    n = rt_mlp_norm()
    for j in range(4):
        n.lo[j], n.hi[j] = float(lo[j]), float(hi[j])
    for k in range(8):
        n.y_mean[k] = 0.0 if y_mean is None else float(y_mean[k])
        n.y_std[k] = 1.0 if y_std is None else float(y_std[k])
    return n


def rt_mlp_set_params(ctx, theta, norm: rt_mlp_norm):
    _need(theta, RT_MLP_PARAMS, 4, "theta")
    _check(lib().rt_mlp_set_params(ctx, _ptr(theta), C.byref(norm)), "rt_mlp_set_params")


def rt_mlp_get_params(ctx, theta=None) -> rt_mlp_norm:
    n = rt_mlp_norm()
    _need(theta, RT_MLP_PARAMS, 4, "theta")
    _check(lib().rt_mlp_get_params(ctx, _ptr(theta), C.byref(n)), "rt_mlp_get_params")
    return n


def rt_mlp_forward(ctx, x, y):
    n = int(x.shape[0])
    _need(x, 4 * n, 4, "x")
    _need(y, 8 * n, 4, "y")
    _check(lib().rt_mlp_forward(ctx, _ptr(x), int(x.shape[0]), _ptr(y)), "rt_mlp_forward")


def rt_mlp_grad(ctx, x, t, grad) -> float:
    n = int(x.shape[0])
    _need(x, 4 * n, 4, "x")
    _need(t, 8 * n, 4, "t")
    _need(grad, RT_MLP_PARAMS, 4, "grad")
    loss = C.c_float(0)
    _check(lib().rt_mlp_grad(ctx, _ptr(x), _ptr(t), int(x.shape[0]), _ptr(grad), C.byref(loss)), "rt_mlp_grad")
    return loss.value


def rt_mlp_train(ctx, x, t, steps: int, batch: int, lr: float, seed: int, loss_curve=None):
    n = int(x.shape[0])
    _need(x, 4 * n, 4, "x")
    _need(t, 8 * n, 4, "t")
    _need(loss_curve, steps, 4, "loss_curve")
    _check(lib().rt_mlp_train(ctx, _ptr(x), _ptr(t), int(x.shape[0]), steps, batch, lr, seed, _ptr(loss_curve)),
           "rt_mlp_train")


def rt_surrogate_dataset(ctx, box, n: int, seed: int, x, y, valid):
    _need(x, 4 * n, 4, "x")
    _need(y, 8 * n, 4, "y")
    _need(valid, n, 4, "valid (int32)")
    b = (C.c_float * 8)(*[float(v) for v in box])
    _check(lib().rt_surrogate_dataset(ctx, b, n, seed, _ptr(x), _ptr(y), _ptr(valid)), "rt_surrogate_dataset")


def rt_surrogate_fit(ctx, x, y, valid, t, lo, hi) -> rt_mlp_norm:
    n = int(x.shape[0])
    _need(x, 4 * n, 4, "x")
    _need(y, 8 * n, 4, "y")
    _need(valid, n, 4, "valid (int32)")
    _need(t, 8 * n, 4, "t")
    """Baseline fit and standardised residual targets; returns the filled rt_mlp_norm."""
    n = mlp_norm(lo, hi)
    _check(lib().rt_surrogate_fit(ctx, _ptr(x), _ptr(y), _ptr(valid), int(x.shape[0]), _ptr(t), C.byref(n)),
           "rt_surrogate_fit")
    return n


def rt_render_adaptive(ctx, form: int, out, status=None, base_step: int = 8, tol: float = 1e-3,
                       check: bool = True) -> int:
    """Adaptive render into device buffers; returns the number of rays traced (with check=False,
    the return code; the rays traced are then rt_last_counters' "rays")."""
    _check_images(ctx, form, out, status)
    n = C.c_longlong(0)
    rc = lib().rt_render_adaptive(ctx, form, _ptr(out), _ptr(status), base_step, tol, C.byref(n))
    if not check:
        return rc
    _check(rc, "rt_render_adaptive")
    return n.value


def rt_image_visibilities(ctx, img, form: int, stokes: int, vis):
    """vis: complex buffer [ny][nx] (complex128 for RT_FP64, complex64 otherwise)."""
    _check_images(ctx, form, img, vis=vis)
    _check(lib().rt_image_visibilities(ctx, _ptr(img), form, stokes, _ptr(vis)), "rt_image_visibilities")


def rt_render_features(ctx, feat) -> int:
    """feat: device float32 [cap, 4]; returns the number of emitting points."""
    _need(feat, 4 * int(feat.shape[0]), 4, "feat")
    n = C.c_longlong(0)
    _check(lib().rt_render_features(ctx, _ptr(feat), int(feat.shape[0]), C.byref(n)), "rt_render_features")
    return n.value


def rt_surrogate_coeffs(ctx, inp, out, inside=None):
    n = int(inp.shape[0])
    _need(inp, 6 * n, 8, "inp")
    _need(out, 8 * n, 8, "out")
    _need(inside, n, 1, "inside")
    _check(lib().rt_surrogate_coeffs(ctx, _ptr(inp), int(inp.shape[0]), _ptr(out), _ptr(inside)),
           "rt_surrogate_coeffs")


def make_jobs(items) -> C.Array:
    """items: iterable of (camera, M_unit, R_high, out_iquv, status, out_depth); camera as for
    rt_set_camera, buffers device tensors (status and out_depth may be None)."""
    items = list(items)
    arr = (rt_job * len(items))()
    arr._buffers = [it[3:] for it in items]  # kept alive with the pointers; sizes checked per form
    for j, (cam, mu, rh, out, st, dep) in zip(arr, items):
        j.cam = _camera(cam)
        j.M_unit = mu
        j.R_high = rh
        j.out_iquv = _ptr(out)
        j.status = _ptr(st)
        j.out_depth = _ptr(dep)
    return arr


def _check_jobs(ctx, form: int, jobs):
    """Every job's buffers (recorded by make_jobs) hold one image of its camera."""
    for j, (out, st, dep) in zip(jobs, getattr(jobs, "_buffers", ())):
        _check_images(ctx, form, out, st, dep, cam=j.cam)


def rt_render_batch(ctx, form: int, jobs, check: bool = True) -> int:
    """Render every job of an rt_job array (see make_jobs) in one persistent launch."""
    _check_jobs(ctx, form, jobs)
    rc = lib().rt_render_batch(ctx, form, jobs, len(jobs))
    if check:
        _check(rc, "rt_render_batch")
    return rc


def rt_batch_autotune(ctx, form: int, jobs) -> dict:
    _check_jobs(ctx, form, jobs)
    b = rt_batch_config()
    _check(lib().rt_batch_autotune(ctx, form, jobs, len(jobs), C.byref(b)), "rt_batch_autotune")
    return {k: getattr(b, k) for k, _ in rt_batch_config._fields_}


class rt_batch_stats(C.Structure):
    _fields_ = [(k, C.c_uint64) for k in ("geo_iters", "geo_sleeps", "xfer_iters", "xfer_sleeps", "ticket_polls",
                                          "ready_polls", "free_spins", "tickets")]


def rt_get_batch_stats(ctx) -> dict:
    """Flow statistics of the last persistent (mode 0) batch."""
    st = rt_batch_stats()
    _check(lib().rt_get_batch_stats(ctx, C.byref(st)), "rt_get_batch_stats")
    return {k: getattr(st, k) for k, _ in rt_batch_stats._fields_}


def rt_set_batch_config(ctx, form: int, geo_warps: int, step_tile: int, blocks_per_sm: int, mode: int = 0,
                        geo_warps_odd: int = 0):
    b = rt_batch_config(geo_warps, step_tile, blocks_per_sm, 0.0, mode, geo_warps_odd)
    _check(lib().rt_set_batch_config(ctx, form, C.byref(b)), "rt_set_batch_config")


def rt_get_batch_config(ctx, form: int) -> dict:
    b = rt_batch_config()
    _check(lib().rt_get_batch_config(ctx, form, C.byref(b)), "rt_get_batch_config")
    return {k: getattr(b, k) for k, _ in rt_batch_config._fields_}


def rt_fp64_fma_peak(device: int = 0) -> float:
    """Measured FP64 FMA rate of the device in TFLOP/s."""
    v = C.c_double(0.0)
    _check(lib().rt_fp64_fma_peak(device, C.byref(v)), "rt_fp64_fma_peak")
    return v.value


def rt_set_grid_fetch(ctx, mode: int):
    """RT_FETCH_AUTO, RT_FETCH_GATHER or RT_FETCH_STAGED (TMA-staged stencils)."""
    _check(lib().rt_set_grid_fetch(ctx, mode), "rt_set_grid_fetch")


def rt_get_grid_fetch(ctx) -> int:
    m = C.c_int(0)
    _check(lib().rt_get_grid_fetch(ctx, C.byref(m)), "rt_get_grid_fetch")
    return m.value


def rt_set_render_config(ctx, geo_blocks_per_sm: int = 0, xfer_blocks_per_sm: int = 0, chunks: int = 0,
                         last_chunk_div: int = 0):
    cfg = rt_render_config(geo_blocks_per_sm, xfer_blocks_per_sm, chunks, last_chunk_div)
    _check(lib().rt_set_render_config(ctx, C.byref(cfg)), "rt_set_render_config")


def rt_get_render_config(ctx) -> dict:
    cfg = rt_render_config()
    _check(lib().rt_get_render_config(ctx, C.byref(cfg)), "rt_get_render_config")
    return {k: getattr(cfg, k) for k, _ in rt_render_config._fields_}


def rt_render_static(ctx, form: int, out_iquv, status=None, check: bool = True) -> int:
    """rt_render with the scratch in the library's static device array (no allocation)."""
    _check_images(ctx, form, out_iquv, status)
    rc = lib().rt_render_static(ctx, form, _ptr(out_iquv), _ptr(status))
    if check:
        _check(rc, "rt_render_static")
    return rc


def rt_render_static_max_pixels() -> int:
    return lib().rt_render_static_max_pixels()


def rt_image_stats(ctx, iquv, form: int):
    _check_images(ctx, form, iquv)
    f, lp, cp = C.c_double(0), C.c_double(0), C.c_double(0)
    _check(lib().rt_image_stats(ctx, _ptr(iquv), form, C.byref(f), C.byref(lp), C.byref(cp)), "rt_image_stats")
    return f.value, lp.value, cp.value


def rt_last_counters(ctx) -> dict:
    c = rt_counters()
    _check(lib().rt_last_counters(ctx, C.byref(c)), "rt_last_counters")
    return {k: getattr(c, k) for k, _ in rt_counters._fields_}


def rt_last_timeline(ctx, cap: int = 256) -> list:
    """Per chunk of the last overlapped render: (geodesic start, geodesic end, transfer start,
    transfer end) in ms from the first geodesic start; [] when it was not overlapped."""
    buf = (C.c_float * (4 * cap))()
    n = C.c_int(0)
    _check(lib().rt_last_timeline(ctx, buf, cap, C.byref(n)), "rt_last_timeline")
    return [tuple(buf[4 * k:4 * k + 4]) for k in range(min(n.value, cap))]


def rt_error_string(code: int) -> str:
    return lib().rt_error_string(code).decode()
