"""ctypes front-end of the plain FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package. The CUDA library never does. ``build()`` compiles ``oracle.c`` and
``kappa.c`` with
gcc, OpenMP and FP contraction off, so the results do not depend on the host's FMA units.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

HORIZON, ESCAPE, NMAX, NAN = 1, 2, 3, 4
MODEL_ADAF, MODEL_GRID, MODEL_SPHERE = 1, 2, 3


def build(force: bool = False) -> str:
    srcs = [os.path.join(_HERE, f) for f in ("oracle.c", "kappa.c")]
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            [os.path.getmtime(f) for f in srcs] + [os.path.getmtime(os.path.join(_HERE, "oracle.h"))]):
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
                               "-fopenmp", "-fPIC", "-shared", "-o", _SO] + srcs + ["-lm"])
    return _SO


class Camera(C.Structure):
    _fields_ = [("a", C.c_double), ("incl_deg", C.c_double), ("r_cam", C.c_double),
                ("freq_hz", C.c_double), ("fov_M", C.c_double), ("nx", C.c_int), ("ny", C.c_int),
                ("M_bh_g", C.c_double), ("dist_cm", C.c_double), ("eps", C.c_double),
                ("nmax", C.c_int)]


class Model(C.Structure):
    _fields_ = [("kind", C.c_int),
                ("n0", C.c_double), ("T0", C.c_double), ("beta", C.c_double), ("f_kep", C.c_double),
                ("Ti_over_Te", C.c_double), ("r_out_emit", C.c_double),
                ("n1", C.c_int), ("n2", C.c_int), ("n3", C.c_int),
                ("r_in", C.c_double), ("r_out", C.c_double), ("hslope", C.c_double),
                ("poly_xt", C.c_double), ("poly_alpha", C.c_double), ("mks_smooth", C.c_double),
                ("prims", C.POINTER(C.c_float)),
                ("M_unit", C.c_double), ("R_high", C.c_double), ("R_low", C.c_double),
                ("sigma_cut", C.c_double), ("gamma_ad", C.c_double),
                ("edf", C.c_int), ("kappa", C.c_double), ("unpol_test", C.c_int),
                ("sph_R", C.c_double), ("sph_ne", C.c_double), ("sph_Te", C.c_double), ("sph_B", C.c_double),
                ("sph_smooth", C.c_int)]


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        L.ora_metric_ks.argtypes = [C.c_double, C.c_double, C.c_double, _D]
        L.ora_invert4.argtypes = [_D, _D]
        L.ora_metric_derivs.argtypes = [C.c_double, C.c_double, C.c_double, _D, _D]
        L.ora_connection.argtypes = [C.c_double, C.c_double, C.c_double, _D]
        L.ora_camera_ray.argtypes = [C.POINTER(Camera), C.c_double, C.c_double, _D, _D]
        L.ora_trace_geodesic.argtypes = [C.POINTER(Camera), C.c_double, C.c_double, C.c_int, _D, _I]
        L.ora_trace_geodesic.restype = C.c_int
        L.ora_transport_vector.argtypes = [C.c_double, _D, C.c_int, _D, _D]
        L.ora_camera_stokes.argtypes = [C.POINTER(Camera), C.c_double, C.c_double, _D, _D, _D]
        L.ora_fmks_theta.argtypes = [C.POINTER(Model), C.c_double, C.c_double, _D, _D]
        L.ora_fmks_theta.restype = C.c_double
        L.ora_fmks_x2.argtypes = [C.POINTER(Model), C.c_double, C.c_double]
        L.ora_fmks_x2.restype = C.c_double
        L.ora_grid_interp.argtypes = [C.POINTER(Model), C.c_double, C.c_double, C.c_double, _D]
        L.ora_plasma.argtypes = [C.POINTER(Camera), C.POINTER(Model), _D, _D]
        L.ora_fluid_tetrad.argtypes = [C.c_double, _D, _D, _D, _D, _D]
        L.ora_fluid_tetrad.restype = C.c_double
        L.ora_bessel_k_scaled.argtypes = [C.c_int, C.c_double]
        L.ora_bessel_k_scaled.restype = C.c_double
        L.ora_thermal_coeffs.argtypes = [C.c_double] * 5 + [_D]
        L.ora_substep.argtypes = [_D, C.c_double, _D, _D]
        L.ora_synch_kernels.argtypes = [C.c_double, _D]
        L.ora_kappa_coeffs.argtypes = [C.c_double] * 6 + [_D]
        L.ora_render_pixels.argtypes = [C.POINTER(Camera), C.POINTER(Model), C.c_int, _I, _I, C.c_int,
                                        _D, _I, _I, _D, _D, C.c_int]
        L.ora_render_pixels.restype = C.c_int
        L.ora_render_unpol.argtypes = [C.POINTER(Camera), C.POINTER(Model), C.c_int, _I, _I, _D, C.c_int]
        L.ora_render_unpol.restype = C.c_int
        L.ora_image_stats.argtypes = [C.POINTER(Camera), _D, C.c_long, _D, _D, _D]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _ip(a: np.ndarray):
    return a.ctypes.data_as(_I)


def camera(cam, eps: float = 0.05, nmax: int = 20000) -> Camera:
    """Oracle camera from a ``synth.Camera`` (or any object with the same fields)."""
    return Camera(cam.a, cam.incl_deg, cam.r_cam, cam.freq_hz, cam.fov_M, cam.nx, cam.ny,
                  cam.M_bh_g, cam.dist_cm, eps, nmax)


class ModelHandle:
    """Keeps the primitive array alive for as long as the ctypes struct points at it."""

    def __init__(self, st: Model, keep=None):
        self.st = st
        self.keep = keep


EDF_THERMAL, EDF_KAPPA = 0, 1


def adaf_model(p, kappa: float = 0.0) -> ModelHandle:
    """kappa > 3 selects kappa electrons (coefficients by quadrature), else thermal."""
    m = Model()
    m.kind = MODEL_ADAF
    m.n0, m.T0, m.beta, m.f_kep, m.Ti_over_Te, m.r_out_emit = p.n0, p.T0, p.beta, p.f_kep, p.Ti_over_Te, p.r_out
    m.edf, m.kappa = (EDF_KAPPA, kappa) if kappa > 3.0 else (EDF_THERMAL, 0.0)
    return ModelHandle(m)


def grid_model(prims: np.ndarray, g, kappa: float = 0.0) -> ModelHandle:
    prims = np.ascontiguousarray(prims, dtype=np.float32)
    m = Model()
    m.kind = MODEL_GRID
    m.n1, m.n2, m.n3 = prims.shape[0], prims.shape[1], prims.shape[2]
    m.r_in, m.r_out, m.hslope, m.poly_xt = g.r_in, g.r_out, g.hslope, g.poly_xt
    m.poly_alpha, m.mks_smooth = g.poly_alpha, g.mks_smooth
    m.prims = prims.ctypes.data_as(C.POINTER(C.c_float))
    m.M_unit, m.R_high, m.R_low, m.sigma_cut, m.gamma_ad = g.M_unit, g.R_high, g.R_low, g.sigma_cut, g.gamma_ad
    m.edf, m.kappa = (EDF_KAPPA, kappa) if kappa > 3.0 else (EDF_THERMAL, 0.0)
    return ModelHandle(m, prims)


def sphere_model(R: float, ne: float, Te: float, B: float, smooth: bool = False) -> ModelHandle:
    """A static sphere (Theta_e and B [G] constant for r < R; n_e [cm^-3] constant, or with
    smooth=True ne (1 - r^2/R^2)^2; fluid at rest, field along d_phi): a test model whose image
    has a closed form, not a model of the paper."""
    m = Model()
    m.kind = MODEL_SPHERE
    m.sph_R, m.sph_ne, m.sph_Te, m.sph_B, m.sph_smooth = R, ne, Te, B, int(smooth)
    return ModelHandle(m)


def render_pixels(cam: Camera, model: ModelHandle, ix, iy, pert: int = 0, nthreads: int = 0,
                  depth: bool = False):
    """Render the listed pixels; returns (iquv[n,4], nsteps[n], status[n], minpol[n]), and
    with depth=True also depth[n,2] = (tau = sum alpha_I ds, phi = sum rho_V ds)."""
    L = lib()
    ix = np.ascontiguousarray(ix, dtype=np.int32)
    iy = np.ascontiguousarray(iy, dtype=np.int32)
    n = ix.size
    out = np.zeros((n, 4))
    ns = np.zeros(n, dtype=np.int32)
    stt = np.zeros(n, dtype=np.int32)
    mp = np.zeros(n)
    dep = np.zeros((n, 2))
    rc = L.ora_render_pixels(C.byref(cam), C.byref(model.st), n, _ip(ix), _ip(iy), pert, _dp(out), _ip(ns),
                             _ip(stt), _dp(mp), _dp(dep) if depth else None, nthreads)
    if rc != 0:
        raise MemoryError("oracle render failed")
    if depth:
        return out, ns, stt, mp, dep
    return out, ns, stt, mp


def render_image(cam: Camera, model: ModelHandle, pert: int = 0, nthreads: int = 0, depth: bool = False):
    """Full image, row-major [ny][nx][4] (and [ny][nx][2] depths with depth=True)."""
    iy, ix = np.meshgrid(np.arange(cam.ny), np.arange(cam.nx), indexing="ij")
    r = render_pixels(cam, model, ix.ravel(), iy.ravel(), pert, nthreads, depth)
    out = (r[0].reshape(cam.ny, cam.nx, 4), r[1].reshape(cam.ny, cam.nx), r[2].reshape(cam.ny, cam.nx),
           r[3].reshape(cam.ny, cam.nx))
    if depth:
        out = out + (r[4].reshape(cam.ny, cam.nx, 2),)
    return out


def render_unpol(cam: Camera, model: ModelHandle, nthreads: int = 0):
    """Stokes I image [ny][nx] of the unpolarized transfer (j_I and a_I only)."""
    iy, ix = np.meshgrid(np.arange(cam.ny), np.arange(cam.nx), indexing="ij")
    ix = np.ascontiguousarray(ix.ravel(), dtype=np.int32)
    iy = np.ascontiguousarray(iy.ravel(), dtype=np.int32)
    out = np.zeros(ix.size)
    if lib().ora_render_unpol(C.byref(cam), C.byref(model.st), ix.size, _ip(ix), _ip(iy), _dp(out), nthreads) != 0:
        raise MemoryError("oracle render failed")
    return out.reshape(cam.ny, cam.nx)


def visibilities(cam: Camera, plane: np.ndarray) -> np.ndarray:
    """V(u, v) = sum over pixels of S dOmega exp(-2 pi i (u x + v y)) [Jy] written out: x, y the
    pixel-centre angles from the image centre, u = k / FOV and v = l / FOV with
    k = -nx/2 .. nx/2 - 1 (rows l likewise); the double sum taken as the two matrix products
    of the separable exponential. plane: [ny][nx] intensities (cgs)."""
    L = 6.67430e-8 * cam.M_bh_g / 2.99792458e10 ** 2
    dx = cam.fov_M * L / (cam.nx * cam.dist_cm)  # pixel angle [rad]
    dy = dx
    x = (np.arange(cam.nx) + 0.5 - cam.nx / 2) * dx
    y = (np.arange(cam.ny) + 0.5 - cam.ny / 2) * dy
    u = (np.arange(cam.nx) - cam.nx // 2) / (cam.nx * dx)
    v = (np.arange(cam.ny) - cam.ny // 2) / (cam.ny * dy)
    Ex = np.exp(-2j * np.pi * np.outer(u, x))  # [k][i]
    Ey = np.exp(-2j * np.pi * np.outer(v, y))  # [l][j]
    return Ey @ (np.asarray(plane, dtype=np.float64) * dx * dy * 1e23) @ Ex.T


def trace_geodesic(cam: Camera, px: float, py: float):
    L = lib()
    maxst = cam.nmax + 2
    st = np.zeros((maxst, 9))
    stat = C.c_int(0)
    n = L.ora_trace_geodesic(C.byref(cam), px, py, maxst, _dp(st), C.byref(stat))
    return st[: n + 1].copy(), stat.value


def transport_vector(a, states, f):
    """The vector f at the last saved state carried back along the path to every state, as
    the transfer carries each index of the coherency tensor; rows follow the states."""
    st = np.ascontiguousarray(states, dtype=np.float64)
    M = st.shape[0] - 1
    fv = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros((M + 1, 4))
    lib().ora_transport_vector(a, _dp(st), M, _dp(fv), _dp(out))
    return out


def camera_stokes(cam: Camera, px, py, N):
    """(I, Q, U, V) that the transfer's camera reads from the coherency tensor N (4 x 4,
    real or complex) for the pixel at image coordinates (px, py)."""
    N = np.asarray(N, dtype=np.complex128)
    re, im = np.ascontiguousarray(N.real), np.ascontiguousarray(N.imag)
    S = np.zeros(4)
    lib().ora_camera_stokes(C.byref(cam), px, py, _dp(re), _dp(im), _dp(S))
    return S


def metric(a, r, th):
    g = np.zeros(16)
    lib().ora_metric_ks(a, r, th, _dp(g))
    return g.reshape(4, 4)


def metric_derivs(a, r, th):
    dr, dt = np.zeros(16), np.zeros(16)
    lib().ora_metric_derivs(a, r, th, _dp(dr), _dp(dt))
    return dr.reshape(4, 4), dt.reshape(4, 4)


def connection(a, r, th):
    G = np.zeros(64)
    lib().ora_connection(a, r, th, _dp(G))
    return G.reshape(4, 4, 4)


def camera_ray(cam: Camera, px, py):
    x, K = np.zeros(4), np.zeros(4)
    lib().ora_camera_ray(C.byref(cam), px, py, _dp(x), _dp(K))
    return x, K


def plasma(cam: Camera, model: ModelHandle, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(12)
    lib().ora_plasma(C.byref(cam), C.byref(model.st), _dp(x), _dp(out))
    return out


def fluid_tetrad(a, x, K, u, b):
    e = np.zeros(16)
    f = lambda v: np.ascontiguousarray(v, dtype=np.float64)
    x, K, u, b = f(x), f(K), f(u), f(b)
    thB = lib().ora_fluid_tetrad(a, _dp(x), _dp(K), _dp(u), _dp(b), _dp(e))
    return e.reshape(4, 4), thB


def fmks_theta(model: ModelHandle, X1, X2):
    d1, d2 = C.c_double(0), C.c_double(0)
    th = lib().ora_fmks_theta(C.byref(model.st), X1, X2, C.byref(d1), C.byref(d2))
    return th, d1.value, d2.value


def fmks_x2(model: ModelHandle, X1, th):
    return lib().ora_fmks_x2(C.byref(model.st), X1, th)


def grid_interp(model: ModelHandle, X1, X2, X3):
    out = np.zeros(8)
    lib().ora_grid_interp(C.byref(model.st), X1, X2, X3, _dp(out))
    return out


def bessel_k_scaled(n, z):
    return lib().ora_bessel_k_scaled(n, z)


def thermal_coeffs(ne, Te, B, nu, thB):
    out = np.zeros(8)
    lib().ora_thermal_coeffs(ne, Te, B, nu, thB, _dp(out))
    return out


def synch_kernels(x):
    """(F, G, H)(x): x int_x^inf K_5/3, x K_2/3(x), x K_1/3(x) + int_x^inf K_1/3."""
    out = np.zeros(3)
    lib().ora_synch_kernels(x, _dp(out))
    return out


def kappa_coeffs(ne, Te, B, nu, thB, kappa):
    """Coefficients (jI jQ jV aI aQ aV rQ rV) by quadrature over a kappa distribution
    (kappa > 3) or, for kappa <= 0, the Maxwell-Juttner distribution."""
    out = np.zeros(8)
    lib().ora_kappa_coeffs(ne, Te, B, nu, thB, kappa, _dp(out))
    return out


def substep(coef11, ds, S0):
    cf = np.ascontiguousarray(coef11, dtype=np.float64)
    s0 = np.ascontiguousarray(S0, dtype=np.float64)
    s1 = np.zeros(4)
    lib().ora_substep(_dp(cf), ds, _dp(s0), _dp(s1))
    return s1


def image_stats(cam: Camera, iquv: np.ndarray):
    iquv = np.ascontiguousarray(iquv, dtype=np.float64)
    f, lp, cp = C.c_double(0), C.c_double(0), C.c_double(0)
    lib().ora_image_stats(C.byref(cam), _dp(iquv), iquv.size // 4, C.byref(f), C.byref(lp), C.byref(cp))
    return f.value, lp.value, cp.value
