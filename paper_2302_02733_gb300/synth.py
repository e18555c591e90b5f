"""Seeded synthetic inputs for the ray tracer: plasma models, camera set-ups and job tables.

This module is the one place that draws random numbers. It builds *inputs* only:

* the semi-analytic ADAF parameter draw (density and temperature normalisations),
* a Fishbone-Moncrief torus sampled on a funky-modified-Kerr-Schild (FMKS) grid with
  log-normal density and field perturbations, standing in for the GRMHD snapshot of the
  paper's Section 3 (one time slice on arrays of about 200^3 cells, Section 2.1),
* the camera/workload descriptions and the batched image-library job table.

It contains none of the ray-tracing method: no geodesic, transport, emissivity or transfer
arithmetic. The CUDA library and the CPU oracle both consume what it returns and share
nothing else.

Random numbers come from a counter-based splitmix64 stream (Steele, Lea & Flood 2014): the
value for (seed, counter) is the splitmix64 finaliser applied to
``seed + (counter + 1) * 0x9E3779B97F4A7C15`` (mod 2^64). Uniforms in (0, 1) take the top
53 bits plus one half ulp; Gaussians use Box-Muller on two consecutive counters.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counter) -> np.ndarray:
    """Counter-based splitmix64: one 64-bit value per counter (array-valued)."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, counter) -> np.ndarray:
    """Uniform doubles in the open interval (0, 1)."""
    z = splitmix64(seed, counter) >> np.uint64(11)
    return (z.astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def gauss(seed: int, counter) -> np.ndarray:
    """Standard normal deviates; deviate n uses counters 2n and 2n+1 (Box-Muller)."""
    c = np.asarray(counter, dtype=np.uint64)
    u1 = uniform(seed, c * np.uint64(2))
    u2 = uniform(seed, c * np.uint64(2) + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


# ----------------------------------------------------------------------------------------
# Semi-analytic ADAF (the "semianalytic model" of Sections 2.1 and 3)
# ----------------------------------------------------------------------------------------
@dataclass
class AdafParams:
    a: float = 0.9375          # black-hole spin
    n0: float = 3.0e7          # electron density normalisation [cm^-3]: n_e = n0 r^-3/2
    T0: float = 1.0e12         # electron temperature normalisation [K]: T_e = T0 / r
    beta: float = 10.0         # plasma beta, B^2/8pi = P_gas / beta
    f_kep: float = 0.5         # sub-Keplerian factor on the specific angular momentum
    Ti_over_Te: float = 3.0    # ion-to-electron temperature ratio in P_gas
    r_out: float = 1000.0      # emission only inside this radius [M]


def adaf_params(seed: int = 1, a: float = 0.9375) -> AdafParams:
    """Seeded ADAF draw: log10 n0 ~ U(7, 8) [cm^-3], log10 T0 ~ U(11.5, 12.5) [K]."""
    u = uniform(seed, [0, 1])
    return AdafParams(a=a, n0=10.0 ** (7.0 + u[0]), T0=10.0 ** (11.5 + u[1]))


# ----------------------------------------------------------------------------------------
# FMKS grid description + Fishbone-Moncrief torus (GRMHD-shaped snapshot)
# ----------------------------------------------------------------------------------------
@dataclass
class GridParams:
    a: float = 0.9375
    n1: int = 288
    n2: int = 128
    n3: int = 128
    r_in: float = 0.0          # filled as 0.8 r_h when 0
    r_out: float = 1000.0
    hslope: float = 0.3
    poly_xt: float = 0.82
    poly_alpha: float = 14.0
    mks_smooth: float = 0.5
    M_unit: float = 1.0e19     # mass unit [g]
    R_high: float = 40.0
    R_low: float = 1.0
    sigma_cut: float = 1.0
    gamma_ad: float = 13.0 / 9.0

    def resolved(self) -> "GridParams":
        g = GridParams(**asdict(self))
        if g.r_in <= 0.0:
            g.r_in = 0.8 * (1.0 + math.sqrt(1.0 - g.a * g.a))
        return g


def _fmks_theta(x1, x2, g: GridParams):
    """FMKS polar angle theta(X1, X2) and its partial derivatives (input-side copy)."""
    x1in = math.log(g.r_in)
    th_g = np.pi * x2 + 0.5 * (1.0 - g.hslope) * np.sin(2.0 * np.pi * x2)
    dthg = np.pi * (1.0 + (1.0 - g.hslope) * np.cos(2.0 * np.pi * x2))
    y = 2.0 * x2 - 1.0
    al = g.poly_alpha
    norm = 0.5 * np.pi / (1.0 + 1.0 / ((al + 1.0) * g.poly_xt ** al))
    th_j = norm * y * (1.0 + (y / g.poly_xt) ** al / (al + 1.0)) + 0.5 * np.pi
    dthj = 2.0 * norm * (1.0 + (y / g.poly_xt) ** al)
    w = np.exp(g.mks_smooth * (x1in - x1))
    th = th_g + w * (th_j - th_g)
    dth_dx1 = -g.mks_smooth * w * (th_j - th_g)
    dth_dx2 = dthg + w * (dthj - dthg)
    return th, dth_dx1, dth_dx2


def _fm_lnh(r, th, a, r_in, r_max):
    """Fishbone & Moncrief (1976) torus: ln(enthalpy), zero at (r_in, pi/2).

    The conserved quantity l = u^t u_phi is taken from the prograde Keplerian circular orbit
    at the pressure maximum r_max (Bardeen, Press & Teukolsky 1972 orbit formulae).
    """
    sq = math.sqrt(r_max)
    l = (r_max ** 1.5 + a) * (r_max ** 2 - 2.0 * a * sq + a * a) / (
        r_max ** 1.5 * (r_max ** 1.5 - 3.0 * sq + 2.0 * a))

    def raw(r, th):
        s2 = np.sin(th) ** 2
        sig = r * r + a * a * np.cos(th) ** 2
        dl = r * r - 2.0 * r + a * a
        A = (r * r + a * a) ** 2 - dl * a * a * s2
        root = np.sqrt(1.0 + 4.0 * l * l * sig * sig * dl / (A * A * s2))
        return 0.5 * np.log((1.0 + root) / (sig * dl / A)) - 0.5 * root - 2.0 * a * r * l / A

    return raw(r, th) - raw(np.asarray(r_in), np.asarray(0.5 * np.pi)), l


@dataclass
class TorusParams:
    r_in: float = 6.0
    r_max: float = 12.0
    kappa_poly: float = 1.0e-3
    beta_min: float = 0.1
    aphi_cut: float = 0.2
    sigma_pert: float = 0.5
    rho_atm: float = 1.0e-5
    u_atm: float = 1.0e-7


def fm_torus_grid(seed: int = 1, grid: GridParams | None = None, torus: TorusParams | None = None):
    """Seeded FM torus on an FMKS grid (see _fm_torus_grid)."""
    with np.errstate(invalid="ignore", divide="ignore"):
        return _fm_torus_grid(seed, grid, torus)


def _fm_torus_grid(seed, grid, torus):
    """Seeded FM torus on an FMKS grid; returns (prims[n1,n2,n3,8] float32, GridParams).

    Primitive order per cell: rho, u, U1, U2, U3, B1, B2, B3, with U^i the fluid velocity
    relative to the normal observer and B^i the field, both in FMKS components (X1 = ln r,
    X2 in [0, 1], X3 = phi in [0, 2 pi)), cell-centred.
    """
    g = (grid or GridParams()).resolved()
    t = torus or TorusParams()
    a, gam = g.a, g.gamma_ad
    x1in, x1out = math.log(g.r_in), math.log(g.r_out)
    dx1 = (x1out - x1in) / g.n1
    x1 = x1in + (np.arange(g.n1) + 0.5) * dx1
    x2 = (np.arange(g.n2) + 0.5) / g.n2
    X1, X2 = np.meshgrid(x1, x2, indexing="ij")
    r = np.exp(X1)
    th, dth1, dth2 = _fmks_theta(X1, X2, g)

    def torus_rho_u(r, th):
        lnh, _ = _fm_lnh(r, th, a, t.r_in, t.r_max)
        inside = (lnh > 0.0) & (r >= t.r_in)
        h = np.exp(np.where(inside, lnh, 0.0))
        rho = np.where(inside, ((h - 1.0) * (gam - 1.0) / (t.kappa_poly * gam)) ** (1.0 / (gam - 1.0)), 0.0)
        u = t.kappa_poly * rho ** gam / (gam - 1.0)
        return rho, u, inside

    rho_t, u_t, inside = torus_rho_u(r, th)
    rho_max = float(rho_t.max())
    rho_t, u_t = rho_t / rho_max, u_t / rho_max
    rho_a = t.rho_atm * r ** -1.5
    u_a = t.u_atm * r ** -2.5
    use_t = inside & (rho_t > rho_a)
    rho = np.where(use_t, rho_t, rho_a)
    uu = np.where(use_t, u_t, u_a)

    # --- spatial Kerr-Schild metric pieces at cell centres (input construction only) ---
    s, c = np.sin(th), np.cos(th)
    sig = r * r + a * a * c * c
    q = 2.0 * r / sig
    # circular FM flow (Boyer-Lindquist u^t, u^phi; u^r = u^theta = 0 so KS components match)
    _, lfm = _fm_lnh(np.asarray(t.r_max), np.asarray(0.5 * np.pi), a, t.r_in, t.r_max)
    dl = r * r - 2.0 * r + a * a
    A = (r * r + a * a) ** 2 - dl * a * a * s * s
    w2 = 0.5 * (-1.0 + np.sqrt(1.0 + 4.0 * lfm * lfm * sig * sig * dl / (A * A * s * s)))
    w = np.sqrt(w2)
    alpha_bl = np.sqrt(sig * dl / A)
    ut_bl = np.sqrt(1.0 + w2) / alpha_bl
    uphi = 2.0 * a * r * np.sqrt(1.0 + w2) / np.sqrt(A * sig * dl) + np.sqrt(sig / A) * w / s
    # KS normal-observer frame: lapse^2 = 1/(1+q), shift^r = q/(1+q)
    ur_tilde_ks = ut_bl * q / (1.0 + q)
    U1 = np.where(use_t, ur_tilde_ks / r, 0.0)
    U2 = np.where(use_t, -dth1 * (ur_tilde_ks / r) / dth2, 0.0)
    U3 = np.where(use_t, uphi, 0.0)

    # --- poloidal field from A_phi = max(rho/rho_max - cut, 0), central differences ---
    def aphi(x1v, x2v):
        rr = np.exp(x1v)
        tt, _, _ = _fmks_theta(x1v, x2v, g)
        rt, _, _ = torus_rho_u(rr, tt)
        return np.maximum(rt / rho_max - t.aphi_cut, 0.0)

    e1, e2 = 0.25 * dx1, 0.25 / g.n2
    dA1 = (aphi(X1 + e1, X2) - aphi(X1 - e1, X2)) / (2 * e1)
    dA2 = (aphi(X1, X2 + e2) - aphi(X1, X2 - e2)) / (2 * e2)
    gdet = sig * s * r * dth2          # sqrt(-g) in FMKS
    B1 = -dA2 / gdet
    B2 = dA1 / gdet
    # b^2 for normalisation: KS components, fluid at rest in phi only
    Br = r * B1
    Bth = dth1 * B1 + dth2 * B2
    g_rr = 1.0 + q
    g_thth = sig
    g_rph = -a * s * s * (1.0 + q)
    g_phph = s * s * (sig + a * a * s * s * (1.0 + q))
    g_tr, g_tph, g_tt = q, -a * s * s * q, -1.0 + q
    # fluid 4-velocity in KS: u^t = ut_bl, u^r = 0, u^phi = uphi (torus)
    ut = np.where(use_t, ut_bl, np.sqrt(1.0 + q))
    up = np.where(use_t, uphi, 0.0)
    u_r = g_tr * ut + g_rph * up
    u_th = 0.0 * ut
    u_ph = g_tph * ut + g_phph * up
    bt = Br * u_r + Bth * u_th
    br = (Br + bt * 0.0) / ut
    bth = Bth / ut
    bph = (bt * up) / ut
    bsq = (g_tt * bt * bt + 2 * g_tr * bt * br + 2 * g_tph * bt * bph + g_rr * br * br
           + 2 * g_rph * br * bph + g_thth * bth * bth + g_phph * bph * bph)
    pg = (gam - 1.0) * uu
    sel = use_t & (bsq > 0)
    beta_now = np.min(pg[sel] / (0.5 * bsq[sel])) if np.any(sel) else 1.0
    norm = math.sqrt(beta_now / t.beta_min)
    B1 *= norm
    B2 *= norm

    # --- 3-D fill with per-cell log-normal factors ---
    n1, n2, n3 = g.n1, g.n2, g.n3
    ncell = n1 * n2 * n3
    cells = np.arange(ncell, dtype=np.uint64)
    sp = t.sigma_pert
    f_rho = np.exp(sp * gauss(seed, cells * np.uint64(2)) - 0.5 * sp * sp).reshape(n1, n2, n3)
    f_b = np.exp(sp * gauss(seed, cells * np.uint64(2) + np.uint64(1)) - 0.5 * sp * sp).reshape(n1, n2, n3)
    prims = np.empty((n1, n2, n3, 8), dtype=np.float32)
    prims[..., 0] = (rho[:, :, None] * f_rho)
    prims[..., 1] = uu[:, :, None]
    prims[..., 2] = U1[:, :, None]
    prims[..., 3] = U2[:, :, None]
    prims[..., 4] = U3[:, :, None]
    prims[..., 5] = B1[:, :, None] * f_b
    prims[..., 6] = B2[:, :, None] * f_b
    prims[..., 7] = 0.0
    return prims, g


# ----------------------------------------------------------------------------------------
# Cameras, workloads and the batched job table
# ----------------------------------------------------------------------------------------
MSUN_G = 1.98847e33
KPC_CM = 3.0856775814913673e21


@dataclass
class Camera:
    a: float = 0.9375
    incl_deg: float = 60.0
    r_cam: float = 1000.0
    freq_hz: float = 230.0e9
    fov_M: float = 40.0
    nx: int = 64
    ny: int = 64
    M_bh_g: float = 4.1e6 * MSUN_G
    dist_cm: float = 8.1 * KPC_CM


@dataclass
class Integrator:
    eps: float = 0.05
    nmax: int = 20000


def workload(name: str) -> dict:
    """Named workloads of the benchmark suite (sizes only; models built on request).

    adaf64:   ADAF, a=0.9375, i=60 deg, 230 GHz, 64x64, FOV 40 M, r_cam = 1000 M, seed 1.
    grmhd1024: FM-torus FMKS grid 288x128x128, R_high = 40, i = 20 deg, 1024x1024.
    adaf4096: the ADAF at 4096x4096.
    """
    if name == "adaf64":
        return {"model": "adaf", "camera": Camera(incl_deg=60.0, nx=64, ny=64)}
    if name == "grmhd1024":
        return {"model": "grid", "camera": Camera(incl_deg=20.0, nx=1024, ny=1024)}
    if name == "adaf4096":
        return {"model": "adaf", "camera": Camera(incl_deg=60.0, nx=4096, ny=4096)}
    raise KeyError(name)


@dataclass
class Job:
    image: int
    n: int
    incl_deg: float
    R_high: float
    M_unit: float
    kappa: float = 0.0


def batch_jobs(seed: int = 7, njobs: int = 96, with_kappa: bool = False) -> list[Job]:
    """Image-library job table: N in {128,256,512}, i ~ U(10,170) deg, log R_high ~ U(0, ln 160),
    log10 M_unit ~ U(17, 20); optionally kappa ~ U(3, 8)."""
    jobs = []
    for j in range(njobs):
        u = uniform(seed, [5 * j + k for k in range(5)])
        n = (128, 256, 512)[min(int(u[0] * 3.0), 2)]
        jobs.append(Job(image=j, n=n, incl_deg=10.0 + 160.0 * float(u[1]),
                        R_high=math.exp(math.log(160.0) * float(u[2])),
                        M_unit=10.0 ** (17.0 + 3.0 * float(u[3])),
                        kappa=(3.0 + 5.0 * float(u[4])) if with_kappa else 0.0))
    return jobs
