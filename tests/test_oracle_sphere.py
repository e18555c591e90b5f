"""Pins of the oracle's camera-to-flux chain and of its depth maps with a static sphere.

A sphere of plasma at rest around a Schwarzschild hole (a = 0) has a closed-form image:

* Optically thick, every ray that enters it reads, at the camera, the Planck intensity of the
  point where it last left the plasma, redshifted by sqrt((1 - 2/r_cam) / (1 - 2/r)) with
  I / nu^3 invariant, and no polarization (Kirchhoff's law for every Stokes component makes
  (B_nu, 0, 0, 0) the fixed point of the constant-coefficient step).
* Its silhouette is the circle of impact parameter b = R / sqrt(1 - 2/R) (R outside the photon
  sphere), which a static camera at r_cam sees at the angle sin(psi) = b sqrt(1 - 2/r_cam) / r_cam
  from the centre, i.e. at image-plane radius r_cam tan(psi).
* So the flux is the Planck intensity times the silhouette's solid angle, pi (r_cam tan psi)^2
  (L / D)^2, in Jy: this fixes the pixel solid angle (FOV, nx, L, D, the 1e23) without restating it.

The depth maps (tau = sum alpha_I ds, phi = sum rho_V ds) are checked against the same integrals
taken along the orbit of an independent Schwarzschild integration (the orbit equation
u'' = 3 u^2 - u, u = 1/r, by scipy's DOP853) for rays in the equatorial plane of an edge-on
camera, where the toroidal field makes cos(theta_B) = -sign(x) (b / r) sqrt(1 - 2/r).
"""
import numpy as np
import pytest
from scipy.integrate import solve_ivp

ME, C, H, KB, G = 9.1093837015e-28, 2.99792458e10, 6.62607015e-27, 1.380649e-16, 6.67430e-8
R = 10.0


def _planck(nu, theta_e):
    T = theta_e * ME * C * C / KB
    return 2 * H * nu ** 3 / C ** 2 / np.expm1(H * nu / (KB * T))


def _pixel(cam, ix, iy):
    """Image-plane coordinates [M] of a pixel centre (square pixels of side FOV / nx)."""
    px = ((ix + 0.5) / cam.nx - 0.5) * cam.fov_M
    py = ((iy + 0.5) / cam.ny - 0.5) * cam.fov_M * cam.ny / cam.nx
    return px, py


def _impact(cam, px, py):
    """Impact parameter of the ray a static camera at r_cam receives from image point (px, py):
    the sky direction makes tan(psi) = |(px, py)| / r_cam with the radial leg, the photon's
    angular momentum is r_cam sin(psi) in units of its camera-frame energy, and its energy at
    infinity is sqrt(1 - 2/r_cam) of that."""
    t = np.hypot(px, py) / cam.r_cam
    return cam.r_cam * t / np.sqrt(1 + t * t) / np.sqrt(1 - 2 / cam.r_cam)


def _thick(ora, synth, eps, nx=48, ny=36, fov=32.0):
    cam = synth.Camera(a=0.0, incl_deg=90.0, fov_M=fov, nx=nx, ny=ny)
    ocam = ora.camera(cam, eps=eps)
    ne, te, B = 1e11, 5.0, 50.0
    model = ora.sphere_model(R, ne, te, B)
    img = ora.render_image(ocam, model)[0]
    return cam, ocam, img, te, model


@pytest.fixture(scope="module")
def thick(ora, synth):
    return {eps: _thick(ora, synth, eps) for eps in (0.05, 0.025)}


def test_thick_sphere_silhouette(ora, thick):
    cam, _, img, _, _ = thick[0.05]
    b_crit = R / np.sqrt(1 - 2 / R)
    iy, ix = np.meshgrid(np.arange(cam.ny), np.arange(cam.nx), indexing="ij")
    b = _impact(cam, *_pixel(cam, ix, iy))
    lit = img[..., 0] > 0
    assert lit[b < b_crit - 0.2].all()
    # a ray that only grazes the surface can step over it: a band of 0.2 M is left open
    assert not lit[b > b_crit].any()
    assert lit.sum() > 600


def test_thick_sphere_planck_intensity_converges(ora, thick):
    """Each lit pixel equals the redshifted Planck intensity of its ray's last point inside the
    sphere, the residual is the transport's second-order error in the step parameter."""
    errs = {}
    for eps, (cam, ocam, img, te, model) in thick.items():
        L = G * cam.M_bh_g / C ** 2
        e, p = [], []
        for iy in range(cam.ny):
            for ix in range(cam.nx):
                if img[iy, ix, 0] <= 0:
                    continue
                states, _ = ora.trace_geodesic(ocam, *_pixel(cam, ix, iy))
                n = np.nonzero(states[:, 1] < R)[0].min()
                x, K = states[n, :4], states[n, 4:8]
                w = np.sqrt((1 - 2 / cam.r_cam) / (1 - 2 / x[1]))
                ref = _planck(cam.freq_hz * w, te) / w ** 3
                # only where the last step alone is optically thick (not the grazing rays):
                # its optical depth alpha_I(nu w, theta_B) w h L above 40
                pl = ora.plasma(ocam, model, x)
                th_b = ora.fluid_tetrad(0.0, x, K, pl[4:8], pl[8:12])[1]
                tau_last = ora.thermal_coeffs(pl[0], te, pl[2], cam.freq_hz * w, th_b)[3] * w * abs(states[n, 8]) * L
                if tau_last > 40:
                    e.append(img[iy, ix, 0] / ref - 1)
                    p.append(np.abs(img[iy, ix, 1:]).max() / img[iy, ix, 0])
                assert img[iy, ix, 0] <= ref * (1 + 1e-3)
        errs[eps] = (np.abs(e).max(), np.max(p), len(e))
    (e1, p1, n1), (e2, p2, n2) = errs[0.05], errs[0.025]
    assert n1 > 600 and n2 > 600
    assert e1 < 1e-3 and p1 < 1e-3
    assert e2 < e1 / 3 and p2 < p1 / 3, errs


def test_thick_sphere_flux_is_planck_times_silhouette(ora, synth, thick):
    """The image-statistics chain (pixel solid angle, L, D, Jy) against B_nu pi rho^2 (L/D)^2, for
    two resolutions of a non-square image and for a wider field of view. The 1% allows for the
    count of pixel centres inside the silhouette and for rays whose last point lies a little
    below the surface (a redshift of up to a few 1e-3)."""
    b_crit = R / np.sqrt(1 - 2 / R)
    cases = [thick[0.05], _thick(ora, synth, 0.05, nx=96, ny=72), _thick(ora, synth, 0.05, nx=120, ny=90, fov=44.0)]
    for cam, ocam, img, te, _ in cases:
        L = G * cam.M_bh_g / C ** 2
        sin_psi = b_crit * np.sqrt(1 - 2 / cam.r_cam) / cam.r_cam
        rho = cam.r_cam * np.tan(np.arcsin(sin_psi))
        w = np.sqrt((1 - 2 / cam.r_cam) / (1 - 2 / R))
        i_surf = _planck(cam.freq_hz * w, te) / w ** 3
        flux_ref = i_surf * np.pi * rho ** 2 * (L / cam.dist_cm) ** 2 * 1e23
        flux, lp, cp = ora.image_stats(ocam, img.reshape(-1, 4))
        assert abs(flux / flux_ref - 1) < 0.01, (cam.nx, cam.ny, flux, flux_ref)
        assert lp < 1e-3 and abs(cp) < 1e-3


def _depth_exact(ora, cam, px, ne, te, B):
    """(tau, phi) along the equatorial ray of image point (px, 0) through the smooth sphere, by
    the orbit equation in Schwarzschild coordinates: d lambda = r^2 d phi / L_z, and the
    fluid-frame length ds = w L d lambda with w = E / sqrt(1 - 2/r), E = sqrt(1 - 2/r_cam)."""
    L = G * cam.M_bh_g / C ** 2
    b = _impact(cam, px, 0.0)
    E = np.sqrt(1 - 2 / cam.r_cam)
    lz = b * E
    sgn = -np.sign(px)

    def rhs(_, y):
        u, up = y[0], y[1]
        r = 1 / u
        w = E / np.sqrt(1 - 2 / r)
        cth = sgn * (b / r) * np.sqrt(1 - 2 / r)
        q = 1 - r * r / (R * R)
        c = ora.thermal_coeffs(ne * q * q, te, B, cam.freq_hz * w, np.arccos(np.clip(cth, -1.0, 1.0)))
        f = w * L * r * r / lz
        return [up, 3 * u * u - u, c[3] * f, c[7] * f]

    def cross(direction):
        ev = lambda _, y: y[0] - 1 / R
        ev.terminal, ev.direction = True, direction
        return ev

    u0 = 1 / cam.r_cam
    y0 = [u0, np.sqrt(1 / b ** 2 - u0 ** 2 * (1 - 2 * u0)), 0.0, 0.0]
    s1 = solve_ivp(lambda _, y: [y[1], 3 * y[0] ** 2 - y[0], 0, 0], (0, 10), y0, events=cross(1),
                   method="DOP853", rtol=1e-12, atol=1e-15)
    ent = s1.y_events[0][0]
    s2 = solve_ivp(rhs, (s1.t_events[0][0], s1.t_events[0][0] + 10), [1 / R, ent[1], 0.0, 0.0], events=cross(-1),
                   method="DOP853", rtol=1e-10, atol=[1e-14, 1e-14, 1e-16, 1e-14])
    out = s2.y_events[0][0]
    return out[2], out[3]


def test_depth_maps_match_the_orbit_integrals(ora, synth):
    """Optical and Faraday depth of escaping rays through the sphere, within the first-order
    error of taking the coefficients at each segment's arrival point, and shrinking with eps."""
    ne, te, B = 1e5, 5.0, 50.0
    model = ora.sphere_model(R, ne, te, B, smooth=True)
    b_crit, b_ph = R / np.sqrt(1 - 2 / R), np.sqrt(27.0)
    worst = {}
    for eps in (0.05, 0.0125):
        cam = synth.Camera(a=0.0, incl_deg=90.0, fov_M=30.0, nx=30, ny=3)
        ix = np.arange(cam.nx)
        dep = ora.render_pixels(ora.camera(cam, eps=eps), model, ix, np.ones_like(ix), depth=True)[4]
        errs = []
        for i in ix:
            px, _ = _pixel(cam, i, 1)
            if not (b_ph + 0.5 < _impact(cam, px, 0.0) < b_crit - 0.3):
                continue
            tau, phi = _depth_exact(ora, cam, px, ne, te, B)
            assert tau > 0 and np.sign(phi) == -np.sign(px)
            errs.append(max(abs(dep[i, 0] / tau - 1), abs(dep[i, 1] / phi - 1)))
        assert len(errs) >= 8
        worst[eps] = max(errs)
    assert worst[0.05] < 1e-3, worst
    assert worst[0.0125] < worst[0.05] / 4, worst
