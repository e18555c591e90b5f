"""Pins of the oracle's plasma models: FMKS coordinates, the trilinear fetch, the HARM
primitive-to-four-vector conversion and the semi-analytic ADAF."""
import numpy as np
import pytest


def test_fmks_end_points_and_monotonic(ora, synth, small_grid):
    prims, g = small_grid
    m = ora.grid_model(prims, g)
    for X1 in (np.log(g.r_in), np.log(5.0), np.log(900.0)):
        assert abs(ora.fmks_theta(m, X1, 0.0)[0]) < 1e-15
        assert abs(ora.fmks_theta(m, X1, 1.0)[0] - np.pi) < 1e-14
        assert abs(ora.fmks_theta(m, X1, 0.5)[0] - np.pi / 2) < 1e-15
        x2 = np.linspace(0, 1, 2001)
        th = np.array([ora.fmks_theta(m, X1, v)[0] for v in x2])
        assert np.all(np.diff(th) > 0)
        # reflection symmetry theta(1 - X2) = pi - theta(X2)
        assert np.allclose(th[::-1], np.pi - th, atol=1e-14)


def test_fmks_derivatives_and_inverse(ora, small_grid):
    prims, g = small_grid
    m = ora.grid_model(prims, g)
    h = 1e-6
    for X1 in (np.log(1.3), np.log(12.0), np.log(300.0)):
        for X2 in (0.02, 0.31, 0.5, 0.77, 0.99):
            th, d1, d2 = ora.fmks_theta(m, X1, X2)
            f1 = (ora.fmks_theta(m, X1 + h, X2)[0] - ora.fmks_theta(m, X1 - h, X2)[0]) / (2 * h)
            f2 = (ora.fmks_theta(m, X1, X2 + h)[0] - ora.fmks_theta(m, X1, X2 - h)[0]) / (2 * h)
            assert abs(d1 - f1) < 1e-7 and abs(d2 - f2) < 1e-7 * abs(d2)
            assert abs(ora.fmks_x2(m, X1, th) - X2) < 1e-14


def test_trilinear_reproduces_linear_fields(ora, synth):
    g = synth.GridParams(n1=10, n2=8, n3=6).resolved()
    i, j, k = np.meshgrid(np.arange(10), np.arange(8), np.arange(6), indexing="ij")
    prims = np.zeros((10, 8, 6, 8), dtype=np.float32)
    for v in range(8):
        prims[..., v] = (0.5 + v) * i - 0.25 * v * j + 2.0 * k * (v % 3) + v
    m = ora.grid_model(prims, g)
    x1in = np.log(g.r_in)
    dx1 = (np.log(g.r_out) - x1in) / 10
    rng = np.random.default_rng(3)
    for _ in range(50):
        fi, fj, fk = rng.uniform(0, 9), rng.uniform(0, 7), rng.uniform(0, 5)
        out = ora.grid_interp(m, x1in + (fi + 0.5) * dx1, (fj + 0.5) / 8, (fk + 0.5) * 2 * np.pi / 6)
        ref = np.array([(0.5 + v) * fi - 0.25 * v * fj + 2.0 * fk * (v % 3) + v for v in range(8)])
        assert np.allclose(out, ref, atol=1e-12)
    # clamped beyond the first / last centres, periodic in X3
    a = ora.grid_interp(m, x1in + 0.1 * dx1, 0.01, 0.0)
    b = ora.grid_interp(m, x1in + 0.5 * dx1, 0.5 / 8, 2 * np.pi)
    assert np.allclose(a, b, atol=1e-12)


def _ks_metric(ora, a, x):
    return ora.metric(a, x[1], x[2])


def test_grid_four_vectors(ora, synth, small_grid):
    prims, g = small_grid
    m = ora.grid_model(prims, g)
    cam = ora.camera(synth.Camera())
    rng = np.random.default_rng(11)
    n_valid = 0
    for _ in range(200):
        x = np.array([0.0, np.exp(rng.uniform(np.log(1.5), np.log(60))), rng.uniform(0.05, np.pi - 0.05),
                      rng.uniform(0, 2 * np.pi)])
        pl = ora.plasma(cam, m, x)
        if pl[3] == 0:
            continue
        n_valid += 1
        gm = _ks_metric(ora, cam.a, x)
        u, b = pl[4:8], pl[8:12]
        assert np.isclose(u @ gm @ u, -1.0, atol=1e-12)
        assert abs(u @ gm @ b) < 1e-12 * max(1.0, np.sqrt(abs(b @ gm @ b)))
        assert u[0] > 0 and pl[0] > 0 and pl[1] > 0
    assert n_valid > 50


def test_grid_static_fluid_is_normal_observer_and_units(ora, synth):
    """U^i = 0 gives the normal observer (u_i = 0); B = 0 gives R = R_high and the
    temperature (m_p/m_e)(gamma - 1) u / (rho (1 + R_high))."""
    g = synth.GridParams(n1=8, n2=8, n3=4, M_unit=3e18, R_high=20.0).resolved()
    prims = np.zeros((8, 8, 4, 8), dtype=np.float32)
    prims[..., 0] = 2.0
    prims[..., 1] = 0.05
    m = ora.grid_model(prims, g)
    cam = ora.camera(synth.Camera())
    x = np.array([0.0, 7.0, 1.1, 0.4])
    pl = ora.plasma(cam, m, x)
    gm = _ks_metric(ora, cam.a, x)
    ul = gm @ pl[4:8]
    assert np.allclose(ul[1:], 0.0, atol=1e-14)
    MP, ME, G, C = 1.67262192369e-24, 9.1093837015e-28, 6.67430e-8, 2.99792458e10
    L = G * cam.M_bh_g / C ** 2
    assert np.isclose(pl[0], 2.0 * 3e18 / L ** 3 / (MP + ME), rtol=1e-12)
    assert np.isclose(pl[1], MP / ME * (g.gamma_ad - 1) * 0.05 / (2.0 * 21.0), rtol=1e-6)
    assert pl[2] == 0.0


def test_grid_sigma_cut_and_outside(ora, synth):
    g = synth.GridParams(n1=8, n2=8, n3=4).resolved()
    prims = np.zeros((8, 8, 4, 8), dtype=np.float32)
    prims[..., 0] = 1e-4
    prims[..., 1] = 1e-6
    prims[..., 5] = 1.0   # strong radial field: sigma = b^2 / rho >> 1
    m = ora.grid_model(prims, g)
    cam = ora.camera(synth.Camera())
    assert ora.plasma(cam, m, np.array([0, 10.0, 1.0, 0.0]))[3] == 0.0
    prims[..., 5] = 0.0
    m = ora.grid_model(prims, g)
    assert ora.plasma(cam, m, np.array([0, 10.0, 1.0, 0.0]))[3] == 1.0
    assert ora.plasma(cam, m, np.array([0, 1.01 * g.r_out, 1.0, 0.0]))[3] == 0.0


def test_adaf_plasma(ora, synth):
    p = synth.adaf_params(1)
    m = ora.adaf_model(p)
    cam = ora.camera(synth.Camera())
    a = cam.a
    KB, ME, C = 1.380649e-16, 9.1093837015e-28, 2.99792458e10
    rng = np.random.default_rng(5)
    for _ in range(60):
        r = np.exp(rng.uniform(np.log(1.42), np.log(900)))
        th = rng.uniform(0.05, np.pi - 0.05)
        x = np.array([0.0, r, th, rng.uniform(0, 6)])
        pl = ora.plasma(cam, m, x)
        assert pl[3] == 1.0
        gm = _ks_metric(ora, a, x)
        u, b = pl[4:8], pl[8:12]
        ul = gm @ u
        assert np.isclose(u @ gm @ u, -1.0, atol=1e-12)
        assert abs(u @ gm @ b) < 1e-10 * np.sqrt(b @ gm @ b)
        # u_t = -1 and u_phi = l are invariant under the BL -> KS map (t and phi shift by f(r))
        z1 = 1 + np.cbrt(1 - a * a) * (np.cbrt(1 + a) + np.cbrt(1 - a))
        z2 = np.sqrt(3 * a * a + z1 * z1)
        rk = max(r, 3 + z2 - np.sqrt((3 - z1) * (3 + z1 + 2 * z2)))
        lK = (rk ** 2 - 2 * a * np.sqrt(rk) + a * a) / (rk ** 1.5 - 2 * np.sqrt(rk) + a)
        assert np.isclose(ul[0], -1.0, rtol=1e-10)
        assert np.isclose(ul[3], p.f_kep * lK * np.sin(th) ** 2, rtol=1e-9, atol=1e-12)
        assert u[1] < 0   # inflow
        # the field has no theta component (B^i along (1, 0, 1/r)) and u^theta = 0, so b^theta = 0
        assert u[2] == 0.0 and abs(b[2]) <= 1e-14 * np.abs(b).max()
        assert np.isclose(pl[0], p.n0 * r ** -1.5, rtol=1e-13)
        Te = p.T0 / r
        assert np.isclose(pl[1], KB * Te / (ME * C * C), rtol=1e-13)
        assert np.isclose(pl[2] ** 2 / (8 * np.pi), pl[0] * KB * Te * (1 + p.Ti_over_Te) / p.beta, rtol=1e-12)
    assert ora.plasma(cam, m, np.array([0.0, 1001.0, 1.0, 0.0]))[3] == 0.0


@pytest.mark.parametrize("scale,r,th", [(1.0, 7.0, 1.1), (0.3, 18.0, 2.3)])
def test_grid_field_and_temperature_by_hand(ora, synth, scale, r, th):
    """A static fluid (U = 0) in a uniform FMKS field, worked by hand at one point.
    - The field's KS components follow from the FMKS Jacobian: B^r = r B^1,
      B^theta = (dtheta/dX1) B^1 + (dtheta/dX2) B^2, B^phi = B^3.
    - For the normal observer (u_i = 0), b^t = 0 and b^i = alpha B^i.
    - B = |b| c sqrt(4 pi rho_unit).
    - beta = 2 (gamma - 1) u / b^2, so R = R_high beta^2/(1 + beta^2) + R_low/(1 + beta^2).
    - Theta_e = (m_p/m_e)(gamma - 1) u / (rho (1 + R)).
    The two cases put beta on either side of one, where both terms of R count."""
    g = synth.GridParams(n1=8, n2=8, n3=4, M_unit=3e18, R_high=20.0).resolved()
    vals = np.array([2.0, 0.05, 0.0, 0.0, 0.0, 0.012 * scale, 0.02 * scale, 0.03 * scale], dtype=np.float32)
    m = ora.grid_model(np.broadcast_to(vals, (8, 8, 4, 8)).copy(), g)
    cam = ora.camera(synth.Camera())
    pl = ora.plasma(cam, m, np.array([0.0, r, th, 0.4]))
    assert pl[3] == 1.0
    v = vals.astype(np.float64)
    X1 = np.log(r)
    th_back, d1, d2 = ora.fmks_theta(m, X1, ora.fmks_x2(m, X1, th))
    assert abs(th_back - th) < 1e-12
    gm = ora.metric(cam.a, r, th)
    alpha = 1.0 / np.sqrt(-np.linalg.inv(gm)[0, 0])
    b = alpha * np.array([0.0, r * v[5], d1 * v[5] + d2 * v[6], v[7]])
    b2 = b @ gm @ b
    MP, ME, G, C = 1.67262192369e-24, 9.1093837015e-28, 6.67430e-8, 2.99792458e10
    L = G * cam.M_bh_g / C ** 2
    beta = 2.0 * (g.gamma_ad - 1.0) * v[1] / b2
    R = g.R_high * beta ** 2 / (1 + beta ** 2) + g.R_low / (1 + beta ** 2)
    assert 0.2 < beta < 5.0 and 1.5 < R < 19.0
    assert np.allclose(pl[8:12], b, rtol=1e-12, atol=1e-15)
    assert np.isclose(pl[2], np.sqrt(b2) * C * np.sqrt(4 * np.pi * g.M_unit / L ** 3), rtol=1e-12)
    assert np.isclose(pl[1], MP / ME * (g.gamma_ad - 1) * v[1] / (v[0] * (1 + R)), rtol=1e-12)
