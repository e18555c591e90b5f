"""Pins of the oracle's geometry: metric, connection, camera and geodesic integration.

Everything here is checked against something other than the oracle's own formula: the
Boyer-Lindquist metric moved to Kerr-Schild coordinates by its Jacobian, finite differences,
closed-form Kerr orbits (the a = 0 photon sphere, Synge's shadow, Bardeen's critical curve)
and the constants of motion E, L and Carter's Q.
"""
import numpy as np
import pytest

A = 0.9375


def ks_from_bl(a, r, th):
    """Textbook Boyer-Lindquist metric pulled back to ingoing Kerr-Schild coordinates."""
    s, c = np.sin(th), np.cos(th)
    sig, D = r * r + a * a * c * c, r * r - 2 * r + a * a
    g = np.zeros((4, 4))
    g[0, 0] = -(1 - 2 * r / sig)
    g[0, 3] = g[3, 0] = -2 * a * r * s * s / sig
    g[1, 1] = sig / D
    g[2, 2] = sig
    g[3, 3] = (r * r + a * a + 2 * a * a * r * s * s / sig) * s * s
    J = np.eye(4)
    J[0, 1] = -2 * r / D
    J[3, 1] = -a / D
    return J.T @ g @ J


@pytest.mark.parametrize("r,th", [(3.0, 1.0), (10.0, 0.3), (1.7, 2.0), (800.0, 1.2), (2.5, 3.1)])
def test_metric_matches_boyer_lindquist(ora, r, th):
    g = ora.metric(A, r, th)
    ref = ks_from_bl(A, r, th)
    assert np.allclose(g, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("r,th", [(3.0, 1.0), (1.5, 0.2), (50.0, 2.9)])
def test_inverse_and_determinant_closed_form(ora, r, th):
    g = ora.metric(A, r, th)
    gi = np.zeros(16)
    ora.lib().ora_invert4(ora._dp(np.ascontiguousarray(g.ravel())), ora._dp(gi))
    gi = gi.reshape(4, 4)
    s, c = np.sin(th), np.cos(th)
    sig = r * r + A * A * c * c
    q = 2 * r / sig
    ref = np.zeros((4, 4))
    ref[0, 0], ref[0, 1], ref[1, 0] = -(1 + q), q, q
    ref[1, 1] = (r * r - 2 * r + A * A) / sig
    ref[1, 3] = ref[3, 1] = A / sig
    ref[2, 2] = 1 / sig
    ref[3, 3] = 1 / (sig * s * s)
    assert np.allclose(gi, ref, rtol=1e-12, atol=1e-14)
    assert np.isclose(np.linalg.det(g), -(sig * s) ** 2, rtol=1e-12)


@pytest.mark.parametrize("r,th", [(2.0, 0.7), (6.0, 1.5), (30.0, 2.4)])
def test_metric_derivatives_vs_finite_differences(ora, r, th):
    dr, dt = ora.metric_derivs(A, r, th)
    h = 1e-6
    fr = (ora.metric(A, r + h * r, th) - ora.metric(A, r - h * r, th)) / (2 * h * r)
    ft = (ora.metric(A, r, th + h) - ora.metric(A, r, th - h)) / (2 * h)
    scale = max(np.abs(fr).max(), np.abs(ft).max())
    assert np.allclose(dr, fr, atol=1e-7 * scale)
    assert np.allclose(dt, ft, atol=1e-7 * scale)


@pytest.mark.parametrize("r,th", [(2.2, 0.9), (7.0, 1.4), (40.0, 0.4)])
def test_connection_vs_numerical_christoffel(ora, r, th):
    """Gamma from central differences of the metric and numpy's inverse."""
    h = 1e-6
    dg = np.zeros((4, 4, 4))
    dg[1] = (ks_from_bl(A, r + h * r, th) - ks_from_bl(A, r - h * r, th)) / (2 * h * r)
    dg[2] = (ks_from_bl(A, r, th + h) - ks_from_bl(A, r, th - h)) / (2 * h)
    gi = np.linalg.inv(ks_from_bl(A, r, th))
    ref = 0.5 * (np.einsum("mn,anb->mab", gi, dg) + np.einsum("mn,bna->mab", gi, dg)
                 - np.einsum("mn,nab->mab", gi, dg))
    G = ora.connection(A, r, th)
    assert np.allclose(G, ref, atol=1e-7 * np.abs(ref).max())


def test_schwarzschild_photon_sphere_is_circular(ora):
    """a = 0: a photon on the circle r = 3 with u^phi/u^t = 1/sqrt(27) has zero acceleration."""
    r, th = 3.0, np.pi / 2
    G = ora.connection(0.0, r, th)
    K = np.array([1.0, 0.0, 0.0, 1.0 / np.sqrt(27.0)])
    acc = -np.einsum("mab,a,b->m", G, K, K)
    g = ora.metric(0.0, r, th)
    assert abs(K @ g @ K) < 1e-14
    assert np.allclose(acc, 0.0, atol=1e-14)


def test_camera_ray_is_null_with_unit_energy(ora, synth):
    cam = ora.camera(synth.Camera(incl_deg=60.0))
    for px, py in [(0.0, 0.0), (7.3, -4.1), (-19.9, 19.9)]:
        x, K = ora.camera_ray(cam, px, py)
        g = ora.metric(cam.a, x[1], x[2])
        u = np.array([1.0 / np.sqrt(-g[0, 0]), 0, 0, 0])
        assert abs(K @ g @ K) < 1e-14
        assert np.isclose(K @ g @ u, 1.0, rtol=1e-14)   # past-directed: -k.u = K.u = 1
        assert K[0] < 0 and K[1] < 0


def _constants(a, st):
    out = []
    for row in st:
        g = ora_metric(a, row[1], row[2])
        K = row[4:8]
        Kl = g @ K
        th = row[2]
        Q = Kl[2] ** 2 + np.cos(th) ** 2 * (Kl[3] ** 2 / np.sin(th) ** 2 - a * a * Kl[0] ** 2)
        out.append(((K @ g @ K) / K[0] ** 2, -Kl[0], Kl[3], Q))
    return np.array(out)


ora_metric = None


@pytest.mark.parametrize("px,py", [(3.0, 2.0), (-8.0, 5.0), (12.0, -11.0), (6.5, 0.3)])
def test_constants_of_motion_conserved_and_converge(ora, synth, px, py):
    global ora_metric
    ora_metric = ora.metric
    drifts = []
    for eps in (0.05, 0.025):
        cam = ora.camera(synth.Camera(incl_deg=60.0), eps=eps)
        st, status = ora.trace_geodesic(cam, px, py)
        assert status in (ora.HORIZON, ora.ESCAPE)
        c = _constants(cam.a, st)
        scale = np.array([1.0, abs(c[0, 1]), max(abs(c[0, 2]), 1.0), max(abs(c[0, 3]), 1.0)])
        d = np.max(np.abs(c - c[0]) / scale, axis=0)
        drifts.append(d)
    assert np.all(drifts[0] < 2e-5), drifts[0]
    ratio = drifts[0][1:] / np.maximum(drifts[1][1:], 1e-300)
    # fourth-order RK: halving eps shrinks the drift ~16x (allow a broad band)
    assert np.all((ratio > 6.0) | (drifts[0][1:] < 1e-12)), ratio


def _edge(ora, cam, px_of, py_of, lo=1.0, hi=10.0, it=40):
    for _ in range(it):
        mid = 0.5 * (lo + hi)
        _, s = ora.trace_geodesic(cam, px_of(mid), py_of(mid))
        if s == ora.HORIZON:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def test_schwarzschild_shadow_radius(ora, synth):
    """Synge: a static observer at r_o sees the shadow at sin(psi) = (3 sqrt3 / r_o) sqrt(1 - 2/r_o);
    on the pinhole image plane x = r_o tan(psi) = 5.191024 M at r_o = 1000."""
    r_o = 1000.0
    target = r_o * np.tan(np.arcsin(3 * np.sqrt(3) / r_o * np.sqrt(1 - 2 / r_o)))
    cam = ora.camera(synth.Camera(a=0.0, incl_deg=60.0, r_cam=r_o), eps=0.025)
    for ang in (0.0, 1.1, 1.5, 2.6, -0.8):
        e = _edge(ora, cam, lambda m: m * np.cos(ang), lambda m: m * np.sin(ang))
        assert abs(e - target) < 2e-5, (ang, e, target)
    # x = 0 exactly: the ray runs through the polar axis, crossed with the floored step
    e = _edge(ora, cam, lambda m: 0.0, lambda m: m)
    assert abs(e - target) < 2e-4, (e, target)


def bardeen_curve(a, incl_deg, n=400001):
    i = np.radians(incl_deg)
    r1 = 2 * (1 + np.cos(2 / 3 * np.arccos(-a)))
    r2 = 2 * (1 + np.cos(2 / 3 * np.arccos(a)))
    rs = np.linspace(r1, r2, n)[1:-1]
    xi = -(rs ** 3 - 3 * rs ** 2 + a * a * rs + a * a) / (a * (rs - 1))
    eta = rs ** 3 * (4 * a * a - rs * (rs - 3) ** 2) / (a * a * (rs - 1) ** 2)
    b2 = eta + a * a * np.cos(i) ** 2 - xi ** 2 / np.tan(i) ** 2
    ok = b2 >= 0
    al, be = -xi[ok] / np.sin(i), np.sqrt(b2[ok])
    return np.concatenate([al, al[::-1]]), np.concatenate([be, -be[::-1]])


@pytest.mark.parametrize("incl", [60.0, 20.0])
def test_kerr_critical_curve_matches_bardeen(ora, synth, incl):
    """Bardeen (1973): spherical photon orbits give the shadow edge (alpha, beta). A camera at
    r_o = 1e4 M matches the closed form to O(M / r_o)."""
    al, be = bardeen_curve(A, incl)
    ang_b, rad_b = np.arctan2(be, al), np.hypot(al, be)
    cam = ora.camera(synth.Camera(a=A, incl_deg=incl, r_cam=1.0e4), eps=0.025)
    for ang in (0.0, 0.7, np.pi / 2, 2.2, np.pi, -1.3):
        e = _edge(ora, cam, lambda m: m * np.cos(ang), lambda m: m * np.sin(ang))
        k = np.argmin(np.abs(np.angle(np.exp(1j * (ang_b - ang)))))
        assert abs(e - rad_b[k]) < 2.5e-3 * rad_b[k], (ang, e, rad_b[k])


def test_axis_crossing_ray_is_reflected_and_conserves(ora, synth):
    """x = 0 at a = 0 is an exactly meridional ray: it must cross the pole (reflection flag)
    and keep E and Q."""
    global ora_metric
    ora_metric = ora.metric
    cam = ora.camera(synth.Camera(a=0.0, incl_deg=60.0))
    st, status = ora.trace_geodesic(cam, 0.0, 6.0)
    assert status == ora.ESCAPE
    assert (st[:, 8] < 0).sum() >= 1
    c = _constants(0.0, st[:-1])
    assert np.max(np.abs(c[:, 1] - c[0, 1])) < 1e-6 * abs(c[0, 1])


def test_step_count_and_status_mix(ora, synth):
    cam = ora.camera(synth.Camera(incl_deg=60.0, nx=16, ny=16))
    st, s = ora.trace_geodesic(cam, 0.0, 0.0)
    assert s == ora.HORIZON and 100 < len(st) < 400
    assert st[-1, 1] < 1.05 * (1 + np.sqrt(1 - cam.a ** 2))
    st, s = ora.trace_geodesic(cam, 19.0, 0.0)
    assert s == ora.ESCAPE and st[-1, 1] > cam.r_cam and st[-1, 5] > 0
