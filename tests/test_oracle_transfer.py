"""Pins of the oracle's radiative transfer: the constant-coefficient substep, the tetrad and
whole-image properties.

The substep is checked against scipy's matrix exponential (a library routine the oracle
does not use), closed forms for pure rotation, conversion, dichroism and absorption, the
semigroup property and a brute-force ODE solve. Images are checked for I >= |P|, mirror
symmetry and convergence in the step parameter.
"""
import numpy as np
import pytest
from scipy import integrate, linalg

RNG = np.random.default_rng(12345)


def mueller(c):
    jI, jQ, jU, jV, aI, aQ, aU, aV, rQ, rU, rV = c
    M = np.array([[aI, aQ, aU, aV], [aQ, aI, rV, -rU], [aU, -rV, aI, rQ], [aV, rU, -rQ, aI]])
    return np.array([jI, jQ, jU, jV]), M


def random_coeffs(scale_a, scale_r):
    aI = scale_a * RNG.uniform(0.5, 1.5)
    ap = RNG.normal(size=3)
    ap *= RNG.uniform(0, 0.95) * aI / np.linalg.norm(ap)
    jI = RNG.uniform(0.5, 2.0)
    jp = RNG.normal(size=3)
    jp *= RNG.uniform(0, 0.99) * jI / np.linalg.norm(jp)
    r = RNG.normal(size=3) * scale_r
    return np.array([jI, jp[0], jp[1], jp[2], aI, ap[0], ap[1], ap[2], r[0], r[1], r[2]])


@pytest.mark.parametrize("sa,sr,ds", [(1.0, 1.0, 0.3), (0.01, 5.0, 1.0), (3.0, 0.1, 2.0),
                                      (1e-6, 1e3, 0.7), (50.0, 50.0, 1.0), (0.2, 0.0, 1.0)])
def test_substep_matches_scipy_expm(ora, sa, sr, ds):
    for _ in range(5):
        c = random_coeffs(sa, sr)
        J, M = mueller(c)
        S0 = np.array([1.0, 0.3, -0.2, 0.1])
        G = np.zeros((5, 5))
        G[:4, :4] = -M * ds
        G[:4, 4] = J * ds
        ref = (linalg.expm(G) @ np.append(S0, 1.0))[:4]
        got = ora.substep(c, ds, S0)
        assert np.allclose(got, ref, rtol=0, atol=2e-12 * max(1.0, np.abs(ref).max())), (got, ref)


def test_substep_semigroup_and_brute_force(ora):
    c = random_coeffs(0.8, 2.0)
    S0 = np.array([0.5, 0.1, 0.2, -0.1])
    one = ora.substep(c, 1.0, S0)
    half = ora.substep(c, 0.5, ora.substep(c, 0.5, S0))
    many = S0
    for _ in range(64):
        many = ora.substep(c, 1.0 / 64, many)
    assert np.allclose(one, half, atol=1e-13) and np.allclose(one, many, atol=1e-12)
    J, M = mueller(c)
    sol = integrate.solve_ivp(lambda s, y: J - M @ y, (0.0, 1.0), S0, method="DOP853", rtol=1e-12, atol=1e-14)
    assert np.allclose(one, sol.y[:, -1], atol=1e-10)


def test_pure_faraday_rotation(ora):
    """Only rho_V: (Q, U) turns by rho_V ds, the EVPA by rho_V ds / 2; I and V unchanged."""
    rV, ds = 2.7, 0.9
    c = np.zeros(11)
    c[10] = rV
    S0 = np.array([1.0, 0.6, 0.2, 0.1])
    S1 = ora.substep(c, ds, S0)
    ph = rV * ds
    assert np.isclose(S1[0], 1.0, atol=1e-15) and np.isclose(S1[3], 0.1, atol=1e-15)
    assert np.allclose(S1[1:3], [0.6 * np.cos(ph) - 0.2 * np.sin(ph), 0.6 * np.sin(ph) + 0.2 * np.cos(ph)],
                       atol=1e-14)
    chi0 = 0.5 * np.arctan2(S0[2], S0[1])
    chi1 = 0.5 * np.arctan2(S1[2], S1[1])
    assert np.isclose(np.angle(np.exp(2j * (chi1 - chi0))) / 2, np.angle(np.exp(1j * ph)) / 2, atol=1e-14)


def test_pure_faraday_conversion(ora):
    """Only rho_Q: (U, V) turns by rho_Q ds; I and Q unchanged."""
    rQ, ds = 1.3, 0.8
    c = np.zeros(11)
    c[8] = rQ
    S0 = np.array([1.0, 0.2, 0.5, -0.3])
    S1 = ora.substep(c, ds, S0)
    ph = rQ * ds
    assert np.allclose(S1[:2], S0[:2], atol=1e-15)
    assert np.allclose(S1[2:], [0.5 * np.cos(ph) + 0.3 * np.sin(ph), 0.5 * np.sin(ph) - 0.3 * np.cos(ph)], atol=1e-14)


def test_linear_dichroism_is_a_boost(ora):
    """Only alpha_I, alpha_Q: I' = e^{-aI s}(I cosh(aQ s) - Q sinh(aQ s)), Q' likewise."""
    aI, aQ, ds = 1.1, 0.7, 0.6
    c = np.zeros(11)
    c[4], c[5] = aI, aQ
    S0 = np.array([1.0, 0.4, 0.1, 0.2])
    S1 = ora.substep(c, ds, S0)
    e, ch, sh = np.exp(-aI * ds), np.cosh(aQ * ds), np.sinh(aQ * ds)
    assert np.allclose(S1, [e * (ch - 0.4 * sh), e * (0.4 * ch - sh), e * 0.1, e * 0.2], atol=1e-15)


@pytest.mark.parametrize("tau", [1e-8, 0.3, 5.0, 200.0])
def test_emission_absorption_closed_form(ora, tau):
    j, a, I0 = 2.0, 0.5, 0.7
    c = np.zeros(11)
    c[0], c[4] = j, a
    ds = tau / a
    S1 = ora.substep(c, ds, np.array([I0, 0, 0, 0]))
    ref = I0 * np.exp(-tau) - (j / a) * np.expm1(-tau)
    assert np.isclose(S1[0], ref, rtol=1e-13)


def test_substep_keeps_light_cone(ora):
    for _ in range(200):
        c = random_coeffs(10 ** RNG.uniform(-4, 2), 10 ** RNG.uniform(-3, 3))
        S0 = np.array([1.0, *(RNG.normal(size=3) * 0.3)])
        S0[1:] *= min(1.0, 0.999 / np.linalg.norm(S0[1:]))
        S1 = ora.substep(c, 10 ** RNG.uniform(-3, 1), S0)
        assert S1[0] >= np.linalg.norm(S1[1:]) * (1 - 1e-12)


def test_fluid_tetrad_orthonormal_and_right_handed(ora, synth):
    cam = ora.camera(synth.Camera())
    m = ora.adaf_model(synth.adaf_params(1))
    for (px, py) in [(3.0, 4.0), (-7.0, 1.0)]:
        st, _ = ora.trace_geodesic(cam, px, py)
        for row in st[5:-5:37]:
            pl = ora.plasma(cam, m, row[:4])
            if pl[3] == 0:
                continue
            e, thB = ora.fluid_tetrad(cam.a, row[:4], row[4:8], pl[4:8], pl[8:12])
            g = ora.metric(cam.a, row[1], row[2])
            eta = e @ g @ e.T
            assert np.allclose(eta, np.diag([-1.0, 1, 1, 1]), atol=1e-10)
            # orientation: sqrt(-g) det[e_a^mu] = +1 for a right-handed (e1, e2, e3)
            assert np.isclose(np.sqrt(-np.linalg.det(g)) * np.linalg.det(e), 1.0, atol=1e-9)
            k = -row[4:8]
            w = -(k @ g @ pl[4:8])
            # e3 along the photon direction, up to the integrator's drift of k.k from zero
            assert np.abs(k / w - e[0] - e[3]).max() <= abs(k @ g @ k) / w ** 2 + 1e-12
            b = pl[8:12]
            assert abs(e[1] @ g @ b) < 1e-10 * np.sqrt(b @ g @ b) and e[2] @ g @ b > 0
            assert np.isclose(np.cos(thB), (e[3] @ g @ b) / np.sqrt(b @ g @ b), atol=1e-12)


def test_images_obey_i_ge_p_everywhere(ora, synth, small_grid):
    cam = ora.camera(synth.Camera(incl_deg=60.0, nx=24, ny=24))
    img, ns, st, mp = ora.render_image(cam, ora.adaf_model(synth.adaf_params(1)))
    assert mp.min() >= -1e-12
    assert np.all(img[..., 0] >= np.linalg.norm(img[..., 1:], axis=-1) * (1 - 1e-12))
    prims, g = small_grid
    cam = ora.camera(synth.Camera(incl_deg=20.0, nx=24, ny=24))
    img, ns, st, mp = ora.render_image(cam, ora.grid_model(prims, g))
    assert mp.min() >= -1e-12
    assert np.all(img[..., 0] >= np.linalg.norm(img[..., 1:], axis=-1) * (1 - 1e-12))


def test_edge_on_image_mirror_symmetry(ora, synth):
    """The unperturbed torus is symmetric about the equator with a dipolar poloidal field
    (B^r odd, B^theta even), which is mirror symmetric for the pseudovector B, and so is the
    Kerr metric. Seen edge-on, y -> -y keeps I and Q and flips U and V (a mirror reverses
    handedness)."""
    prims, g = synth.fm_torus_grid(2, grid=synth.GridParams(n1=48, n2=32, n3=8),
                                   torus=synth.TorusParams(sigma_pert=0.0))
    cam = ora.camera(synth.Camera(incl_deg=90.0, nx=10, ny=10, fov_M=30.0))
    img, *_ = ora.render_image(cam, ora.grid_model(prims, g))
    mir = img[::-1]
    scale = np.abs(img[..., 0]).max()
    assert scale > 0
    assert np.allclose(mir[..., 0], img[..., 0], atol=1e-10 * scale)
    assert np.allclose(mir[..., 1], img[..., 1], atol=1e-10 * scale)
    assert np.allclose(mir[..., 2], -img[..., 2], atol=1e-10 * scale)
    assert np.allclose(mir[..., 3], -img[..., 3], atol=1e-10 * scale)
    assert np.abs(img[..., 3]).max() > 1e-4 * scale   # V is not trivially zero


def test_image_converges_in_step_parameter(ora, synth):
    m = ora.adaf_model(synth.adaf_params(1))
    ix = np.array([3, 7, 10, 12, 5, 14])
    iy = np.array([8, 2, 9, 6, 13, 11])
    res = []
    for eps in (0.05, 0.025, 0.0125, 0.00625):
        cam = ora.camera(synth.Camera(incl_deg=60.0, nx=16, ny=16), eps=eps)
        res.append(ora.render_pixels(cam, m, ix, iy)[0][:, 0])
    e1 = np.abs(res[0] - res[3])
    e2 = np.abs(res[1] - res[3])
    e3 = np.abs(res[2] - res[3])
    assert np.all(e1 > e2) and np.all(e2 > e3)
    # first order at least (the coefficients are taken at the arrival point of each step)
    assert np.median(e1 / e2) > 1.8


def test_image_stats_scale_with_distance(ora, synth):
    cam = ora.camera(synth.Camera(incl_deg=60.0, nx=8, ny=8))
    img, *_ = ora.render_image(cam, ora.adaf_model(synth.adaf_params(1)))
    f1, lp, cp = ora.image_stats(cam, img)
    cam2 = ora.camera(synth.Camera(incl_deg=60.0, nx=8, ny=8, dist_cm=2 * cam.dist_cm))
    f2, lp2, cp2 = ora.image_stats(cam2, img)
    assert np.isclose(f1, 4 * f2, rtol=1e-14) and lp == lp2 and cp == cp2
    s = img.reshape(-1, 4).sum(axis=0)
    assert np.isclose(lp, np.hypot(s[1], s[2]) / s[0], rtol=1e-12)
    assert np.isclose(cp, s[3] / s[0], rtol=1e-12)


def test_unpolarized_transfer_equals_polarized_without_polarization(ora, synth):
    """The scalar (Stokes I) transfer against the pinned polarized transfer run with every
    polarized coefficient set to zero. In exact arithmetic an unpolarized coherency stays
    unpolarized and its I obeys the scalar equation; the polarized path's Heun propagator is
    an isometry of the screen only to O(h^3) per step, so the two agree to O(eps^2) and the
    difference must shrink about four-fold when eps halves."""
    diffs = []
    for eps in (0.05, 0.025):
        cam = ora.camera(synth.Camera(incl_deg=60.0, nx=12, ny=12), eps=eps)
        m = ora.adaf_model(synth.adaf_params(1))
        u = ora.render_unpol(cam, m)
        m.st.unpol_test = 1
        img = ora.render_image(cam, m)[0]
        assert u.max() > 0
        scale = np.maximum(img[..., 0], 1e-8 * img[..., 0].max())
        diffs.append((np.abs(u - img[..., 0]) / scale).max())
        # the polarization the transport error creates is of the same order
        assert np.abs(img[..., 1:]).max() <= 2 * diffs[-1] * img[..., 0].max()
    assert diffs[0] < 1e-3 and 2.5 < diffs[0] / diffs[1] < 6.0, diffs
