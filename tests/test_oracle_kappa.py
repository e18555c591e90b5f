"""Pins of the oracle's kappa-distribution quadrature (oracle/kappa.c).

- the synchrotron kernels F, G, H against scipy's Bessel functions;
- Maxwell-Juttner electrons through the same quadrature: the rotativity kernels reproduce the
  Bessel ratios K0/K2 and K1/K2 + 6 Theta exactly, and emission/absorption agree with the
  thermal fits within their accuracy (the fits approximate the same integrals);
- kappa -> infinity tends to Maxwell-Juttner at rate 1/kappa;
- far above the knee the kappa tail is a power law N0 g^-p with p = kappa - 1, and the
  coefficients tend to the closed forms of Rybicki & Lightman (6.36, 6.38, 6.53);
- the light cone and the parity of the circular terms in cos(theta).
"""
import math
import warnings

import numpy as np
import pytest

scipy = pytest.importorskip("scipy")
from scipy import integrate, special  # noqa: E402

E, ME, C = 4.80320471257e-10, 9.1093837015e-28, 2.99792458e10


def kint(nu, x):
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        return integrate.quad(lambda t: special.kv(nu, t), x, x + 800.0, limit=800, epsabs=0, epsrel=1e-13)[0]


@pytest.mark.parametrize("x", [1e-4, 1e-2, 0.3, 1.0, 4.0, 20.0, 100.0, 300.0, 600.0])
def test_synchrotron_kernels_match_bessel_functions(ora, x):
    F, G, H = ora.synch_kernels(x)
    # int_x K_5/3 = 2 K_2/3(x) - int_x K_1/3 (from K_5/3 = -2 K'_2/3 - K_1/3)
    Fr = x * (2.0 * special.kv(2 / 3, x) - kint(1 / 3, x))
    Gr = x * special.kv(2 / 3, x)
    Hr = x * special.kv(1 / 3, x) + kint(1 / 3, x)
    for a, b in ((F, Fr), (G, Gr), (H, Hr)):
        assert abs(a / b - 1) < 1e-11, (x, a, b)
    assert G < F  # the linear polarization of one electron is below 100%


def test_maxwell_juttner_rotativity_kernels_are_exact(ora):
    for Te in (0.05, 0.5, 3.0, 30.0):
        for th in (0.3, 1.1):
            q = ora.kappa_coeffs(1e6, Te, 30.0, 230e9, th, 0.0)
            f = ora.thermal_coeffs(1e6, Te, 30.0, 230e9, th)
            assert abs(q[6] / f[6] - 1) < 1e-9 and abs(q[7] / f[7] - 1) < 1e-9, (Te, th, q[6:], f[6:])


@pytest.mark.parametrize("Te", [10.0, 40.0])
@pytest.mark.parametrize("th", [0.4, 1.0, 1.45])
def test_maxwell_juttner_emission_matches_thermal_fits(ora, Te, th):
    nuB = E * 30.0 / (2 * math.pi * ME * C)
    for x in (0.3, 3.0, 30.0, 300.0):
        nu = x * 1.5 * nuB * math.sin(th) * Te * Te
        q = ora.kappa_coeffs(1e6, Te, 30.0, nu, th, 0.0)
        f = ora.thermal_coeffs(1e6, Te, 30.0, nu, th)
        # j_I, j_Q, j_V and absorption (Kirchhoff) within the fits' percent-level accuracy
        for k in (0, 1, 2, 3, 4, 5):
            assert abs(q[k] / f[k] - 1) < 0.02, (Te, th, x, k, q[k] / f[k])


def test_kappa_tends_to_maxwell_juttner(ora):
    mj = ora.kappa_coeffs(1e6, 10.0, 30.0, 230e9, 0.9, 0.0)
    e3 = np.abs(ora.kappa_coeffs(1e6, 10.0, 30.0, 230e9, 0.9, 1e3) / mj - 1).max()
    e4 = np.abs(ora.kappa_coeffs(1e6, 10.0, 30.0, 230e9, 0.9, 1e4) / mj - 1).max()
    assert e4 < 3e-4 and 5.0 < e3 / e4 < 20.0, (e3, e4)


def test_power_law_tail_closed_forms(ora):
    """kappa = 4, Theta = 10 (knee kappa w = 10): at X = 1e10 the emission comes from g ~ 1e5,
    where N = N0 g^-3 (1 + O(kappa w / g))."""
    kap, Te, B, th, ne = 4.0, 10.0, 30.0, 1.0, 1e6
    w = (kap - 3) * Te / kap
    kw = kap * w
    p = kap - 1.0
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        # normalisation int g sqrt(g^2-1) (1 + (g-1)/kw)^-(kappa+1) dg, with g - 1 = kw (e^v - 1)
        f = lambda v: ((1 + kw * math.expm1(v)) * math.sqrt(kw * math.expm1(v) * (2 + kw * math.expm1(v)))
                       * math.exp(-(kap + 1) * v) * kw * math.exp(v))
        Cn = 1.0 / integrate.quad(f, 0.0, 200.0, limit=500)[0]
    N0 = ne * Cn * kw ** (kap + 1)
    nuB = E * B / (2 * math.pi * ME * C)
    nu = 1e10 * 1.5 * nuB * math.sin(th)
    q = ora.kappa_coeffs(ne, Te, B, nu, th, kap)
    s = math.sin(th)
    jI = (math.sqrt(3) * E ** 3 * N0 * B * s / (4 * math.pi * ME * C * C * (p + 1)) * special.gamma(p / 4 + 19 / 12)
          * special.gamma(p / 4 - 1 / 12) * (2 * math.pi * ME * C * nu / (3 * E * B * s)) ** (-(p - 1) / 2))
    assert abs(q[0] / jI - 1) < 2e-3, q[0] / jI
    assert abs(q[1] / q[0] - (p + 1) / (p + 7 / 3)) < 2e-3, q[1] / q[0]
    # Rybicki & Lightman 6.53 with N(E) dE = C_E E^-p dE, C_E = N0 (m c^2)^(p-1)
    CE = N0 * (ME * C * C) ** (p - 1)
    aI = (math.sqrt(3) * E ** 3 / (8 * math.pi * ME) * (3 * E / (2 * math.pi * ME ** 3 * C ** 5)) ** (p / 2) * CE
          * (B * s) ** ((p + 2) / 2) * special.gamma((3 * p + 2) / 12) * special.gamma((3 * p + 22) / 12)
          * nu ** (-(p + 4) / 2))
    assert abs(q[3] / aI - 1) < 2e-3, q[3] / aI


def test_light_cone_and_circular_parity(ora):
    rng = np.random.default_rng(11)
    for _ in range(12):
        Te = 10 ** rng.uniform(0, 2)
        kap = rng.uniform(3.5, 8.0)
        th = rng.uniform(0.2, 1.4)
        nu = 10 ** rng.uniform(10.5, 12)
        a = ora.kappa_coeffs(1e6, Te, 30.0, nu, th, kap)
        b = ora.kappa_coeffs(1e6, Te, 30.0, nu, math.pi - th, kap)
        assert a[0] > 0 and a[3] > 0
        assert math.hypot(a[1], a[2]) <= a[0] * (1 + 1e-12)
        assert math.hypot(a[4], a[5]) <= a[3] * (1 + 1e-12)
        # theta -> pi - theta flips the circular terms and keeps the rest
        sign = np.array([1, 1, -1, 1, 1, -1, 1, -1])
        assert np.allclose(b, sign * a, rtol=1e-9, atol=0), (a, b)


def _kappa_average(kernel, Te, kappa):
    """<kernel(g)> over the kappa distribution N ~ g p (1 + (g - 1)/(kappa w))^-(kappa+1),
    w = (kappa - 3) Theta / kappa, by scipy's adaptive quadrature over s = ln p on fixed
    breakpoints (not the oracle's Gauss-Legendre rule); the heaviest tail, kappa = 3.5 with the
    kernel 2 g, falls only as e^(-s/2), so the range runs to s = 90."""
    kw = (kappa - 3.0) * Te

    def weight(s):
        p = math.exp(s)
        g = math.sqrt(1.0 + p * p)
        return g * p * (1.0 + p * p / (g + 1.0) / kw) ** -(kappa + 1.0) * p * p / g, g, p

    def num_f(s):
        w, g, p = weight(s)
        return w * kernel(g, p)

    pts = [-14.0, -4.0, -1.0, 0.0, 1.0, 2.0, 3.0, 4.0, 6.0, 8.0, 11.0, 15.0, 20.0, 30.0, 45.0, 60.0, 90.0]
    num = den = 0.0
    for a, b in zip(pts, pts[1:]):
        num += integrate.quad(num_f, a, b, limit=200, epsabs=0, epsrel=1e-13)[0]
        den += integrate.quad(lambda s: weight(s)[0], a, b, limit=200, epsabs=0, epsrel=1e-13)[0]
    return num / den


@pytest.mark.parametrize("kappa", [3.5, 4.5, 8.0])
@pytest.mark.parametrize("Te", [0.3, 3.0, 30.0])
def test_kappa_rotativities_are_the_distribution_averages(ora, kappa, Te):
    """The kappa rotativities are the thermal ones with the Bessel ratios K0/K2 and
    K1/K2 + 6 Theta replaced by the averages of asinh(p)/(g p) and 2 g - 1/g over the kappa
    distribution (the same Shcherbakov corrections at the same X multiply both, so they cancel
    in the ratio). The averages are taken here by an independent quadrature; a wrong w, a wrong
    normalisation or a wrong kernel in the oracle's rule would show."""
    th, nu = 0.9, 230e9
    q = ora.kappa_coeffs(1e6, Te, 30.0, nu, th, kappa)
    f = ora.thermal_coeffs(1e6, Te, 30.0, nu, th)
    z = 1.0 / Te
    k0, k1, k2 = special.kve(0, z), special.kve(1, z), special.kve(2, z)
    aV = _kappa_average(lambda g, p: math.asinh(p) / (g * p), Te, kappa)
    aQ = _kappa_average(lambda g, p: 2.0 * g - 1.0 / g, Te, kappa)
    assert abs((q[7] / f[7]) / (aV / (k0 / k2)) - 1) < 1e-8, (q[7] / f[7], aV / (k0 / k2))
    assert abs((q[6] / f[6]) / (aQ / (k1 / k2 + 6.0 * Te)) - 1) < 1e-8, (q[6] / f[6], aQ / (k1 / k2 + 6.0 * Te))


def test_kappa_mean_energy_closed_form(ora):
    """Ultrarelativistic kappa electrons have <g> = kappa w 3/(kappa - 3) = 3 Theta (Beta-function
    integrals of g^2 (1 + g/(kappa w))^-(kappa+1)), so the Faraday-conversion average
    <2 g - 1/g> tends to 6 Theta, as for thermal electrons (up to terms of order 1/Theta)."""
    for kappa in (4.0, 6.0):
        Te = 3000.0
        q = ora.kappa_coeffs(1e6, Te, 30.0, 230e9, 0.9, kappa)
        f = ora.thermal_coeffs(1e6, Te, 30.0, 230e9, 0.9)
        z = 1.0 / Te
        ratio_mj = special.kve(1, z) / special.kve(2, z) + 6.0 * Te
        avg = (q[6] / f[6]) * ratio_mj
        assert abs(avg / (6.0 * Te) - 1) < 1e-3, (kappa, avg / (6 * Te))
