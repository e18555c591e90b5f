"""Pins of the oracle's thermal synchrotron coefficients.

* e^z K_n(z) against scipy.special.kve;
* j_I and j_Q against a direct quadrature of the ultra-relativistic single-electron spectra,
  F(y) = y int_y^inf K_5/3 and G(y) = y K_2/3(y), over the Maxwell-Juttner distribution;
* Kirchhoff's law against an independent Planck function;
* the cold-plasma limits of the rotativities against the textbook rotation measure and
  conversion rates;
* parity in cos(theta_B) and the light-cone bound |j_P| <= j_I.
"""
import numpy as np
import pytest
from scipy import integrate, special

ME, C, QE, H, KB = 9.1093837015e-28, 2.99792458e10, 4.80320471257e-10, 6.62607015e-27, 1.380649e-16


@pytest.mark.parametrize("n", [0, 1, 2])
def test_scaled_bessel_k(ora, n):
    for z in np.logspace(-4, 4, 33):
        assert np.isclose(ora.bessel_k_scaled(n, z), special.kve(n, z), rtol=2e-13)


def _ultrarel(x, kind):
    """(1/x) int_0^inf u^2 e^{-u} S(x/u^2) du with S = F or G."""
    def S(y):
        if kind == "I":
            return y * integrate.quad(lambda t: special.kv(5.0 / 3.0, t), y, np.inf, limit=200)[0]
        return y * special.kv(2.0 / 3.0, y)
    u0 = (2 * x) ** (1.0 / 3.0)
    f = lambda u: u * u * np.exp(-u) * S(x / (u * u))
    val = integrate.quad(f, 0.0, u0, limit=200)[0] + integrate.quad(f, u0, np.inf, limit=200)[0]
    return val / x


@pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")
@pytest.mark.parametrize("x", [1.0, 10.0, 100.0, 1000.0])
def test_emissivity_fits_against_quadrature(ora, x):
    """j_I = n e^2 nu / (2 sqrt3 c Theta^2) I(x), with nu_c = (3/2) nu_B sin(th) Theta^2;
    the published fits are accurate to a few per cent over this range."""
    ne, Te, B, th = 1.0e6, 20.0, 30.0, 1.0
    nuB = QE * B / (2 * np.pi * ME * C)
    nu = x * 1.5 * nuB * np.sin(th) * Te * Te
    c = ora.thermal_coeffs(ne, Te, B, nu, th)
    pre = ne * QE * QE * nu / (2 * np.sqrt(3) * C * Te * Te)
    jI_ref = pre * _ultrarel(x, "I")
    jQ_ref = pre * _ultrarel(x, "Q")
    assert abs(c[0] / jI_ref - 1) < 0.05, (c[0], jI_ref)
    assert abs(c[1] / jQ_ref - 1) < 0.06, (c[1], jQ_ref)


def test_kirchhoff(ora):
    ne, Te, B, nu, th = 3.0e5, 8.0, 12.0, 2.3e11, 0.8
    c = ora.thermal_coeffs(ne, Te, B, nu, th)
    T = Te * ME * C * C / KB
    Bnu = 2 * H * nu ** 3 / C ** 2 / np.expm1(H * nu / (KB * T))
    assert np.allclose(c[3:6] * Bnu, c[0:3], rtol=1e-10)


def test_cold_plasma_rotativities(ora):
    """Theta_e -> 0 at high frequency: rho_V -> n e^3 B cos/(pi m^2 c^2 nu^2) (rotation measure)
    and rho_Q -> n e^2 nu_B^2 sin^2 / (m c nu^3) = w_p^2 w_B^2 sin^2/(2 c w^3)."""
    ne, Te, B, nu, th = 1.0e5, 1e-5, 10.0, 1.0e13, 0.6
    c = ora.thermal_coeffs(ne, Te, B, nu, th)
    rv = ne * QE ** 3 * B * np.cos(th) / (np.pi * ME ** 2 * C ** 2 * nu ** 2)
    wp2 = 4 * np.pi * ne * QE ** 2 / ME
    wB = QE * B / (ME * C)
    rq = wp2 * wB ** 2 * np.sin(th) ** 2 / (2 * C * (2 * np.pi * nu) ** 3)
    assert np.isclose(c[7], rv, rtol=1e-4)
    assert np.isclose(c[6], rq, rtol=1e-4)
    assert c[0] == 0.0  # no emission from a cold plasma at this frequency


def test_hot_plasma_faraday_suppression(ora):
    """Relativistic electrons rotate less: rho_V / rho_V(cold) -> ln(Theta)/(2 Theta^2) order."""
    ne, B, nu, th = 1.0e5, 10.0, 1.0e14, 0.6
    cold = ora.thermal_coeffs(ne, 1e-5, B, nu, th)[7]
    for Te in (10.0, 100.0):
        hot = ora.thermal_coeffs(ne, Te, B, nu, th)[7]
        r = hot / cold
        assert 0.5 * np.log(2 * Te) / (2 * Te * Te) < r < 1.5 * np.log(2 * Te) / (2 * Te * Te)


def test_parity_in_cos_theta(ora):
    ne, Te, B, nu = 1e6, 15.0, 20.0, 2.3e11
    for th in (0.3, 0.9, 1.3):
        a = ora.thermal_coeffs(ne, Te, B, nu, th)
        b = ora.thermal_coeffs(ne, Te, B, nu, np.pi - th)
        even = [0, 1, 3, 4, 6]
        odd = [2, 5, 7]
        assert np.allclose(a[even], b[even], rtol=1e-12)
        assert np.allclose(a[odd], -b[odd], rtol=1e-12)
        assert a[2] > 0 and a[7] > 0   # circular terms carry the sign of cos(theta_B)


def test_light_cone_bound(ora):
    rng = np.random.default_rng(7)
    for _ in range(400):
        ne = 10 ** rng.uniform(2, 9)
        Te = 10 ** rng.uniform(-2, 2.5)
        B = 10 ** rng.uniform(-2, 3)
        nu = 10 ** rng.uniform(9, 13)
        th = rng.uniform(1e-4, np.pi - 1e-4)
        c = ora.thermal_coeffs(ne, Te, B, nu, th)
        assert c[0] >= 0 and c[3] >= 0
        if c[0] > 0:
            assert np.hypot(c[1] / c[0], c[2] / c[0]) <= 1 + 1e-12
            assert np.hypot(c[4] / c[3], c[5] / c[3]) <= 1 + 1e-12


def _conversion_factor(ora, Te, nu, th=1.0, ne=1e5, B=100.0):
    """rho_Q / (rho_Q of cold electrons x (K1/K2 + 6 Theta)): the oracle's Shcherbakov factor
    f(X) read through the whole coefficient, with the cold-plasma rate written as
    w_p^2 w_B^2 sin^2 / (2 c w^3) and the Bessel ratio from scipy."""
    c = ora.thermal_coeffs(ne, Te, B, nu, th)
    wp2 = 4 * np.pi * ne * QE ** 2 / ME
    wB = QE * B / (ME * C)
    rq = wp2 * wB ** 2 * np.sin(th) ** 2 / (2 * C * (2 * np.pi * nu) ** 3)
    z = 1.0 / Te
    X = Te * np.sqrt(np.sqrt(2.0) * np.sin(th) * 1e3 * (QE * B / (2 * np.pi * ME * C)) / nu)
    return c[6] / (rq * (special.kve(1, z) / special.kve(2, z) + 6 * Te)), X


def test_conversion_correction_large_X_asymptote(ora):
    """Far above the switch at X = 120 the published correction falls as
    -2^(-1/3) 3^(-23/6) 1e4 pi X^(-8/3): the exponential terms have died, the two 0.011 e^(-X/47.2)
    terms cancel and the tanh switch is fully on. A wrong sign in the switch, a dropped
    cancellation or a wrong power would show here."""
    C83 = 2.0 ** (-1.0 / 3.0) * 3.0 ** (-23.0 / 6.0) * 1e4 * np.pi
    for X_target in (1e3, 4e3, 2e4):
        Te = 50.0
        nuB = QE * 100.0 / (2 * np.pi * ME * C)
        nu = np.sqrt(2.0) * np.sin(1.0) * 1e3 * nuB * (Te / X_target) ** 2
        f, X = _conversion_factor(ora, Te, nu)
        assert abs(X / X_target - 1) < 1e-12
        assert abs(f / (-C83 * X ** (-8.0 / 3.0)) - 1) < 1e-9, (X, f, -C83 * X ** (-8.0 / 3.0))


def test_conversion_correction_small_X_and_switch(ora):
    """f -> 1 as X -> 0 (the high-frequency limit that the cold-plasma pin fixes at finite
    temperature), and f is continuous through the switch around X = 120 (no step larger than the
    fit's own variation over the grid)."""
    Te = 50.0
    nuB = QE * 100.0 / (2 * np.pi * ME * C)
    f0, X0 = _conversion_factor(ora, Te, np.sqrt(2.0) * np.sin(1.0) * 1e3 * nuB * (Te / 1e-6) ** 2)
    assert X0 < 2e-6 and abs(f0 - 1) < 1e-5
    xs = np.linspace(60.0, 240.0, 721)
    fs = np.array([_conversion_factor(ora, Te, np.sqrt(2.0) * np.sin(1.0) * 1e3 * nuB * (Te / x) ** 2)[0] for x in xs])
    d = np.abs(np.diff(fs))
    assert d.max() < 10 * np.median(d), (d.max(), np.median(d))
