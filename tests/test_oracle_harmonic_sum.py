"""The oracle's synchrotron emissivities against the exact emissivity of gyrating electrons,
summed over cyclotron harmonics.

The oracle's quadrature (oracle/kappa.c) and the thermal fits it shares with the CUDA path
both rest on the ultrarelativistic synchrotron kernels, and the quadrature's circular kernel
(x K_1/3 + int K_1/3, with its factor 4/3 cot(theta) / gamma) was chosen to agree with the
fits. Neither check is independent of that choice. The harmonic series does not use it: for
one electron of Lorentz factor gamma and pitch angle xi in a field B, the power emitted at
frequency nu into the direction at angle theta to B is, per unit solid angle and frequency,

    (2 pi e^2 nu^2 / c) sum_{n >= 1} K_S delta(n nu_B / gamma - nu (1 - beta cos xi cos theta)),
    K_I = M^2 J_n^2 + N^2 J_n'^2,  K_Q = M^2 J_n^2 - N^2 J_n'^2,  K_V = 2 M N J_n J_n',
    M = (cos theta - beta cos xi) / sin theta,  N = beta sin xi,
    z = (nu / nu_B) gamma beta sin theta sin xi  (the argument of J_n),

with nu_B = e B / (2 pi m c) (the Schott series; Westfold 1959, and Leung, Gammie & Noble
2011 for this form). The M term is the field component along the sky projection of B, the N
term the one across it, so the sum's Q is the oracle's -Q (the oracle counts Q across the
field). V is positive for the sense in which the electrons gyrate when B points toward the
observer: at the fundamental (n = 1, beta -> 0) J_1 and J_1' are positive and so is M for
theta < pi/2.

For an isotropic distribution N(gamma) per d gamma the delta function fixes cos xi for each
harmonic, with weight 1 / (nu beta |cos theta|), and the solid angle of the momenta gives a
factor 1/2. The sum is exact for any gamma; the kernels are its leading order in 1/gamma.
So at Theta_e = 10 the two agree to a few per cent, and at Theta_e = 30 about ten times
closer. A dropped or wrong factor in the circular kernel (the 4/3, the cot, the 1/gamma) or
a flipped sign fails.
"""
import math

import numpy as np
import pytest

scipy = pytest.importorskip("scipy")
from scipy import integrate, special  # noqa: E402

E, ME, C = 4.80320471257e-10, 9.1093837015e-28, 2.99792458e10
NE, BFIELD = 1.0e6, 30.0
NU_B = E * BFIELD / (2 * math.pi * ME * C)


def harmonic_sum(dist, nu, th, gamma_max, panels=6, nodes=12):
    """(j_I, j_Q, j_V) of the electrons dist(gamma) per d gamma by the harmonic series,
    Gauss-Legendre over gamma on panels equal in ln(gamma)."""
    ct, st = math.cos(th), math.sin(th)
    X = nu / NU_B
    xg, wg = np.polynomial.legendre.leggauss(nodes)
    edges = np.geomspace(1.0 + 1e-6, gamma_max, panels + 1)
    acc = np.zeros(3)
    for a, b in zip(edges[:-1], edges[1:]):
        for g, w in zip(0.5 * (b - a) * xg + 0.5 * (b + a), 0.5 * (b - a) * wg):
            beta = math.sqrt(1.0 - 1.0 / (g * g))
            # harmonics whose resonance has |cos xi| < 1
            n_lo = max(1, math.floor(g * X * (1.0 - beta * abs(ct))))
            n_hi = math.ceil(g * X * (1.0 + beta * abs(ct)))
            n = np.arange(n_lo, n_hi + 1, dtype=np.float64)
            cx = (1.0 - n / (g * X)) / (beta * ct)
            keep = np.abs(cx) < 1.0
            n, cx = n[keep], cx[keep]
            sx = np.sqrt(1.0 - cx * cx)
            z = X * g * beta * st * sx
            Jn, Jp = special.jv(n, z), special.jvp(n, z)
            M, N = (ct - beta * cx) / st, beta * sx
            K = np.array([(M * M * Jn * Jn + N * N * Jp * Jp).sum(),
                          (M * M * Jn * Jn - N * N * Jp * Jp).sum(),
                          (2.0 * M * N * Jn * Jp).sum()])
            acc += w * 0.5 * dist(g) * K / (nu * beta * abs(ct))
    return 2.0 * math.pi * E * E * nu * nu / C * acc


def maxwell_juttner(Te):
    k2 = special.kn(2, 1.0 / Te)
    return lambda g: NE * g * math.sqrt(g * g - 1.0) * math.exp(-g / Te) / (Te * k2)


def kappa_dist(Te, kap):
    kw = (kap - 3.0) * Te  # kappa w, w = (kappa - 3) Theta_e / kappa
    shape = lambda g: g * math.sqrt(g * g - 1.0) * (1.0 + (g - 1.0) / kw) ** (-(kap + 1.0))
    Z = integrate.quad(shape, 1.0, np.inf, limit=400, epsrel=1e-12)[0]
    return lambda g: NE * shape(g) / Z


def nu_at(Te, th):
    """nu = nu_s = (2/9) nu_B Theta_e^2 sin(theta): the frequency the thermal fits are scaled to."""
    return (2.0 / 9.0) * NU_B * Te * Te * math.sin(th)


def rel_gap(ora_coeffs, exact):
    """oracle / exact - 1 for (j_I, j_Q, j_V), with the sum's Q turned to the oracle's axis."""
    return ora_coeffs[:3] / (exact * np.array([1.0, -1.0, 1.0])) - 1.0


@pytest.mark.parametrize("th", [0.6, 1.0])
def test_thermal_emission_against_harmonic_sum(ora, th):
    Te = 10.0
    nu = nu_at(Te, th)
    exact = harmonic_sum(maxwell_juttner(Te), nu, th, 40.0 * Te)
    quad = rel_gap(ora.kappa_coeffs(NE, Te, BFIELD, nu, th, 0.0), exact)
    fit = rel_gap(ora.thermal_coeffs(NE, Te, BFIELD, nu, th), exact)
    assert np.abs(quad).max() < 0.025, quad
    assert np.abs(fit).max() < 0.03, fit


@pytest.mark.parametrize("th", [0.6, 1.0])
def test_kappa_emission_against_harmonic_sum(ora, th):
    Te, kap = 10.0, 4.0
    nu = nu_at(Te, th)
    exact = harmonic_sum(kappa_dist(Te, kap), nu, th, 40.0 * Te)
    quad = rel_gap(ora.kappa_coeffs(NE, Te, BFIELD, nu, th, kap), exact)
    assert np.abs(quad).max() < 0.035, quad


def test_gap_closes_as_gamma_grows(ora):
    """The kernels are the series' leading order in 1/gamma: from Theta_e = 10 to 30 the gap
    falls by about 1/Theta_e^2, for both distributions and every Stokes component."""
    th = 1.0
    for kap in (0.0, 4.0):
        gaps = []
        for Te in (10.0, 30.0):
            dist = maxwell_juttner(Te) if kap == 0.0 else kappa_dist(Te, kap)
            nu = nu_at(Te, th)
            exact = harmonic_sum(dist, nu, th, 40.0 * Te)
            gaps.append(np.abs(rel_gap(ora.kappa_coeffs(NE, Te, BFIELD, nu, th, kap), exact)))
            if kap == 0.0 and Te == 30.0:
                fit = rel_gap(ora.thermal_coeffs(NE, Te, BFIELD, nu, th), exact)
                assert np.abs(fit).max() < 0.01, fit
        assert gaps[1].max() < 0.005, (kap, gaps)
        assert (gaps[1] * 4.0 < gaps[0]).all(), (kap, gaps)
