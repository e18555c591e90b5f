"""The FP64 reference of the surrogate network (oracle/mlp.py): its hand-written backward pass
against central finite differences of its loss (the reference the GPU gradients are checked against),
and its target variables against the thermal fits they are built from."""
import math

import numpy as np

import oracle.mlp as M


def test_backward_matches_central_differences():
    rng = np.random.default_rng(3)
    theta = rng.normal(0.0, 0.3, M.NPARAM)
    x = rng.uniform(-1, 1, (96, 4))
    t = rng.normal(0, 1, (96, 8))
    loss, g = M.loss_and_grad(theta, x, t)
    assert loss > 0 and g.shape == (M.NPARAM,)
    # every layer's weights and biases
    idx = np.concatenate([rng.integers(a, b, 12) for a, b in ((0, 320), (320, 4480), (4480, 8640), (8640, 9160))])
    fd = M.finite_difference(theta, x, t, idx)
    assert np.abs(fd - g[idx]).max() <= 1e-6 * np.abs(g[idx]).max() + 1e-12


def test_targets_of_thermal_coefficients(ora):
    """For Maxwell-Juttner electrons the thermal fits are exactly the targets' prefactors times
    the fit functions, so the targets of ora.thermal_coeffs are those functions' logarithms."""
    ne, Te, B, th = 1e5, 20.0, 10.0, 0.8
    nuB = M.E * B / (2 * math.pi * M.ME * M.C)
    x = 5.0
    nu = x * 1.5 * nuB * math.sin(th) * Te * Te
    y = M.targets(ora.thermal_coeffs(ne, Te, B, nu, th), ne, Te, B, nu, th)
    x13 = x ** (1 / 3)
    ex = math.exp(-1.8899 * x13)
    iI = 2.5651 * (1 + 1.92 / x13 + 0.9977 / x13 ** 2) * ex
    iV = (1.81348 / x + 3.42319 / x13 ** 2 + 0.0292545 / math.sqrt(x) + 2.03773 / x13) * ex
    assert abs(y[0] - math.log(iI)) < 1e-12 and abs(y[2] - math.log(iV)) < 1e-12
    # rotativities: the Bessel ratios K1/K2 + 6 Theta and K0/K2
    k0, k1, k2 = (ora.bessel_k_scaled(n, 1 / Te) for n in (0, 1, 2))
    assert abs(y[6] - math.log(k1 / k2 + 6 * Te)) < 1e-9 and abs(y[7] - math.log(k0 / k2)) < 1e-9
