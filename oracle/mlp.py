"""FP64 reference of the coefficient surrogate (test infrastructure only, like the rest of
this package): the 4 -> 64 -> 64 -> 64 -> 8 SiLU perceptron, its mean-squared-error loss and
gradient by hand-written backpropagation, central finite differences of the loss, and the
surrogate's target variables computed from the quadrature coefficients.

Parameter layout (one vector of 9160 numbers): layer after layer (4 -> 64, 64 -> 64,
64 -> 64, 64 -> 8), each a matrix [out][in + 1] whose last column is the bias.
"""
from __future__ import annotations

import math

import numpy as np

SHAPES = [(64, 4), (64, 64), (64, 64), (8, 64)]
NPARAM = sum(o * (i + 1) for o, i in SHAPES)

E, ME, C = 4.80320471257e-10, 9.1093837015e-28, 2.99792458e10


def unpack(theta):
    out, k = [], 0
    for o, i in SHAPES:
        m = np.asarray(theta[k:k + o * (i + 1)], dtype=np.float64).reshape(o, i + 1)
        out.append((m[:, :i], m[:, i]))
        k += o * (i + 1)
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(theta, x, keep=False):
    """x [n, 4] -> y [n, 8]; with keep=True also the pre-activations and activations."""
    layers = unpack(theta)
    a, zs, acts = np.asarray(x, dtype=np.float64), [], []
    for li, (W, b) in enumerate(layers):
        acts.append(a)
        z = a @ W.T + b
        if li < 3:
            zs.append(z)
            a = silu(z)
        else:
            a = z
    return (a, zs, acts) if keep else a


def loss_and_grad(theta, x, t):
    """loss = sum (y - t)^2 / (8 n) and its gradient in the parameter layout."""
    y, zs, acts = forward(theta, x, keep=True)
    n = x.shape[0]
    d = 2.0 * (y - t) / (8.0 * n)
    loss = float(((y - t) ** 2).sum() / (8.0 * n))
    layers = unpack(theta)
    grads = [None] * 4
    for li in range(3, -1, -1):
        W, _ = layers[li]
        gW = d.T @ acts[li]
        gb = d.sum(axis=0)
        grads[li] = np.concatenate([gW, gb[:, None]], axis=1).ravel()
        if li > 0:
            d = (d @ W) * dsilu(zs[li - 1])
    return loss, np.concatenate(grads)


def finite_difference(theta, x, t, idx, h=1e-6):
    g = []
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        g.append((loss_and_grad(tp, x, t)[0] - loss_and_grad(tm, x, t)[0]) / (2 * h))
    return np.array(g)


def shcherbakov_f(X):
    f = 2.011 * math.exp(-X ** 1.035 / 4.7) - math.cos(0.5 * X) * math.exp(-X ** 1.2 / 2.73) - 0.011 * math.exp(-X / 47.2)
    if X > 1.0:
        f += ((0.011 * math.exp(-X / 47.2) - 2.0 ** (-1 / 3) / 3.0 ** (23 / 6) * 1e4 * math.pi * X ** (-8 / 3))
              * 0.5 * (1.0 + math.tanh(10.0 * math.log(X / 120.0))))
    return f


def targets(coef, ne, Te, B, nu, th):
    """The surrogate's target variables (logarithms of the coefficients over their prefactors)
    from quadrature coefficients (jI jQ jV aI aQ aV rQ rV)."""
    s, c = math.sin(th), math.cos(th)
    nuB = E * B / (2 * math.pi * ME * C)
    cot = abs(c) / abs(s)
    sg = -1.0 if c < 0 else 1.0
    Pj = ne * E * E * nu / (2 * math.sqrt(3) * C * Te * Te)
    PjV = Pj * 4.0 / (3.0 * Te) * cot
    Pa = ne * E * E / (4 * math.sqrt(3) * ME * C * nu * Te ** 3)
    X = Te * math.sqrt(math.sqrt(2) * abs(s) * 1e3 * nuB / nu)
    PrQ = ne * E * E * nuB ** 2 * s * s / (ME * C * nu ** 3) * shcherbakov_f(X)
    PrV = 2 * ne * E * E * nuB * abs(c) / (ME * C * nu * nu) * (1 - 0.11 * math.log1p(0.035 * X))
    q = [coef[0] / Pj, coef[1] / Pj, sg * coef[2] / PjV, coef[3] / Pa, coef[4] / Pa, sg * coef[5] / (Pa * cot),
         coef[6] / PrQ, sg * coef[7] / PrV]
    return np.log(np.array(q))
