"""Pins of the oracle's transport of the coherency tensor, through the vector transport it
applies to each index (oracle/oracle.c, the transfer's own segment propagator), and of the
camera's reading of it (the transfer's own camera_stokes).

Along a null geodesic k of the Kerr metric, a parallel-transported vector f keeps f.f and f.k,
and the Walker-Penrose quantity (Walker & Penrose 1970; in this form Connors, Piran & Stark
1980 and Chandrasekhar 1983)

    kappa = (A - i B)(r - i a cos(theta)),
    A = (k^t f^r - k^r f^t) + a sin^2(theta) (k^r f^phi - k^phi f^r),
    B = [(r^2 + a^2)(k^phi f^theta - k^theta f^phi) - a (k^t f^theta - k^theta f^t)] sin(theta),

in Boyer-Lindquist components. The oracle integrates in Kerr-Schild coordinates, whose
components differ by v^t_BL = v^t - (2r/Delta) v^r and v^phi_BL = v^phi - (a/Delta) v^r. The
transport is Heun's method, second order, so every invariant drifts by O(eps^2) and falls
about fourfold when the step parameter halves. A sign slip in the transport matrix, or the
two factors of its h^2 term swapped, breaks that order. The rays are strongly lensed ones that
escape or fall in at a = 0.9375, plus a ray that crosses the polar axis at a = 0. kappa is
unchanged by the axis reflection: sin(theta) and every theta component change sign together.
"""
import math

import numpy as np
import pytest

A_SPIN = 0.9375


def screen_vector(ora, a, x, K, angle):
    """A unit vector normal to K and to the Kerr-Schild normal observer at x."""
    g = ora.metric(a, x[1], x[2])
    gi = np.linalg.inv(g)
    u = -gi[:, 0] / math.sqrt(-gi[0, 0])
    dot = lambda p, q: p @ g @ q
    w = -dot(K, u)
    e3 = K / w - u
    basis = []
    for v in (np.array([0.0, 0.0, 1.0, 0.0]), np.array([0.0, 0.0, 0.0, 1.0]), np.array([0.0, 1.0, 0.0, 0.0])):
        v = v + dot(v, u) * u - dot(v, e3) * e3
        for b in basis:
            v = v - dot(v, b) * b
        if dot(v, v) > 1e-12:
            basis.append(v / math.sqrt(dot(v, v)))
        if len(basis) == 2:
            break
    return math.cos(angle) * basis[0] + math.sin(angle) * basis[1]


def to_boyer_lindquist(a, r, v):
    D = r * r - 2.0 * r + a * a
    return np.array([v[0] - 2.0 * r / D * v[1], v[1], v[2], v[3] - a / D * v[1]])


def walker_penrose(a, r, th, k, f):
    k, f = to_boyer_lindquist(a, r, k), to_boyer_lindquist(a, r, f)
    s, c = math.sin(th), math.cos(th)
    A = (k[0] * f[1] - k[1] * f[0]) + a * s * s * (k[1] * f[3] - k[3] * f[1])
    B = ((r * r + a * a) * (k[3] * f[2] - k[2] * f[3]) - a * (k[0] * f[2] - k[2] * f[0])) * s
    return complex(A, -B) * complex(r, -a * c)


def drifts(ora, synth, a, incl, px, py, eps):
    """(status, axis crossings, max |f.f - 1|, max |f.k|, max |kappa - kappa_far| / |kappa_far|)
    for a unit screen vector given at the far end of the ray and carried to the camera."""
    cam = ora.camera(synth.Camera(a=a, incl_deg=incl), eps=eps, nmax=20000)
    st, status = ora.trace_geodesic(cam, px, py)
    M = len(st) - 1
    fs = ora.transport_vector(a, st, screen_vector(ora, a, st[M, :4], st[M, 4:8], 0.7))
    ff, fk, kap = [], [], []
    for n in range(M + 1):
        g = ora.metric(a, st[n, 1], st[n, 2])
        K = st[n, 4:8]
        ff.append(fs[n] @ g @ fs[n] - 1.0)
        fk.append(fs[n] @ g @ K)
        kap.append(walker_penrose(a, st[n, 1], st[n, 2], K, fs[n]))
    kap = np.array(kap)
    return (status, int((st[:, 8] < 0).sum()), np.abs(ff).max(), np.abs(fk).max(),
            np.abs(kap - kap[M]).max() / abs(kap[M]))


# (spin, inclination, pixel x, pixel y, expected status, bounds on the three drifts at eps 0.05)
RAYS = [
    (A_SPIN, 60.0, -4.0, 2.0, "ESCAPE", (1e-3, 1e-3, 0.15)),
    (A_SPIN, 60.0, 0.05, 5.2, "ESCAPE", (2e-3, 1e-3, 0.12)),
    (A_SPIN, 20.0, 2.0, 1.0, "HORIZON", (1e-3, 3e-3, 1.0)),
    (0.0, 60.0, 0.0, 6.0, "ESCAPE", (5e-4, 5e-4, 0.01)),
]


@pytest.mark.parametrize("a,incl,px,py,status,bounds", RAYS)
def test_transport_invariants_converge_at_second_order(ora, synth, a, incl, px, py, status, bounds):
    coarse = drifts(ora, synth, a, incl, px, py, 0.05)
    fine = drifts(ora, synth, a, incl, px, py, 0.025)
    assert coarse[0] == getattr(ora, status) and fine[0] == coarse[0]
    if a == 0.0:
        assert coarse[1] >= 1 and fine[1] >= 1  # the ray crossed the axis
    for j in range(3):
        assert coarse[2 + j] < bounds[j], (j, coarse)
        assert coarse[2 + j] > 3.0 * fine[2 + j], (j, coarse, fine)  # O(eps^2): about 4x


def test_walker_penrose_detects_a_sign_slip(ora, synth):
    """Heun's transport with the connection's sign flipped (the plausible slip), written here
    from the oracle's connection, breaks kappa at order one on the same ray, where the oracle's
    transport holds it to 0.15."""
    a = A_SPIN
    cam = ora.camera(synth.Camera(a=a, incl_deg=60.0), eps=0.05, nmax=20000)
    st, _ = ora.trace_geodesic(cam, -4.0, 2.0)
    assert (st[:, 8] >= 0).all()  # no axis crossing on this ray
    M = len(st) - 1

    def tmat(n):
        G = ora.connection(a, st[n, 1], st[n, 2]).reshape(4, 4, 4)  # [mu][alpha][beta]
        return np.einsum("mab,a->mb", G, st[n, 4:8])

    f = screen_vector(ora, a, st[M, :4], st[M, 4:8], 0.7)
    k0 = walker_penrose(a, st[M, 1], st[M, 2], st[M, 4:8], f)
    worst, T1 = 0.0, -tmat(M)
    for n in range(M - 1, -1, -1):
        h, T0 = abs(st[n, 8]), -tmat(n)
        f = f + 0.5 * h * (T1 @ f + T0 @ f) + 0.5 * h * h * (T0 @ (T1 @ f))
        worst = max(worst, abs(walker_penrose(a, st[n, 1], st[n, 2], st[n, 4:8], f) - k0) / abs(k0))
        T1 = T0
    assert worst > 0.5, worst


def wrap_half_turn(d):
    """An angle difference taken modulo pi into [-pi/2, pi/2)."""
    return (d + math.pi / 2) % math.pi - math.pi / 2


@pytest.mark.parametrize("a,incl", [(A_SPIN, 60.0), (A_SPIN, 20.0), (0.0, 60.0), (-0.7, 75.0)])
def test_camera_polarization_angle_matches_connors_piran_stark(ora, synth, a, incl):
    """The camera's Stokes basis and Q/U convention, through the transfer's own camera reading
    (oracle camera_stokes). A unit vector f is placed in the screen deep in the field (the
    closest approach of an escaping ray, the far end of one that falls in) and carried to the
    camera. The reading of N = f f^T gives the angle chi = atan2(U, Q) / 2 from the image's x axis
    toward its y axis. Connors, Piran & Stark (1980) give the same angle at infinity from the
    Walker-Penrose constant and the image coordinates (alpha, beta) = (x, y):
        E_alpha = (beta k2 - nu k1) / (beta^2 + nu^2),  E_beta = (beta k1 + nu k2) / (beta^2 + nu^2),
        nu = -(alpha + a sin(i)),  kappa = k1 + i k2.
    The camera sits at r = 1e4 M, so the two agree to about M / r. A swapped or flipped image
    axis, or a wrong sign of Q or U, misses by up to pi/2."""
    cam = ora.camera(synth.Camera(a=a, incl_deg=incl, r_cam=1.0e4), eps=0.025, nmax=200000)
    for al, be in ((6.0, 2.0), (-5.0, 3.0), (3.0, -6.0), (0.5, 7.0), (-7.5, -1.0), (12.0, 9.0)):
        st, status = ora.trace_geodesic(cam, al, be)
        assert status in (ora.ESCAPE, ora.HORIZON)
        n0 = int(np.argmin(st[:, 1])) if status == ora.ESCAPE else len(st) - 1
        f = screen_vector(ora, a, st[n0, :4], st[n0, 4:8], 0.4)
        fs = ora.transport_vector(a, st[: n0 + 1], f)
        kap = walker_penrose(a, st[n0, 1], st[n0, 2], -st[n0, 4:8], f)  # forward momentum
        nu = -(al + a * math.sin(math.radians(incl)))
        Ea = (be * kap.imag - nu * kap.real) / (be * be + nu * nu)
        Eb = (be * kap.real + nu * kap.imag) / (be * be + nu * nu)
        S = ora.camera_stokes(cam, al, be, np.outer(fs[0], fs[0]))
        assert abs(math.hypot(S[1], S[2]) / S[0] - 1.0) < 1e-9 and abs(S[3]) < 1e-12 * S[0]
        d = wrap_half_turn(0.5 * math.atan2(S[2], S[1]) - math.atan2(Eb, Ea))
        assert abs(d) < 2e-3, (al, be, status, d)
