"""Pins of the oracle's visibilities (the definition V = sum S dOmega e^{-2 pi i (u x + v y)}
written out): V(0, 0) is the flux, a real image gives Hermitian visibilities, Parseval's
relation holds on the full grid, and moving the image by one pixel multiplies V by the
phase e^{-2 pi i u dx}."""
import numpy as np


def test_visibility_identities(ora, synth):
    cam = ora.camera(synth.Camera(nx=16, ny=12))
    rng = np.random.default_rng(4)
    img = rng.uniform(0, 1, (12, 16))
    V = ora.visibilities(cam, img)
    L = 6.67430e-8 * cam.M_bh_g / 2.99792458e10 ** 2
    dx = cam.fov_M * L / (cam.nx * cam.dist_cm)
    # zero spacing: the flux
    flux = ora.image_stats(cam, np.stack([img, 0 * img, 0 * img, 0 * img], axis=-1))[0]
    assert abs(V[6, 8] / flux - 1) < 1e-12
    # Hermitian: V(-u, -v) = conj V(u, v) (indices away from the unpaired Nyquist row/column)
    for l in range(1, 12):
        for k in range(1, 16):
            assert abs(V[12 - l, 16 - k] - np.conj(V[l, k])) < 1e-12 * abs(V).max()
    # Parseval on the full grid
    a = img * dx * dx * 1e23
    assert abs((np.abs(V) ** 2).sum() / (16 * 12 * (a ** 2).sum()) - 1) < 1e-12
    # shift theorem: moving the image one pixel along +x (periodic) multiplies V by e^{-2 pi i u dx}
    Vs = ora.visibilities(cam, np.roll(img, 1, axis=1))
    u = (np.arange(16) - 8) / (16 * dx)
    ratio = Vs / V
    assert np.allclose(ratio, np.exp(-2j * np.pi * u * dx)[None, :], rtol=1e-10, atol=0)
