"""The oracle against its stored image (tests/golden/adaf16_i60.txt, written by
tests/golden/make_golden.py from the oracle alone). A change to the oracle's arithmetic shows
up here first; the stored file is only rewritten on purpose, by that script."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "adaf16_i60.txt")


def load_golden():
    d = np.loadtxt(GOLDEN)
    n = int(d[:, 0].max()) + 1
    img = d[:, 2:6].reshape(n, n, 4)
    return img, d[:, 6].reshape(n, n).astype(int), d[:, 7].reshape(n, n).astype(int), d[:, 8].reshape(n, n) > 0


def test_oracle_reproduces_stored_image(ora, synth):
    img0, ns0, st0, mask = load_golden()
    cam = ora.camera(synth.Camera(incl_deg=60.0, nx=16, ny=16), eps=0.05, nmax=20000)
    img, ns, st, _ = ora.render_image(cam, ora.adaf_model(synth.adaf_params(1)))
    assert np.array_equal(ns, ns0) and np.array_equal(st, st0)
    scale = np.maximum(img0[..., 0], 1e-8 * img0[..., 0].max())
    err = np.abs(img - img0).max(axis=-1) / scale
    assert err[~mask].max() <= 1e-12, err.max()
    assert img0[..., 0].min() > 0 and mask.mean() < 0.05
