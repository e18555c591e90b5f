"""Write the stored oracle image under tests/golden/ from the oracle and the seeded input
generators only (no GPU code). Run it again only when the oracle's arithmetic changes on
purpose; the commit that does so names the passage of the paper that justifies the change.

    python tests/golden/make_golden.py

adaf16_i60.txt: the ADAF (seed 1) seen from i = 60 deg at 230 GHz, a = 0.9375, FOV 40 M,
r_cam = 1000 M, 16 x 16 pixels, eps = 0.05, N_max = 20000: per pixel the oracle's I, Q, U, V
[erg s^-1 cm^-2 sr^-1 Hz^-1], step count, stop status, and whether the pixel is in the
sensitivity mask (its output moves by more than 1e-10 of max(I_pixel, 1e-8 max I) under a
one-ulp nudge of the pixel position, or its step count moves).
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2302_02733_gb300 import synth  # noqa: E402


def adaf16():
    cam = oracle.camera(synth.Camera(incl_deg=60.0, nx=16, ny=16), eps=0.05, nmax=20000)
    m = oracle.adaf_model(synth.adaf_params(1))
    img, ns, st, _ = oracle.render_image(cam, m)
    scale = np.maximum(img[..., 0], 1e-8 * img[..., 0].max())
    mask = np.zeros(ns.shape, dtype=bool)
    for pert in (1, 2):
        im2, ns2, _, _ = oracle.render_image(cam, m, pert=pert)
        mask |= (np.abs(im2 - img).max(axis=-1) / scale > 1e-10) | (ns2 != ns)
    return img, ns, st, mask


def main():
    img, ns, st, mask = adaf16()
    path = os.path.join(HERE, "adaf16_i60.txt")
    with open(path, "w") as f:
        f.write("# oracle image, written by tests/golden/make_golden.py (recipe in its docstring)\n")
        f.write("# iy ix I Q U V nsteps status masked\n")
        for iy in range(img.shape[0]):
            for ix in range(img.shape[1]):
                I, Q, U, V = img[iy, ix]
                f.write(f"{iy} {ix} {I:.17e} {Q:.17e} {U:.17e} {V:.17e} {ns[iy, ix]} {st[iy, ix]} "
                        f"{int(mask[iy, ix])}\n")
    print(f"wrote {path}: {mask.sum()} masked pixels")


if __name__ == "__main__":
    main()
