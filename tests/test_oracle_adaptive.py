"""Pins of the oracle's adaptive ray tracing (oracle/adaptive.py) on closed-form images.

* A bilinear image is predicted exactly by every block's corners: nothing refines, and every
  filled pixel equals the function (the fill formula and the block corners are right).
* With an unreachable tolerance only the lattice and the first level's centres are traced: a
  count fixed by the image size and the base step.
* A strictly convex image (x^2 + y^2) makes every centre differ from its corners' bilinear
  prediction, so with tol = 0 every block refines down to side 2 and every pixel is traced,
  for ragged image sizes as well (the children cover the image).
* A status boundary (rays that end differently) is refined down to single pixels: every pixel
  whose neighbour ended differently is traced, when the base step resolves the region.
"""
import numpy as np
import pytest

from oracle.adaptive import FILLED, TRACED, adaptive_image


def analytic(fn, status_fn=None, nc=4):
    def render(ix, iy):
        v = fn(ix.astype(float), iy.astype(float))
        vals = np.repeat(v[:, None], nc, axis=1) * np.array([1.0, 0.5, -0.25, 0.125])[:nc]
        st = status_fn(ix, iy) if status_fn else np.ones(ix.size, dtype=np.int32)
        return vals, st
    return render


@pytest.mark.parametrize("nx,ny,s", [(33, 33, 8), (40, 27, 4), (17, 64, 16)])
def test_bilinear_image_is_filled_exactly(nx, ny, s):
    fn = lambda x, y: 3.0 + 0.7 * x - 0.2 * y + 0.01 * x * y
    img, state, status, n = adaptive_image(analytic(fn), nx, ny, 4, s, 1e-9)
    iy, ix = np.mgrid[0:ny, 0:nx]
    ref = analytic(fn)(ix.ravel(), iy.ravel())[0].reshape(ny, nx, 4)
    assert np.abs(img - ref).max() <= 1e-11 * np.abs(ref).max()
    assert ((state == TRACED) | (state == FILLED)).all()
    assert (state == FILLED).sum() > 0.6 * nx * ny


@pytest.mark.parametrize("nx,ny,s", [(33, 33, 8), (40, 27, 4), (17, 64, 16)])
def test_unreachable_tolerance_traces_lattice_and_centres(nx, ny, s):
    fn = lambda x, y: np.sin(0.3 * x) * np.cos(0.2 * y) + 2.0
    _, state, _, n = adaptive_image(analytic(fn), nx, ny, 4, s, 1e30)
    cols = len({i for i in range(nx) if i % s == 0} | {nx - 1})
    rows = len({j for j in range(ny) if j % s == 0} | {ny - 1})
    nbx, nby = -(-(nx - 1) // s), -(-(ny - 1) // s)
    with_centre = sum(1 for bi in range(nbx) for bj in range(nby)
                      if bi * s + s // 2 < min(bi * s + s, nx - 1) and bj * s + s // 2 < min(bj * s + s, ny - 1))
    assert n == cols * rows + with_centre == (state == TRACED).sum()


@pytest.mark.parametrize("nx,ny,s", [(33, 33, 8), (37, 29, 8), (20, 45, 4)])
def test_convex_image_with_zero_tolerance_traces_every_pixel(nx, ny, s):
    fn = lambda x, y: (x - 3.3) ** 2 + (y + 1.7) ** 2 + 1.0
    _, state, _, n = adaptive_image(analytic(fn), nx, ny, 4, s, 0.0)
    assert n == nx * ny and (state == TRACED).all()


def test_status_boundary_is_refined_to_pixels():
    nx = ny = 64
    inside = lambda ix, iy: ((ix - 30.3) ** 2 + (iy - 33.1) ** 2 < 18.0 ** 2)
    st_fn = lambda ix, iy: np.where(inside(ix, iy), 1, 2).astype(np.int32)
    fn = lambda x, y: np.ones_like(x)  # constant values: only the status can refine
    _, state, status, n = adaptive_image(analytic(fn, st_fn), nx, ny, 4, 4, 1e-3)
    iy, ix = np.mgrid[0:ny, 0:nx]
    st = st_fn(ix, iy)
    edge = np.zeros((ny, nx), dtype=bool)
    edge[:, :-1] |= st[:, :-1] != st[:, 1:]
    edge[:, 1:] |= st[:, :-1] != st[:, 1:]
    edge[:-1, :] |= st[:-1, :] != st[1:, :]
    edge[1:, :] |= st[:-1, :] != st[1:, :]
    assert (state[edge] == TRACED).all()
    assert n < 0.5 * nx * ny
    # traced pixels carry their own status; filled ones none
    assert (status[state == TRACED] == st[state == TRACED]).all() and (status[state == FILLED] == 0).all()
