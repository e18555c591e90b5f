"""Adaptive ray tracing, written out plainly (test infrastructure only).

The paper names adaptive ray tracing, which traces rays densely only where the image has
structure, as the route to high resolution (introduction; outlook in Section 4), and gives
no algorithm. This module restates the reading the library implements, step by step and
sequentially, so that its decisions (which pixels are traced, which blocks refine) and its
filled values can be checked against the GPU's:

1. Trace the lattice: every pixel whose column is a multiple of the base step s or the last
   column, and whose row is a multiple of s or the last row.
2. The threshold is tol times the largest Stokes I among the lattice pixels.
3. Every block of side s between lattice pixels is active. Then for side = s, s/2, ..., 2:
   a. the centre pixel of each active block (where the block has both midlines) is traced;
   b. each active block is refined when its four corners and its centre ended their rays
      differently (status codes), or, for some Stokes component, the centre differs from the
      bilinear prediction of the corners by more than the threshold (a block without a centre:
      when the corners' spread exceeds it). A refined block traces its edge midpoints and makes
      its children of side s/2 active. A block that is not refined fills its untraced pixels
      by bilinear interpolation of its corners;
   c. a pixel that some block traces is never filled (tracing wins over filling), and a pixel
      filled by two blocks (a shared edge) takes the same value from both.

The renderer is a callback, so that the same steps can run on the oracle's own pixels or on
values read from another image (to check the decisions alone). Nothing here depends on the
order in which blocks are visited: the decisions read only traced pixels, and queued pixels
are marked before any block fills.
"""
from __future__ import annotations

import numpy as np

UNTOUCHED, TRACED, FILLED = 0, 1, 2


def _blocks(n: int, s: int) -> int:
    """Blocks of side s between pixels 0 .. n-1 (the last one clamped to n-1)."""
    return (n - 1 + s - 1) // s


def adaptive_image(render, nx: int, ny: int, nc: int, base_step: int, tol: float):
    """render(ix, iy) -> (values[n, nc], status[n]) for listed pixels.

    Returns (image[ny, nx, nc], state[ny, nx] with TRACED / FILLED, status[ny, nx] of the traced
    pixels (0 elsewhere), number of rays traced)."""
    assert base_step >= 2 and base_step & (base_step - 1) == 0
    img = np.zeros((ny, nx, nc))
    state = np.zeros((ny, nx), dtype=np.int8)
    status = np.zeros((ny, nx), dtype=np.int32)
    traced = 0

    def trace(pixels):
        nonlocal traced
        todo = sorted({p for p in pixels if state[p[1], p[0]] != TRACED})
        if not todo:
            return
        ix = np.array([p[0] for p in todo])
        iy = np.array([p[1] for p in todo])
        vals, st = render(ix, iy)
        img[iy, ix] = np.asarray(vals).reshape(len(todo), nc)
        status[iy, ix] = st
        state[iy, ix] = TRACED
        traced += len(todo)

    s = base_step
    cols = [i for i in range(nx) if i % s == 0 or i == nx - 1]
    rows = [j for j in range(ny) if j % s == 0 or j == ny - 1]
    trace([(i, j) for j in rows for i in cols])
    thr = tol * img[..., 0][state == TRACED].max()

    active = {(bi, bj) for bj in range(_blocks(ny, s)) for bi in range(_blocks(nx, s))}
    side = s
    while side >= 2:
        h = side // 2

        def corners(bi, bj):
            i0, j0 = bi * side, bj * side
            i1, j1 = min(i0 + side, nx - 1), min(j0 + side, ny - 1)
            im = i0 + h if i0 + h < i1 else -1
            jm = j0 + h if j0 + h < j1 else -1
            return i0, j0, i1, j1, im, jm

        # a. centres
        trace([(im, jm) for (bi, bj) in active for (_, _, _, _, im, jm) in [corners(bi, bj)] if im >= 0 and jm >= 0])
        # b. decisions, from traced pixels only
        queue, fills, children = set(), [], set()
        for (bi, bj) in sorted(active):
            i0, j0, i1, j1, im, jm = corners(bi, bj)
            centre = im >= 0 and jm >= 0
            ci, cj = (im, jm) if centre else (i0, j0)
            codes = {status[j0, i0], status[j0, i1], status[j1, i0], status[j1, i1], status[cj, ci]}
            refine = len(codes) > 1
            a, b, c, d = img[j0, i0], img[j0, i1], img[j1, i0], img[j1, i1]
            for q in range(nc):
                if refine:
                    break
                if centre:
                    fx = (im - i0) / (i1 - i0)
                    fy = (jm - j0) / (j1 - j0)
                    pred = (1 - fx) * (1 - fy) * a[q] + fx * (1 - fy) * b[q] + (1 - fx) * fy * c[q] + fx * fy * d[q]
                    refine = abs(img[jm, im, q] - pred) > thr
                else:
                    refine = max(a[q], b[q], c[q], d[q]) - min(a[q], b[q], c[q], d[q]) > thr
            if refine:
                if im >= 0:
                    queue |= {(im, j0), (im, j1)}
                if jm >= 0:
                    queue |= {(i0, jm), (i1, jm)}
                if h >= 2:
                    for dj in (0, 1):
                        for di in (0, 1):
                            x, y = 2 * bi + di, 2 * bj + dj
                            if x * h < i1 and y * h < j1 and x * h < nx - 1 and y * h < ny - 1:
                                children.add((x, y))
            else:
                fills.append((i0, j0, i1, j1))
        # c. tracing wins: mark the queued pixels first, then fill what is left untouched
        for (i, j) in queue:
            if state[j, i] != TRACED:
                state[j, i] = -1  # queued this level
        for (i0, j0, i1, j1) in fills:
            a, b, c, d = img[j0, i0].copy(), img[j0, i1].copy(), img[j1, i0].copy(), img[j1, i1].copy()
            for j in range(j0, j1 + 1):
                for i in range(i0, i1 + 1):
                    if state[j, i] != UNTOUCHED:
                        continue
                    fx = (i - i0) / (i1 - i0)
                    fy = (j - j0) / (j1 - j0)
                    img[j, i] = (1 - fx) * (1 - fy) * a + fx * (1 - fy) * b + (1 - fx) * fy * c + fx * fy * d
                    state[j, i] = FILLED
        state[state == -1] = UNTOUCHED
        trace(sorted(queue))
        active = children
        side = h
    return img, state, status, traced
