"""Oracle for a two-level refinement hierarchy: prolongation, restriction and
the Berger-Oliger time step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import this module.  It shares no code
with the CUDA library in ``paper_1308_1343_gb300`` and never imports it.

The paper lists prolongation, boundary prolongation and restriction among the
operators a refinement level derives from the bboxset algebra (arXiv
1308.1343, Sec. 2, introduction, and its reference to block-structured AMR,
Berger 1984), but defines none of them.  The readings taken here:

* Vertex-centred refinement by 2: fine index f (per axis) lies at coarse
  coordinate f / 2, so even fine indices coincide with coarse points.
* Prolongation: cubic Lagrange interpolation along each axis, applied as a
  tensor product, i.e. as successive one-dimensional interpolations: along
  z for each coarse (y, x) column of the stencil, then along y, then along
  x.  At an odd fine index f the coarse points (f-3)/2 ... (f+3)/2 get the
  weights (-1, 9, 9, -1) / 16, at an even one the coarse point f/2 gets
  weight 1.  It is exact for polynomials of degree <= 3 per axis.  In time,
  linear interpolation between the coarse levels at t and t + dt:
  data = (1 - alpha) * old + alpha * new, applied before the spatial
  interpolation.
* Restriction: injection, coarse point c takes the fine value at 2c.
* Berger-Oliger sub-cycling with a buffer zone.  The fine level's region R
  (a box of fine points, not periodic) carries a buffer band of width B >= 4
  inside its faces; the trusted region is T = R shrunk by B.  One step of
  the hierarchy (coarse step dt):
    1. the coarse level takes one RK4 step of dt (periodic);
    2. the fine level takes two RK4 steps of dt/2.  Before each, the buffer
       band R \\ T and the ghost shell of R are filled by prolongation from
       the coarse levels at t and t + dt, at alpha = 0 and alpha = 1/2;
       during a step those boundary values are held fixed (rk4_padded);
    3. every coarse point c with 2c in T takes the fine value (restriction).
  One RK4 step of this scheme changes a point from data within 4 points, so
  points of T, at least B >= 4 from R's faces, only depend on data inside R
  that the scheme itself maintains.

Arrays are float64 with shape (nz, ny, nx) (x fastest): the coarse level is
one whole periodic domain, the fine level one padded box over R (ghost width
2), element [k + 2, j + 2, i + 2] holding fine point R.lo + (i, j, k).
"""
from __future__ import annotations

import numpy as np

from . import oracle

W_ODD = (-1.0 / 16.0, 9.0 / 16.0, 9.0 / 16.0, -1.0 / 16.0)


def stencil_1d(f: int):
    """(coarse indices, weights) that give fine index f along one axis."""
    if f % 2 == 0:
        return [f // 2], [1.0]
    c = (f - 1) // 2
    return [c - 1, c, c + 1, c + 2], list(W_ODD)


def prolongate(c_old, c_new, alpha: float, fpts) -> np.ndarray:
    """Values at fine points fpts (int array (n, 3) of fine (x, y, z)) from
    the coarse periodic levels c_old (time t) and c_new (t + dt), at time
    t + alpha dt, with data = (1 - alpha) old + alpha new at each coarse
    point.  One-dimensional interpolation along z of each of the 4 x 4
    coarse (y, x) columns of the stencil, then along y of the four results
    per x, then along x: each is 0 plus its four weighted terms in order,
    every product and sum rounded (an even index has one term along its
    axis; the zero weights padding it to four add exact zeros)."""
    c_old = np.asarray(c_old, dtype=np.float64)
    c_new = np.asarray(c_new, dtype=np.float64)
    nz, ny, nx = c_old.shape
    fpts = np.asarray(fpts, dtype=np.int64).reshape(-1, 3)

    def axis(f):
        # stencil_1d of every distinct coordinate, mapped back to the points
        vals, inv = np.unique(f, return_inverse=True)
        idx = np.empty((len(vals), 4), dtype=np.int64)
        w = np.zeros((len(vals), 4))
        for n, fv in enumerate(vals):
            ci, wi = stencil_1d(int(fv))
            idx[n, :] = ci[0]
            idx[n, :len(ci)] = ci
            w[n, :len(wi)] = wi
        return idx[inv], w[inv]

    (ix, wx), (iy, wy), (iz, wz) = axis(fpts[:, 0]), axis(fpts[:, 1]), axis(fpts[:, 2])
    data = (1.0 - alpha) * c_old + alpha * c_new

    def interp(w, vals):  # 0 + w0 v0 + w1 v1 + w2 v2 + w3 v3, left to right
        acc = np.zeros(len(fpts))
        for k in range(4):
            acc = acc + w[:, k] * vals[k]
        return acc

    along_x = []
    for c in range(4):
        along_y = [interp(wz, [data[iz[:, a] % nz, iy[:, b] % ny, ix[:, c] % nx]
                               for a in range(4)])
                   for b in range(4)]
        along_x.append(interp(wy, along_y))
    return interp(wx, along_x)


def shell_and_buffer(r_lo, r_hi, buffer: int):
    """Fine points (n, 3) that prolongation fills: the buffer band R \\ T and
    the star-shaped ghost shell of R (points outside R along exactly one
    axis, within 2 of R), in z-major, then y, then x order."""
    lo = np.array(r_lo)
    hi = np.array(r_hi)
    z, y, x = np.meshgrid(*[np.arange(lo[d] - 2, hi[d] + 2) for d in (2, 1, 0)], indexing="ij")
    p = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    out_axes = np.sum((p < lo) | (p >= hi), axis=1)
    inner = np.all((p >= lo + buffer) & (p < hi - buffer), axis=1)
    keep = (out_axes == 1) | ((out_axes == 0) & ~inner)
    return p[keep].astype(np.int64)


def restriction_points(t_lo, t_hi):
    """Coarse points c (n, 3) whose fine counterpart 2c lies in T."""
    ranges = [range(-(-int(t_lo[d]) // 2), -(-int(t_hi[d]) // 2)) for d in range(3)]
    pts = [(x, y, z) for z in ranges[2] for y in ranges[1] for x in ranges[0]]
    return np.array(pts, dtype=np.int64).reshape(-1, 3)


def fill(fine_p, r_lo, fpts, values) -> None:
    """Write values at fine points fpts into the padded fine array."""
    f = np.asarray(fpts)
    fine_p[f[:, 2] - r_lo[2] + 2, f[:, 1] - r_lo[1] + 2, f[:, 0] - r_lo[0] + 2] = values


def bo_step(cu, cpi, cc2, h: float, dt: float, fu_p, fpi_p, fc2_p, r_lo, r_hi,
            buffer: int = 4):
    """One step of the two-level hierarchy (see the module docstring).
    Returns new (cu, cpi, fu_p, fpi_p); inputs are not modified."""
    assert buffer >= 4
    cu1, cpi1 = oracle.rk4_periodic(cu, cpi, cc2, h, dt, 1)
    fpts = shell_and_buffer(r_lo, r_hi, buffer)
    fu_p = np.array(fu_p, dtype=np.float64)
    fpi_p = np.array(fpi_p, dtype=np.float64)
    for alpha in (0.0, 0.5):
        fill(fu_p, r_lo, fpts, prolongate(cu, cu1, alpha, fpts))
        fill(fpi_p, r_lo, fpts, prolongate(cpi, cpi1, alpha, fpts))
        fu_p, fpi_p = oracle.rk4_padded(fu_p, fpi_p, fc2_p, h / 2.0, dt / 2.0)
    t_lo = tuple(r_lo[d] + buffer for d in range(3))
    t_hi = tuple(r_hi[d] - buffer for d in range(3))
    for cx, cy, cz in restriction_points(t_lo, t_hi):
        k = (2 * cz - r_lo[2] + 2, 2 * cy - r_lo[1] + 2, 2 * cx - r_lo[0] + 2)
        cu1[cz, cy, cx] = fu_p[k]
        cpi1[cz, cy, cx] = fpi_p[k]
    return cu1, cpi1, fu_p, fpi_p
