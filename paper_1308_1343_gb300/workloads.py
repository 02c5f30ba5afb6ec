"""Seeded synthetic inputs shaped like the level workloads.

This module only draws random numbers and evaluates the initial data and the
wave-speed field on the host; it contains none of the method's arithmetic
(no stencil, no time stepping, no ghost exchange).  Both the CUDA library's
tests and the CPU oracle's tests take their inputs from here.

Recipe (all arrays float64, shape (nz, ny, nx), x fastest):

* Grid: a periodic domain of n_d points per axis, spacing h, coordinates
  x_i = i*h (i = 0..n-1), physical length n_d*h.  dt = 0.25*h.
* Plane wave: u = sin(2 pi (x + 2y + 3z)), pi = 0, c2 = 1 on [0,1)^3.
* Wave speed: c2 = 1 + 0.5*tanh(sum_{k<8} a_k exp(-r_k^2 / (2 w_k^2))) with
  r_k the minimum-image periodic distance to centre k; centres uniform in
  the domain, widths w_k ~ U[0.05, 0.2], amplitudes a_k ~ N(0, 1).
* Pulse: u0 = exp(-r^2 / (2 * 0.05^2)) around a seeded centre, pi0 = 0.
* Draw order from numpy.random.default_rng(seed) (PCG64): the 8 centres
  (8x3 uniforms), the 8 widths, the 8 amplitudes, the pulse centre (3), and
  -- for the differentiation workload only -- a 9th centre and width whose
  bump, with amplitude 0.1, is added to c2 outside the tanh to make the
  "observed" wave speed.
* Uneven level: a periodic domain bisected breadth-first for 6 levels (64
  boxes); each box splits across its longest axis (ties to the lower axis
  index) at lo + 8*round(f*len/8), f ~ U[0.3, 0.7], round half to even,
  clamped so both halves keep >= 8 points.
* Ensemble: instance edges uniform in {24, 32, ..., 96}; instance i draws its
  fields with seed 5000 + i on [0,1)^3 with h = 1/n.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np


@dataclass
class Domain:
    """A periodic domain of n = (nx, ny, nz) points with spacing h."""
    n: Tuple[int, int, int]
    h: float
    lo: Tuple[int, int, int] = (0, 0, 0)

    @property
    def lengths(self) -> Tuple[float, float, float]:
        return tuple(ni * self.h for ni in self.n)

    @property
    def shape(self) -> Tuple[int, int, int]:
        """numpy shape (nz, ny, nx)."""
        return (self.n[2], self.n[1], self.n[0])


@dataclass
class Instance:
    """Fields of one periodic domain plus the boxes that tile it."""
    dom: Domain
    u: np.ndarray
    pi: np.ndarray
    c2: np.ndarray
    dt: float
    boxes: List[Tuple[Tuple[int, int, int], Tuple[int, int, int]]] = field(default_factory=list)
    c2_obs: Optional[np.ndarray] = None

    def __post_init__(self):
        if not self.boxes:
            self.boxes = [((0, 0, 0), tuple(self.dom.n))]


def _axis_coords(n: int, h: float) -> np.ndarray:
    return np.arange(n, dtype=np.float64) * h


def _min_image_sq(n: int, h: float, c: float) -> np.ndarray:
    """Squared minimum-image distance along one periodic axis."""
    L = n * h
    d = np.abs(_axis_coords(n, h) - c)
    d = np.minimum(d, L - d)
    return d * d


def gaussian(dom: Domain, centre, width: float) -> np.ndarray:
    """exp(-r^2 / (2 w^2)), r the minimum-image distance to centre.

    Evaluated as a product of three 1D factors (the exponential of a sum of
    per-axis squares), which is exact algebra and fast on large grids."""
    nx, ny, nz = dom.n
    fx = np.exp(-_min_image_sq(nx, dom.h, centre[0]) / (2.0 * width * width))
    fy = np.exp(-_min_image_sq(ny, dom.h, centre[1]) / (2.0 * width * width))
    fz = np.exp(-_min_image_sq(nz, dom.h, centre[2]) / (2.0 * width * width))
    return fz[:, None, None] * (fy[None, :, None] * fx[None, None, :])


def plane_wave(n: int) -> Instance:
    """u = sin(2 pi (x + 2y + 3z)), pi = 0, c2 = 1 on the unit periodic cube."""
    h = 1.0 / n
    dom = Domain((n, n, n), h)
    x = _axis_coords(n, h)
    ph = 2.0 * np.pi * (x[None, None, :] + 2.0 * x[None, :, None] + 3.0 * x[:, None, None])
    u = np.sin(ph)
    return Instance(dom, np.ascontiguousarray(u), np.zeros_like(u), np.ones_like(u), 0.25 * h)


def bumpy_instance(dom: Domain, seed: int, with_obs: bool = False) -> Instance:
    """Variable wave speed from 8 seeded bumps and a Gaussian pulse."""
    rng = np.random.default_rng(seed)
    L = np.array(dom.lengths)
    centres = rng.uniform(0.0, 1.0, size=(8, 3)) * L
    widths = rng.uniform(0.05, 0.2, size=8)
    amps = rng.normal(0.0, 1.0, size=8)
    pulse_c = rng.uniform(0.0, 1.0, size=3) * L
    s = np.zeros(dom.shape)
    for k in range(8):
        s += amps[k] * gaussian(dom, centres[k], widths[k])
    c2 = 1.0 + 0.5 * np.tanh(s)
    u = gaussian(dom, pulse_c, 0.05)
    c2_obs = None
    if with_obs:
        c9 = rng.uniform(0.0, 1.0, size=3) * L
        w9 = rng.uniform(0.05, 0.2)
        c2_obs = c2 + 0.1 * gaussian(dom, c9, w9)
    return Instance(dom, np.ascontiguousarray(u), np.zeros(dom.shape),
                    np.ascontiguousarray(c2), 0.25 * dom.h, c2_obs=c2_obs)


def bisect_boxes(n: Tuple[int, int, int], levels: int, seed: int, quantum: int = 8,
                 min_edge: int = 8):
    """Breadth-first recursive bisection of [0, n) into 2**levels boxes."""
    rng = np.random.default_rng(seed)
    boxes = [((0, 0, 0), tuple(n))]
    for _ in range(levels):
        nxt = []
        for lo, hi in boxes:
            ext = [hi[d] - lo[d] for d in range(3)]
            ax = int(np.argmax(ext))  # first maximum: ties go to the lower axis
            f = rng.uniform(0.3, 0.7)
            cut = quantum * int(np.round(f * ext[ax] / quantum))  # half to even
            cut = min(max(cut, min_edge), ext[ax] - min_edge)
            if ext[ax] < 2 * min_edge:
                nxt.append((lo, hi))
                continue
            hi1 = list(hi)
            hi1[ax] = lo[ax] + cut
            lo2 = list(lo)
            lo2[ax] = lo[ax] + cut
            nxt.append((tuple(lo), tuple(hi1)))
            nxt.append((tuple(lo2), tuple(hi)))
        boxes = nxt
    return boxes


def single_box(n: int = 256, seed: int = 2) -> Instance:
    """One periodic n^3 box on [0,1)^3, variable c2, Gaussian pulse."""
    return bumpy_instance(Domain((n, n, n), 1.0 / n), seed)


def uneven_level(n=(512, 512, 256), h: float = 1.0 / 256, levels: int = 6,
                 seed: int = 3, box_seed: int = 30) -> Instance:
    """A periodic domain tiled by 2**levels uneven boxes, variable c2, pulse."""
    inst = bumpy_instance(Domain(tuple(n), h), seed)
    inst.boxes = bisect_boxes(tuple(n), levels, box_seed)
    return inst


def gradient_problem(n: int = 128, seed: int = 4) -> Instance:
    """n^3 periodic box with c2 and the perturbed c2_obs."""
    return bumpy_instance(Domain((n, n, n), 1.0 / n), seed, with_obs=True)


def ensemble_edges(count: int = 256, seed: int = 5, edges=tuple(range(24, 97, 8))):
    rng = np.random.default_rng(seed)
    return [int(e) for e in rng.choice(np.array(edges), size=count)]


def ensemble(count: int = 256, seed: int = 5, edges=tuple(range(24, 97, 8))) -> List[Instance]:
    """Independent periodic cubes, each with its own seeded fields."""
    out = []
    for i, n in enumerate(ensemble_edges(count, seed, edges)):
        out.append(bumpy_instance(Domain((n, n, n), 1.0 / n), 5000 + i))
    return out


def refined_pair(n: int, seed: int, r_lo, r_hi, width: float = 0.05) -> Instance:
    """Inputs of a two-level hierarchy on the unit periodic cube: the fine grid
    (2n)^3 (spacing 1/(2n)) carries seed's bumpy wave speed and a Gaussian
    pulse of the given width centred in the refined region [r_lo, r_hi)
    (fine indices).  The coarse level's fields are these fields at even
    fine indices, the points the two grids share."""
    fine = bumpy_instance(Domain((2 * n,) * 3, 0.5 / n), seed)
    centre = [(r_lo[d] + r_hi[d] - 1) * 0.5 * fine.dom.h for d in range(3)]
    fine.u = np.ascontiguousarray(gaussian(fine.dom, centre, width))
    return fine


def refined_fields(n: int, seed: int, r_lo, r_hi, width: float = 0.05):
    """The fields of refined_pair(n, seed, r_lo, r_hi, width) without the
    whole fine grid: returns (coarse Instance on n^3, (u, pi, c2) on the fine
    region [r_lo, r_hi) only).  Same draws and the same per-point operations
    in the same order, so the values are refined_pair's, bit for bit."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.0, 1.0, size=(8, 3))
    widths = rng.uniform(0.05, 0.2, size=8)
    amps = rng.normal(0.0, 1.0, size=8)
    hf = 0.5 / n
    pulse = [(r_lo[d] + r_hi[d] - 1) * 0.5 * hf for d in range(3)]

    def on(ix, iy, iz, h, m):
        """Fields at integer grid indices (per axis) of spacing h, period m."""
        def g(c, w):
            f = []
            for idx, cd in zip((ix, iy, iz), c):
                d = np.abs(np.asarray(idx, dtype=np.float64) * h - cd)
                d = np.minimum(d, m * h - d)
                f.append(np.exp(-(d * d) / (2.0 * w * w)))
            return f[2][:, None, None] * (f[1][None, :, None] * f[0][None, None, :])
        s = np.zeros((len(iz), len(iy), len(ix)))
        for k in range(8):
            s += amps[k] * g(centres[k], widths[k])
        return np.ascontiguousarray(g(pulse, width)), np.zeros(s.shape), 1.0 + 0.5 * np.tanh(s)

    a = np.arange(n)
    cu, cpi, cc2 = on(a, a, a, 1.0 / n, n)
    coarse = Instance(Domain((n, n, n), 1.0 / n), cu, cpi, np.ascontiguousarray(cc2), 0.25 / n)
    rng_ = [np.arange(r_lo[d], r_hi[d]) for d in range(3)]
    fine = on(rng_[0], rng_[1], rng_[2], hf, 2 * n)
    return coarse, fine


def random_direction(shape, seed: int) -> np.ndarray:
    """N(0,1) per point, scaled to unit RMS."""
    d = np.random.default_rng(seed).normal(size=shape)
    return d / np.sqrt(np.mean(d * d))
