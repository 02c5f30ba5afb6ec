"""Brute-force point-set algebra on a uniform integer grid (test oracle).

TEST INFRASTRUCTURE ONLY.  A region of a refinement level is represented
here the naive way the paper sets aside for production use (Sec. 2.1,
"Background"): as the explicit set of its integer grid points.  Every set
operation is then Python's own set operation, which *defines* the result
the production bboxset (stored as discrete derivatives, swept per Sec. 2.3)
must reproduce.

Conventions (the paper leaves them open; these are the readings used):
* a box is half-open, [lo, hi) per axis, unit stride on the level;
* the discrete derivative along axis i marks where membership changes
  between p - e_i and p:  (d_i R)(p) = R(p) xor R(p - e_i).  The paper calls
  its difference "leftward" and recovers R by a left-to-right scan
  (Sec. 2.2), which is this convention; with it the derivative of a cuboid
  is exactly its 2^D corner points {lo, hi}^D.
"""
from __future__ import annotations

from itertools import product
from typing import Iterable, Sequence, Set, Tuple

Point = Tuple[int, ...]


def box_points(lo: Sequence[int], hi: Sequence[int]) -> Set[Point]:
    """All grid points of the half-open box [lo, hi)."""
    return set(product(*[range(a, b) for a, b in zip(lo, hi)]))


def union_of_boxes(boxes: Iterable[Tuple[Sequence[int], Sequence[int]]]) -> Set[Point]:
    s: Set[Point] = set()
    for lo, hi in boxes:
        s |= box_points(lo, hi)
    return s


def shift(s: Set[Point], v: Sequence[int]) -> Set[Point]:
    """shift(R, v) = { p + v : p in R } (paper Sec. 2, list of operations)."""
    return {tuple(a + b for a, b in zip(p, v)) for p in s}


def expand(s: Set[Point], lo_by: Sequence[int], hi_by: Sequence[int]) -> Set[Point]:
    """Grow R by lo_by[d] points downward and hi_by[d] upward along each axis
    (the 'expand' operation of Sec. 2): the union of all shifts of R by
    vectors v with -lo_by[d] <= v[d] <= hi_by[d]."""
    out: Set[Point] = set()
    for v in product(*[range(-a, b + 1) for a, b in zip(lo_by, hi_by)]):
        out |= shift(s, v)
    return out


def expand_axis(s: Set[Point], axis: int, w: int) -> Set[Point]:
    """Grow R by w points on both sides along one axis only."""
    D = len(next(iter(s))) if s else 3
    lo = [0] * D
    hi = [0] * D
    lo[axis] = hi[axis] = w
    return expand(s, lo, hi)


def derivative(s: Set[Point], axis: int) -> Set[Point]:
    """(d_axis R)(p) = R(p) xor R(p - e_axis)."""
    if not s:
        return set()
    D = len(next(iter(s)))
    e = [0] * D
    e[axis] = 1
    return s ^ shift(s, e)


def full_derivative(s: Set[Point], D: int) -> Set[Point]:
    """dR = d_0 d_1 ... d_{D-1} R (the set the paper stores, Sec. 2.2)."""
    for a in range(D):
        s = derivative(s, a)
    return s


def antiderivative(ds: Set[Point], axis: int) -> Set[Point]:
    """Undo derivative(., axis) by a left-to-right prefix-xor scan along the
    axis: R(p) = xor of dR(q) over q <= p on p's grid line."""
    lines = {}
    for p in ds:
        key = p[:axis] + p[axis + 1:]
        lines.setdefault(key, []).append(p[axis])
    out: Set[Point] = set()
    for key, xs in lines.items():
        xs.sort()
        # membership toggles at every stored point; a finite set has an even
        # number of toggles on each line
        for a, b in zip(xs[0::2], xs[1::2]):
            for x in range(a, b):
                out.add(key[:axis] + (x,) + key[axis:])
    return out


def full_antiderivative(ds: Set[Point], D: int) -> Set[Point]:
    for a in reversed(range(D)):
        ds = antiderivative(ds, a)
    return ds


def star_ghosts(lo: Sequence[int], hi: Sequence[int], g: int = 2) -> Set[Point]:
    """Ghost region of one box: (union_d expand_d(box, g)) minus the box --
    exactly the points a centred stencil of half-width g reads outside it."""
    b = box_points(lo, hi)
    out: Set[Point] = set()
    for d in range(len(lo)):
        out |= expand_axis(b, d, g)
    return out - b
