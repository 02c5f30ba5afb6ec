"""CPU tests of the two-level hierarchy's host side: the bboxset spacing
change equals point enumeration; hierarchy creation enforces its rules; and
the prolongation and restriction point sets the library derives with the
bboxset algebra equal the oracle's sets, exactly.  No kernel is launched."""
import ctypes
import random

import numpy as np
import pytest

from oracle import hierarchy as H
from oracle import pointset as P


@pytest.fixture(scope="module")
def B():
    from paper_1308_1343_gb300 import binding, build
    build.build()
    binding.lib()
    return binding


def _arr(boxes):
    return np.ascontiguousarray(np.array([list(lo) + list(hi) for lo, hi in boxes],
                                         dtype=np.int64).reshape(-1, 6))


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


@pytest.mark.parametrize("seed", range(20))
def test_coarsen_matches_point_enumeration(B, seed):
    rng = random.Random(500 + seed)
    boxes = []
    for _ in range(rng.randrange(1, 5)):
        lo = [rng.randrange(-6, 10) for _ in range(3)]
        hi = [rng.randrange(l, 14) for l in lo]
        boxes.append((lo, hi))
    a = _arr(boxes)
    n = ctypes.c_int64()
    for r in (1, 2, 3):
        B.check(B.lib().sc_bboxset_coarsen(_p(a), len(boxes), r, None, 0, ctypes.byref(n)))
        out = np.zeros((max(n.value, 1), 6), dtype=np.int64)
        B.check(B.lib().sc_bboxset_coarsen(_p(a), len(boxes), r, _p(out), n.value,
                                           ctypes.byref(n)))
        got = set()
        for row in out[:n.value]:
            got |= P.box_points(row[:3], row[3:])
        pts = P.union_of_boxes(boxes)
        want = {c for c in {tuple(v // r for v in p) for p in pts}
                if tuple(r * v for v in c) in pts}
        assert got == want, (boxes, r)
    with pytest.raises(B.ScError, match="ratio"):
        B.check(B.lib().sc_bboxset_coarsen(_p(a), len(boxes), 0, None, 0, ctypes.byref(n)))


def _levels(n, r_lo, r_hi, fine_boxes=None, coarse_periodic=7, fine_periodic=0, fine_h=None,
            coarse_boxes=None):
    from paper_1308_1343_gb300.level import Level
    coarse = Level(coarse_boxes or [((0, 0, 0), (n, n, n), 0)],
                   [dict(hi=(n, n, n), h=1.0 / n, periodic=coarse_periodic)])
    fb = fine_boxes or [(r_lo, r_hi)]
    fine = Level([(lo, hi, 0) for lo, hi in fb],
                 [dict(lo=r_lo, hi=r_hi, h=fine_h or 0.5 / n, periodic=fine_periodic)])
    return coarse, fine


def test_creation_rules(B):
    from paper_1308_1343_gb300.level import Hierarchy
    c, f = _levels(32, (8, 8, 8), (40, 40, 40))
    Hierarchy(c, f).close()
    with pytest.raises(B.ScError, match="ratio"):
        Hierarchy(c, f, ratio=3)
    with pytest.raises(B.ScError, match="buffer"):
        Hierarchy(c, f, buffer=3)
    c2, f2 = _levels(32, (8, 8, 8), (40, 40, 40), fine_periodic=7)
    with pytest.raises(B.ScError, match="periodic on no axis"):
        Hierarchy(c2, f2)
    c3, f3 = _levels(32, (8, 8, 8), (40, 40, 40), coarse_periodic=3)
    with pytest.raises(B.ScError, match="periodic on every axis"):
        Hierarchy(c3, f3)
    c4, f4 = _levels(32, (8, 8, 8), (40, 40, 40), fine_h=0.4 / 32)
    with pytest.raises(B.ScError, match="half the coarse"):
        Hierarchy(c4, f4)
    c5, f5 = _levels(32, (8, 8, 8), (16, 40, 40))
    with pytest.raises(B.ScError, match="beyond its buffer"):
        Hierarchy(c5, f5)
    c6, f6 = _levels(32, (2, 8, 8), (40, 40, 40))
    with pytest.raises(B.ScError, match="no coarse box interior"):
        Hierarchy(c6, f6)


def _split(lo, hi, cuts):
    """Boxes of [lo, hi) cut at x = cuts[0] and y = cuts[1]."""
    xs = [lo[0], cuts[0], hi[0]]
    ys = [lo[1], cuts[1], hi[1]]
    return [((xs[i], ys[j], lo[2]), (xs[i + 1], ys[j + 1], hi[2]))
            for i in range(2) for j in range(2)]


@pytest.mark.parametrize("case", [
    dict(n=32, lo=(8, 8, 8), hi=(40, 40, 40), boxes=None, buffer=4),
    dict(n=32, lo=(7, 9, 11), hi=(45, 39, 41), boxes=None, buffer=5),
    dict(n=32, lo=(8, 8, 8), hi=(40, 40, 40), boxes=_split((8, 8, 8), (40, 40, 40), (21, 30)),
         buffer=4),
    dict(n=24, lo=(6, 6, 6), hi=(38, 38, 30), boxes=_split((6, 6, 6), (38, 38, 30), (13, 33)),
         buffer=6),
])
def test_point_sets_match_the_oracle(B, case):
    from paper_1308_1343_gb300.level import Hierarchy
    c, f = _levels(case["n"], case["lo"], case["hi"], case["boxes"])
    h = Hierarchy(c, f, buffer=case["buffer"])
    pp = h.prolongation_points()
    rp = h.restriction_points()
    np_, nr = h.counts()
    assert len(pp) == np_ and len(rp) == nr
    assert len({tuple(p) for p in pp}) == len(pp)  # each target filled once
    want_p = {tuple(int(v) for v in p)
              for p in H.shell_and_buffer(case["lo"], case["hi"], case["buffer"])}
    assert {tuple(int(v) for v in p) for p in pp} == want_p
    t_lo = tuple(v + case["buffer"] for v in case["lo"])
    t_hi = tuple(v - case["buffer"] for v in case["hi"])
    want_r = {tuple(int(v) for v in p) for p in H.restriction_points(t_lo, t_hi)}
    assert {tuple(int(v) for v in p) for p in rp} == want_r
    h.close()


def test_coarse_level_of_several_boxes(B):
    """Targets are split across coarse boxes so that every stencil lies in
    one coarse box's interior; the sets stay the oracle's."""
    from paper_1308_1343_gb300.level import Hierarchy
    n = 32
    cb = [((0, 0, 0), (16, n, n), 0), ((16, 0, 0), (n, n, n), 0)]
    lo, hi = (6, 8, 8), (20, 40, 40)
    c, f = _levels(n, lo, hi, coarse_boxes=cb)
    h = Hierarchy(c, f)
    want = {tuple(int(v) for v in p) for p in H.shell_and_buffer(lo, hi, 4)}
    assert {tuple(int(v) for v in p) for p in h.prolongation_points()} == want
    h.close()
    # a fine region whose stencils straddle the coarse boxes' common face
    lo2, hi2 = (20, 8, 8), (44, 40, 40)
    c2, f2 = _levels(n, lo2, hi2, coarse_boxes=cb)
    with pytest.raises(B.ScError, match="no coarse box interior"):
        Hierarchy(c2, f2)


def test_region_fields_equal_the_whole_fine_grid():
    """The benchmark's inputs, evaluated only on the coarse grid and the fine
    region, are the whole fine grid's values there, bit for bit."""
    from paper_1308_1343_gb300 import workloads as W
    n, lo, hi = 16, (5, 7, 6), (25, 23, 27)
    fine = W.refined_pair(n, 9, lo, hi)
    coarse, (u, pi, c2) = W.refined_fields(n, 9, lo, hi)
    sub = (slice(None, None, 2),) * 3
    reg = (slice(lo[2], hi[2]), slice(lo[1], hi[1]), slice(lo[0], hi[0]))
    assert np.array_equal(fine.u[reg], u) and np.array_equal(fine.c2[reg], c2)
    assert np.array_equal(fine.u[sub], coarse.u) and np.array_equal(fine.c2[sub], coarse.c2)
    assert not np.any(pi) and not np.any(coarse.pi)
