"""Pins of the brute-force point-set algebra against the paper's worked
examples (Sec. 2.2 and Fig. 'derivatives') and the identities it states:
the xor identity of Eq. (xor), commuting derivatives, and recovery of a set
from its derivative by a left-to-right scan."""
import json
import os
import random

import pytest

from oracle import pointset as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "bboxset_examples.json")


def _cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_paper_worked_example_counts(case):
    s = P.union_of_boxes([(lo, hi) for lo, hi in case["boxes"]])
    d = P.full_derivative(s, case["dim"])
    assert len(d) == case["full_derivative_points"]
    if "corner_points" in case:
        assert d == {tuple(p) for p in case["corner_points"]}
    assert P.full_antiderivative(d, case["dim"]) == s


def _random_set(rng, dim, n, nboxes):
    boxes = []
    for _ in range(nboxes):
        lo = [rng.randrange(0, n) for _ in range(dim)]
        hi = [rng.randrange(l + 1, n + 1) for l in lo]
        boxes.append((lo, hi))
    return P.union_of_boxes(boxes)


@pytest.mark.parametrize("seed", range(20))
def test_xor_identity_and_commuting_derivatives(seed):
    rng = random.Random(seed)
    dim = 2 + seed % 2
    R = _random_set(rng, dim, 7, 3)
    S = _random_set(rng, dim, 7, 3)
    assert P.full_derivative(R ^ S, dim) == P.full_derivative(R, dim) ^ P.full_derivative(S, dim)
    assert P.derivative(P.derivative(R, 0), 1) == P.derivative(P.derivative(R, 1), 0)
    assert P.full_antiderivative(P.full_derivative(R, dim), dim) == R
    for a in range(dim):
        assert P.antiderivative(P.derivative(R, a), a) == R


def test_star_ghost_count():
    # ghost width 2 on each of the 6 faces: 2*2*(nx*ny + ny*nz + nx*nz)
    g = P.star_ghosts((0, 0, 0), (5, 4, 3))
    assert len(g) == 4 * (5 * 4 + 4 * 3 + 5 * 3)
