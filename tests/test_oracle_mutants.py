"""Planted mistakes: each test compiles a copy of the oracle with one
plausible error (a dropped term, a wrong sign, a wrong index, an operand on
the wrong side) and checks that one of the oracle's pins rejects it, while
the unmodified oracle passes the same pin.  Everything runs on the CPU."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1308_1343_gb300 import workloads as W

SRC = os.path.join(os.path.dirname(O.__file__), "oracle.c")


def _sigma(t):
    return (15.0 - 16.0 * np.cos(t) + np.cos(2 * t)) / 6.0


def pin_plane_wave_eigen():
    inst = W.plane_wave(16)
    h = inst.dom.h
    mu = sum(_sigma(2 * np.pi * k * h) for k in (1, 2, 3)) / h ** 2
    return np.abs(O.lap_periodic(inst.u, h) + mu * inst.u).max() <= 1e-12 * mu


def pin_padded_poly():
    n, h = 6, 0.1
    g = h * np.arange(-2, n + 2)
    X, Y, Z = np.meshgrid(g, g, g, indexing="xy")
    f = X ** 5 - 2 * Y ** 4 * X + Z ** 3 * Y ** 2 + X * Y * Z
    lap = 20 * X ** 3 - 24 * Y ** 2 * X + 2 * Z ** 3 + 6 * Z * Y ** 2
    t = lambda a: np.ascontiguousarray(np.transpose(a, (2, 0, 1)))
    got = O.lap_padded(t(f), h)
    return np.abs(got - t(lap)[2:-2, 2:-2, 2:-2]).max() <= 1e-9


def pin_rk4_closed_form():
    inst = W.plane_wave(16)
    h, dt = inst.dom.h, inst.dt
    mu = sum(_sigma(2 * np.pi * k * h) for k in (1, 2, 3)) / h ** 2
    z2 = dt * dt * mu
    a, b = 1 - z2 / 2 + z2 * z2 / 24, 1 - z2 / 6
    M = np.array([[a, b * dt], [-b * dt * mu, a]])
    ab = np.linalg.matrix_power(M, 5) @ np.array([1.0, 0.0])
    u, pi = O.rk4_periodic(inst.u, inst.pi, inst.c2, h, dt, 5)
    return (np.abs(u - ab[0] * inst.u).max() <= 1e-12 and
            np.abs(pi - ab[1] * inst.u).max() <= 1e-12 * abs(ab[1]))


def pin_dot_identity():
    inst = W.gradient_problem(8, 4)
    sh = inst.dom.shape
    r = lambda s: np.random.default_rng(s).normal(size=sh)
    du, dc2, bu, bpi = r(1), r(2), r(3), r(4)
    _, _, tu, tp = O.tlm_periodic(inst.u, inst.pi, inst.c2, du, np.zeros(sh), dc2,
                                  inst.dom.h, inst.dt, 3)
    gu, gp, gc = O.grad_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, 3, 2, bu, bpi)
    lhs = np.sum(tu * bu) + np.sum(tp * bpi)
    rhs = np.sum(du * gu) + np.sum(dc2 * gc)
    return abs(lhs - rhs) <= 1e-12 * abs(lhs)


def pin_tlm_fd():
    inst = W.gradient_problem(8, 4)
    sh = inst.dom.shape
    dc2 = W.random_direction(sh, 40)
    eps = 1e-5
    _, _, tu, _ = O.tlm_periodic(inst.u, inst.pi, inst.c2, np.zeros(sh), np.zeros(sh), dc2,
                                 inst.dom.h, inst.dt, 3)
    up, _ = O.rk4_periodic(inst.u, inst.pi, inst.c2 + eps * dc2, inst.dom.h, inst.dt, 3)
    um, _ = O.rk4_periodic(inst.u, inst.pi, inst.c2 - eps * dc2, inst.dom.h, inst.dt, 3)
    return np.abs((up - um) / (2 * eps) - tu).max() <= 1e-6 * np.abs(tu).max()


def pin_ghosts_wrap():
    n = (24, 16, 16)
    boxes = W.bisect_boxes(n, 2, 3)
    g = np.random.default_rng(0).normal(size=(n[2], n[1], n[0]))
    f = []
    for lo, hi in boxes:
        a = np.full((hi[2] - lo[2] + 4, hi[1] - lo[1] + 4, hi[0] - lo[0] + 4), np.nan)
        a[2:-2, 2:-2, 2:-2] = g[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        f.append(a)
    O.fill_ghosts([lo + hi for lo, hi in boxes], (0, 0, 0) + n, 7, f)
    ref = np.pad(g, 2, mode="wrap")
    for (lo, hi), a in zip(boxes, f):
        sub = ref[lo[2]:hi[2] + 4, lo[1]:hi[1] + 4, lo[0]:hi[0] + 4]
        m = np.zeros(a.shape, bool)
        m[2:-2, 2:-2, :] = m[2:-2, :, 2:-2] = m[:, 2:-2, 2:-2] = True
        if not np.array_equal(a[m], sub[m]):
            return False
    return True


MUTANTS = [
    ("drop x+2 term", "+ 16.0 * U(i + 1, j, k) - U(i + 2, j, k);",
     "+ 16.0 * U(i + 1, j, k);", pin_plane_wave_eigen),
    ("z+2 wrong sign", "+ 16.0 * U(i, j, k + 1) - U(i, j, k + 2);",
     "+ 16.0 * U(i, j, k + 1) + U(i, j, k + 2);", pin_plane_wave_eigen),
    ("padded y index swapped", "+ 16.0 * P(i, j + 1, k) - P(i, j + 2, k);",
     "+ 16.0 * P(i + 1, j, k) - P(i, j + 2, k);", pin_padded_poly),
    ("wrong RK weight", "2.0 * Ku[2][i] + Ku[3][i]) / 6.0",
     "1.0 * Ku[2][i] + Ku[3][i]) / 6.0", pin_rk4_closed_form),
    ("wrong RK node", "{0.0, 0.5, 0.5, 1.0}", "{0.0, 0.5, 1.0, 1.0}", pin_rk4_closed_form),
    ("c2 dropped in A^T", "t[i] = c2[i] * Kbp[s][i];", "t[i] = Kbp[s][i];", pin_dot_identity),
    ("c2 adjoint uses wrong stage", "bc2[i] += Kbp[s][i] * lapU[s][i];",
     "bc2[i] += Kbp[s][i] * lapU[3 - s][i];", pin_dot_identity),
    ("tangent misses dc2 term", "dKp[s][i] = c2[i] * dlap[i] + dc2[i] * lap[i];",
     "dKp[s][i] = c2[i] * dlap[i];", pin_tlm_fd),
    ("ghost owner off by one", "q[d] = dom[d] + wrap(p[d] - dom[d], len);",
     "q[d] = dom[d] + wrap(p[d] - dom[d] + 1, len);", pin_ghosts_wrap),
]


@pytest.mark.parametrize("name,old,new,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_rejects_planted_mistake(tmp_path, name, old, new, pin):
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    assert pin(), "unmodified oracle must pass " + pin.__name__
    lib = O.compile_variant(src.replace(old, new), str(tmp_path / "mutant.so"))
    with O.using_library(lib):
        assert not pin(), "pin %s did not catch: %s" % (pin.__name__, name)
