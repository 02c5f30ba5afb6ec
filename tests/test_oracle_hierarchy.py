"""Pins of the two-level hierarchy oracle (oracle/hierarchy.py) against what
mathematics fixes: cubic Lagrange interpolation reproduces cubics and not
quartics; time interpolation is linear; the prolongation and restriction
sets follow their definitions; one Berger-Oliger step equals the
single-level runs bit for bit wherever its dependence cone stays in data
the scheme maintains; and the two-level solution converges."""
import math

import numpy as np
import pytest

from exact_sums import tensor_sum_exact
from oracle import hierarchy as H
from paper_1308_1343_gb300 import workloads as W


def test_stencil_reproduces_cubics_not_quartics():
    for f in range(-7, 9):
        idx, w = H.stencil_1d(f)
        assert abs(sum(w) - 1.0) == 0.0
        for deg in range(4):
            got = sum(wi * float(c) ** deg for c, wi in zip(idx, w))
            assert got == (f / 2.0) ** deg, (f, deg)
        if f % 2:
            got = sum(wi * float(c) ** 4 for c, wi in zip(idx, w))
            assert got != (f / 2.0) ** 4
            # x^4 minus its cubic interpolant at the midpoint of nodes -1, 0, 1, 2
            # is (1.5)(0.5)(-0.5)(-1.5) = 9/16 (unit spacing, x^4's 4th derivative / 4! = 1)
            assert got - (f / 2.0) ** 4 == -9.0 / 16.0


def _poly(coef, x, y, z):
    out = np.zeros(np.broadcast(x, y, z).shape)
    for (i, j, k), a in coef.items():
        out = out + a * x ** i * y ** j * z ** k
    return out


def test_prolongation_exact_for_tensor_cubics():
    rng = np.random.default_rng(7)
    coef = {(i, j, k): rng.normal() for i in range(4) for j in range(4) for k in range(4)}
    n = 16
    z, y, x = np.meshgrid(*[np.arange(n, dtype=float)] * 3, indexing="ij")
    coarse = _poly(coef, x, y, z)
    pts = H.shell_and_buffer((8, 8, 8), (22, 22, 22), 4)
    got = H.prolongate(coarse, coarse, 0.0, pts)
    want = _poly(coef, pts[:, 0] / 2.0, pts[:, 1] / 2.0, pts[:, 2] / 2.0)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    # a quartic term along x is not reproduced at odd x indices
    coef[(4, 0, 0)] = 1.0
    coarse4 = _poly(coef, x, y, z)
    got4 = H.prolongate(coarse4, coarse4, 0.0, pts)
    want4 = _poly(coef, pts[:, 0] / 2.0, pts[:, 1] / 2.0, pts[:, 2] / 2.0)
    err = np.abs(got4 - want4)
    odd_x = pts[:, 0] % 2 == 1
    assert err[odd_x].min() > 0.1 and err[~odd_x].max() <= 1e-9 * np.abs(want4).max()


def test_time_interpolation_is_linear():
    rng = np.random.default_rng(3)
    a, b = rng.normal(size=(2, 12, 12, 12))
    pts = H.shell_and_buffer((6, 6, 6), (18, 18, 18), 4)
    pa = H.prolongate(a, a, 0.0, pts)
    pb = H.prolongate(b, b, 0.0, pts)
    assert np.array_equal(H.prolongate(a, b, 0.0, pts), pa)
    assert np.array_equal(H.prolongate(a, b, 1.0, pts), pb)
    half = H.prolongate(a, b, 0.5, pts)
    assert np.abs(half - 0.5 * (pa + pb)).max() <= 1e-14 * np.abs(pa).max()


def test_prolongation_nested_equals_exact_tensor_sum():
    """The oracle's successive 1-D interpolations equal the tensor-product sum
    rounded once: exactly for dyadic data (every product and partial sum is
    then exact in FP64, in any evaluation order), and within a few ulps of
    the data's scale otherwise.  A wrong weight, a wrong index, or a stencil
    applied along the wrong axis fails the exact case."""
    rng = np.random.default_rng(17)
    pts = H.shell_and_buffer((6, 6, 6), (18, 18, 18), 4)[::7]
    dyadic = rng.integers(-2 ** 20, 2 ** 20, size=(12, 12, 12)).astype(np.float64)
    got = H.prolongate(dyadic, dyadic, 0.0, pts)
    want = np.array([tensor_sum_exact(dyadic, p) for p in pts])
    assert np.array_equal(got, want)
    # x, y and z are not interchangeable: a transposed copy gives other values
    assert not np.array_equal(H.prolongate(dyadic.transpose(2, 1, 0).copy(),
                                           dyadic.transpose(2, 1, 0).copy(), 0.0, pts), want)
    data = rng.normal(size=(12, 12, 12))
    got = H.prolongate(data, data, 0.0, pts)
    want = np.array([tensor_sum_exact(data, p) for p in pts])
    assert np.abs(got - want).max() <= 4 * np.finfo(float).eps * np.abs(data).max()


def test_prolongation_and_restriction_sets():
    lo, hi, B = (3, 5, 7), (17, 16, 19), 4
    pts = H.shell_and_buffer(lo, hi, B)
    n = np.array(hi) - np.array(lo)
    inner = np.prod(n - 2 * B)
    shell = 2 * 2 * (n[0] * n[1] + n[1] * n[2] + n[0] * n[2])
    assert len(pts) == np.prod(n) - inner + shell
    assert len({tuple(p) for p in pts}) == len(pts)
    for p in pts:
        out = [(p[d] < lo[d]) or (p[d] >= hi[d]) for d in range(3)]
        far = [(p[d] < lo[d] - 2) or (p[d] >= hi[d] + 2) for d in range(3)]
        assert sum(out) <= 1 and not any(far)
        if not any(out):
            assert any(p[d] < lo[d] + B or p[d] >= hi[d] - B for d in range(3))
    t_lo, t_hi = (3, 4, 5), (10, 9, 12)
    rp = H.restriction_points(t_lo, t_hi)
    want = {(x, y, z) for x in range(-3, 12) for y in range(-3, 12) for z in range(-3, 12)
            if all(t_lo[d] <= 2 * (x, y, z)[d] < t_hi[d] for d in range(3))}
    assert {tuple(int(v) for v in p) for p in rp} == want


def _bumpy_pair(n_coarse, seed):
    fine = W.bumpy_instance(W.Domain((2 * n_coarse,) * 3, 0.5 / n_coarse), seed)
    sub = (slice(None, None, 2),) * 3
    return fine, fine.u[sub].copy(), fine.pi[sub].copy(), fine.c2[sub].copy()


def _pad_region(a, lo, hi):
    return a[lo[2] - 2:hi[2] + 2, lo[1] - 2:hi[1] + 2, lo[0] - 2:hi[0] + 2].copy()


def test_one_step_equals_single_level_runs_where_cones_stay_trusted(orc):
    n = 32
    fine, cu, cpi, cc2 = _bumpy_pair(n, 12)
    h = 1.0 / n
    dt = 0.25 * h
    lo, hi, B = (8, 8, 8), (56, 56, 56), 4
    fu = _pad_region(fine.u, lo, hi)
    fp = _pad_region(fine.pi, lo, hi)
    fc = _pad_region(fine.c2, lo, hi)
    cu1, cp1, fu1, fp1 = H.bo_step(cu, cpi, cc2, h, dt, fu, fp, fc, lo, hi, B)
    # coarse points not covered by the trusted region: the coarse-only step
    ru, rp = orc.rk4_periodic(cu, cpi, cc2, h, dt, 1)
    covered = np.zeros(cu.shape, bool)
    for cx, cy, cz in H.restriction_points((12,) * 3, (52,) * 3):
        covered[cz, cy, cx] = True
    assert covered.sum() == 20 ** 3
    assert np.array_equal(cu1[~covered], ru[~covered])
    assert np.array_equal(cp1[~covered], rp[~covered])
    # fine points farther than 2 x 4 from the buffer: two steps of the
    # periodic fine grid, bit for bit
    gu, gp = orc.rk4_periodic(fine.u, fine.pi, fine.c2, h / 2, dt / 2, 2)
    deep = (slice(20 - lo[2] + 2, 44 - lo[2] + 2),) * 3
    assert np.array_equal(fu1[deep], gu[20:44, 20:44, 20:44])
    assert np.array_equal(fp1[deep], gp[20:44, 20:44, 20:44])
    # restriction: covered coarse points carry the fine values at 2c
    assert np.array_equal(cu1[covered], fu1[2:-2:2, 2:-2:2, 2:-2:2][2:-2, 2:-2, 2:-2].ravel())
    # the prolongation-filled band holds values close to the fine grid's
    shell = H.shell_and_buffer(lo, hi, B)
    assert len(shell) > 0


def _plane_wave_errors(n, coarse_steps):
    fine = W.plane_wave(2 * n)
    sub = (slice(None, None, 2),) * 3
    cu, cpi, cc2 = fine.u[sub].copy(), fine.pi[sub].copy(), fine.c2[sub].copy()
    h = 1.0 / n
    dt = 0.25 * h
    lo, hi = (n // 2,) * 3, (3 * n // 2,) * 3
    fu, fp, fc = (_pad_region(a, lo, hi) for a in (fine.u, fine.pi, fine.c2))
    for _ in range(coarse_steps):
        cu, cpi, fu, fp = H.bo_step(cu, cpi, cc2, h, dt, fu, fp, fc, lo, hi, 4)
    t = coarse_steps * dt
    w = 2 * np.pi * np.sqrt(14.0)
    ec = np.abs(cu - fine.u[sub] * np.cos(w * t)).max()
    tl, th = n // 2 + 4, 3 * n // 2 - 4
    s = (slice(tl - lo[0] + 2, th - lo[0] + 2),) * 3
    ef = np.abs(fu[s] - fine.u[tl:th, tl:th, tl:th] * np.cos(w * t)).max()
    return ec, ef


def test_two_level_plane_wave_converges():
    """T = 0.0625 (4 coarse steps at 16^3, 8 at 32^3): the error of both
    levels falls at least 4x per halving of h (the boundary data's linear
    time interpolation is second order; the interior scheme fourth)."""
    e16 = _plane_wave_errors(16, 4)
    e32 = _plane_wave_errors(32, 8)
    assert all(np.isfinite(e16)) and all(np.isfinite(e32))
    assert e32[0] < e16[0] / 4.0
    assert e32[1] < e16[1] / 4.0


def test_planted_mistakes_are_caught(monkeypatch, orc):
    """Two plausible mistakes, planted in the oracle on the CPU, each fail a
    pin above: symmetric weights that sum to 1 but are not the cubic
    interpolant's, and restriction from the neighbouring fine point."""
    monkeypatch.setattr(H, "W_ODD", (-2.0 / 16.0, 10.0 / 16.0, 10.0 / 16.0, -2.0 / 16.0))
    with pytest.raises(AssertionError):
        test_prolongation_exact_for_tensor_cubics()
    monkeypatch.undo()
    real = H.restriction_points
    monkeypatch.setattr(H, "restriction_points",
                        lambda lo, hi: real((lo[0] + 1,) + tuple(lo[1:]), (hi[0] + 1,) + tuple(hi[1:])))
    with pytest.raises(AssertionError):
        test_one_step_equals_single_level_runs_where_cones_stay_trusted(orc)
