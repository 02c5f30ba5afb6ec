"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test checks the oracle against mathematics it does not itself encode:
polynomial exactness and the leading truncation error of the 4th-order
stencil, the exact discrete eigenvalue of a plane wave, the closed-form RK4
amplification matrix and energy factor, 4th-order convergence to the
continuum solution, numpy's periodic padding, the identities a correct
adjoint must satisfy (dot tests against the independent tangent-linear code,
central finite differences, exact quadratic dependence on u0), and
invariances (checkpoint interval, thread count).
"""
import math

import numpy as np
import pytest

from paper_1308_1343_gb300 import workloads as W


# ----------------------------------------------------------------------------
# Stencil
# ----------------------------------------------------------------------------

def _padded_grid(n, h, origin):
    nx, ny, nz = n
    x = origin[0] + h * np.arange(-2, nx + 2)
    y = origin[1] + h * np.arange(-2, ny + 2)
    z = origin[2] + h * np.arange(-2, nz + 2)
    return np.meshgrid(x, y, z, indexing="xy")  # shapes (ny+4, nx+4, nz+4)


def _to_zyx(a):
    return np.ascontiguousarray(np.transpose(a, (2, 0, 1)))


def _random_poly(rng, deg):
    """Random polynomial sum c_abc x^a y^b z^c with a+b+c <= deg."""
    terms = [(a, b, c) for a in range(deg + 1) for b in range(deg + 1)
             for c in range(deg + 1) if a + b + c <= deg]
    coef = rng.normal(size=len(terms))
    return list(zip(terms, coef))


def _eval_poly(terms, X, Y, Z):
    return sum(c * X ** a * Y ** b * Z ** e for (a, b, e), c in terms)


def _eval_lap(terms, X, Y, Z):
    out = np.zeros_like(X)
    for (a, b, e), c in terms:
        if a >= 2:
            out += c * a * (a - 1) * X ** (a - 2) * Y ** b * Z ** e
        if b >= 2:
            out += c * b * (b - 1) * X ** a * Y ** (b - 2) * Z ** e
        if e >= 2:
            out += c * e * (e - 1) * X ** a * Y ** b * Z ** (e - 2)
    return out


@pytest.mark.parametrize("seed", range(6))
def test_stencil_exact_on_degree_5_polynomials(orc, seed):
    rng = np.random.default_rng(seed)
    n = (9, 7, 6)
    h = 0.1
    terms = _random_poly(rng, 5)
    X, Y, Z = _padded_grid(n, h, rng.uniform(-0.5, 0.5, size=3))
    up = _to_zyx(_eval_poly(terms, X, Y, Z))
    got = orc.lap_padded(up, h)
    want = _to_zyx(_eval_lap(terms, X, Y, Z))[2:-2, 2:-2, 2:-2]
    scale = max(1.0, np.abs(want).max())
    assert np.abs(got - want).max() <= 1e-10 * scale


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_stencil_sixth_power_error_is_minus_8_h4(orc, axis):
    # For f = s^6 the Taylor series of the 4th-order centred second
    # difference stops after the h^4 term: L f - f'' = -h^4 f^(6) / 90 = -8 h^4.
    n = (6, 6, 6)
    h = 0.125
    X, Y, Z = _padded_grid(n, h, (0.3, -0.2, 0.1))
    S = (X, Y, Z)[axis]
    up = _to_zyx(S ** 6)
    got = orc.lap_padded(up, h)
    exact = _to_zyx(30.0 * S ** 4)[2:-2, 2:-2, 2:-2]
    err = got - exact
    assert np.allclose(err, -8.0 * h ** 4, rtol=0, atol=1e-9)


def test_stencil_single_axis_weights(orc):
    # A unit impulse reveals the stencil weights directly: (L delta) at offset
    # +-1 is 16/(12 h^2), at +-2 is -1/(12 h^2), at 0 is -90/(12 h^2).
    n = 11
    h = 0.5
    u = np.zeros((n, n, n))
    u[5, 5, 5] = 1.0
    L = orc.lap_periodic(u, h) * (12 * h * h)
    assert L[5, 5, 5] == -90.0
    for d in range(3):
        for off, w in ((1, 16.0), (2, -1.0)):
            for sgn in (-1, 1):
                idx = [5, 5, 5]
                idx[d] += sgn * off
                assert L[tuple(idx)] == w
    assert np.count_nonzero(L) == 13


def test_periodic_laplacian_equals_padded_with_wrap(orc):
    rng = np.random.default_rng(7)
    u = rng.normal(size=(10, 9, 12))
    a = orc.lap_periodic(u, 0.3)
    b = orc.lap_padded(np.pad(u, 2, mode="wrap"), 0.3)
    assert np.array_equal(a, b)


def _sigma(theta):
    return (15.0 - 16.0 * np.cos(theta) + np.cos(2 * theta)) / 6.0


def test_plane_wave_is_discrete_eigenvector(orc):
    inst = W.plane_wave(24)
    h = inst.dom.h
    k = 2 * np.pi * np.array([1.0, 2.0, 3.0])
    mu = sum(_sigma(kd * h) for kd in k) / h ** 2
    got = orc.lap_periodic(inst.u, h)
    assert np.abs(got + mu * inst.u).max() <= 1e-12 * mu


def test_laplacian_symmetric(orc):
    rng = np.random.default_rng(3)
    u = rng.normal(size=(8, 10, 9))
    v = rng.normal(size=(8, 10, 9))
    a = np.sum(orc.lap_periodic(u, 0.2) * v)
    b = np.sum(u * orc.lap_periodic(v, 0.2))
    assert abs(a - b) <= 1e-12 * np.sum(np.abs(orc.lap_periodic(u, 0.2) * v))


# ----------------------------------------------------------------------------
# RK4 closed forms
# ----------------------------------------------------------------------------

def _rk4_matrix(z2, dt):
    alpha = 1 - z2 / 2 + z2 * z2 / 24
    beta = 1 - z2 / 6
    mu = z2 / dt ** 2
    return np.array([[alpha, beta * dt], [-beta * dt * mu, alpha]])


@pytest.mark.parametrize("n,steps", [(16, 10), (32, 20)])
def test_rk4_plane_wave_closed_form(orc, n, steps):
    inst = W.plane_wave(n)
    h, dt = inst.dom.h, inst.dt
    k = 2 * np.pi * np.array([1.0, 2.0, 3.0])
    mu = sum(_sigma(kd * h) for kd in k) / h ** 2
    M = _rk4_matrix(dt * dt * mu, dt)
    ab = np.linalg.matrix_power(M, steps) @ np.array([1.0, 0.0])
    u, pi = orc.rk4_periodic(inst.u, inst.pi, inst.c2, h, dt, steps)
    s = inst.u
    assert np.abs(u - ab[0] * s).max() <= 1e-12 * np.abs(ab[0] * s).max() + 1e-13
    assert np.abs(pi - ab[1] * s).max() <= 1e-12 * np.abs(ab[1] * s).max()


def test_rk4_energy_factor(orc):
    # For a single mode, RK4 scales the discrete energy by exactly
    # 1 - z^6/72 + z^8/576 per step, z^2 = dt^2 mu.
    inst = W.plane_wave(32)
    h, dt = inst.dom.h, inst.dt
    k = 2 * np.pi * np.array([1.0, 2.0, 3.0])
    mu = sum(_sigma(kd * h) for kd in k) / h ** 2
    z2 = dt * dt * mu
    f = 1 - z2 ** 3 / 72 + z2 ** 4 / 576
    e0 = orc.energy(inst.u, inst.pi, inst.c2, h)
    u, pi = orc.rk4_periodic(inst.u, inst.pi, inst.c2, h, dt, 20)
    e20 = orc.energy(u, pi, inst.c2, h)
    assert abs(e20 / e0 - f ** 20) <= 1e-12
    assert 1 - f ** 20 > 1e-6  # the decay is far above rounding


def test_energy_non_increasing_variable_c2(orc):
    inst = W.single_box(32, seed=2)
    h, dt = inst.dom.h, inst.dt
    u, pi = inst.u, inst.pi
    e_prev = orc.energy(u, pi, inst.c2, h)
    for _ in range(5):
        u, pi = orc.rk4_periodic(u, pi, inst.c2, h, dt, 2)
        e = orc.energy(u, pi, inst.c2, h)
        assert e <= e_prev * (1 + 1e-14)
        e_prev = e
    assert e_prev > 0


def test_fourth_order_convergence(orc):
    # continuum: u = sin(k.x) cos(w t), w = 2 pi sqrt(14); fixed T = 0.15625
    T = 20 * 0.25 / 32
    errs = {}
    for n in (16, 32, 64):
        inst = W.plane_wave(n)
        steps = int(round(T / inst.dt))
        u, _ = orc.rk4_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, steps)
        exact = inst.u * math.cos(2 * math.pi * math.sqrt(14.0) * T)
        errs[n] = np.abs(u - exact).max()
    ratio = errs[32] / errs[64]
    assert 14.0 <= ratio <= 18.0, (errs, ratio)


def test_thread_count_bit_identical(orc):
    if not orc.has_openmp():
        pytest.skip("oracle built without OpenMP")
    inst = W.single_box(20, seed=9)
    orc.set_threads(1)
    a = orc.rk4_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, 3)
    orc.set_threads(4)
    b = orc.rk4_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, 3)
    orc.set_threads(1)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


# ----------------------------------------------------------------------------
# Ghost exchange
# ----------------------------------------------------------------------------

def _scatter(glob, boxes, poison=np.nan):
    out = []
    for lo, hi in boxes:
        f = np.full((hi[2] - lo[2] + 4, hi[1] - lo[1] + 4, hi[0] - lo[0] + 4), poison)
        f[2:-2, 2:-2, 2:-2] = glob[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        out.append(f)
    return out


def _star_mask(shape):
    nz, ny, nx = (s - 4 for s in shape)
    m = np.zeros(shape, dtype=bool)
    m[2:-2, 2:-2, :] = True
    m[2:-2, :, 2:-2] = True
    m[:, 2:-2, 2:-2] = True
    m[2:-2, 2:-2, 2:-2] = False
    return m


def test_single_box_ghosts_equal_numpy_wrap(orc):
    rng = np.random.default_rng(1)
    g = rng.normal(size=(6, 7, 9))
    n = (9, 7, 6)
    f = _scatter(g, [((0, 0, 0), n)])
    orc.fill_ghosts([(0, 0, 0) + n], (0, 0, 0) + n, 7, f)
    ref = np.pad(g, 2, mode="wrap")
    m = _star_mask(f[0].shape)
    assert np.array_equal(f[0][m], ref[m])
    # edges and corners of the padded box are not ghosts and stay untouched
    inner = np.zeros_like(m)
    inner[2:-2, 2:-2, 2:-2] = True
    assert np.all(np.isnan(f[0][~m & ~inner]))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_multibox_ghosts_equal_wrapped_global(orc, seed):
    n = (48, 40, 32)
    boxes = W.bisect_boxes(n, 3, seed)
    rng = np.random.default_rng(seed)
    g = rng.normal(size=(n[2], n[1], n[0]))
    f = _scatter(g, boxes)
    orc.fill_ghosts([lo + hi for lo, hi in boxes], (0, 0, 0) + n, 7, f)
    ref = np.pad(g, 2, mode="wrap")
    for (lo, hi), fb in zip(boxes, f):
        m = _star_mask(fb.shape)
        sub = ref[lo[2]:hi[2] + 4, lo[1]:hi[1] + 4, lo[0]:hi[0] + 4]
        assert np.array_equal(fb[m], sub[m])


def test_ghost_owner_rows(orc):
    from oracle import pointset as P
    n = (24, 16, 16)
    boxes = W.bisect_boxes(n, 2, 11)
    rows = orc.ghost_owners([lo + hi for lo, hi in boxes], (0, 0, 0) + n, 7)
    want = sum(len(P.star_ghosts(lo, hi)) for lo, hi in boxes)
    assert len(rows) == want
    N = np.array(n)
    assert np.array_equal(rows[:, 5:8], rows[:, 1:4] % N)
    for r in rows[:: max(1, len(rows) // 500)]:
        lo, hi = boxes[r[4]]
        assert all(lo[d] <= r[5 + d] < hi[d] for d in range(3))
        dlo, dhi = boxes[r[0]]
        assert not all(dlo[d] <= r[1 + d] < dhi[d] for d in range(3))


def test_nonperiodic_ghosts_without_owner_untouched(orc):
    n = (8, 8, 8)
    g = np.arange(512, dtype=np.float64).reshape(8, 8, 8)
    f = _scatter(g, [((0, 0, 0), n)])
    orc.fill_ghosts([(0, 0, 0) + n], (0, 0, 0) + n, 0, f)
    assert np.all(np.isnan(f[0][_star_mask(f[0].shape)]))
