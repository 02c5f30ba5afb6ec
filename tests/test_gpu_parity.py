"""GPU parity of the CUDA path against the CPU oracle, through the C ABI.

Bars: ghost copies bit-exact; u and pi within 1e-12 relative max norm of
the oracle after the stated steps; decomposition independence and the three
launch modes bit-identical; full-size checks on the 256^3 and 512x512x256
workloads in the benchmark's launch configuration (graph mode)."""
import os

import numpy as np
import pytest

from paper_1308_1343_gb300 import workloads as W

from gpu_helpers import make_level, rel_err, run_gpu, upload

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1308_1343_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def B():
    from paper_1308_1343_gb300 import binding
    return binding


def _sigma(t):
    return (15.0 - 16.0 * np.cos(t) + np.cos(2 * t)) / 6.0


# ----------------------------------------------------------------------------
# ghost exchange
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("levels", [0, 2, 4])
def test_fill_ghosts_bit_exact(orc, levels):
    import torch
    n = (40, 36, 24)
    boxes = W.bisect_boxes(n, levels, 11)
    inst = W.Instance(W.Domain(n, 0.1), np.zeros(1), np.zeros(1), np.zeros(1), 0.1,
                      boxes=boxes)
    lev = make_level([inst])
    g = np.random.default_rng(levels).normal(size=(n[2], n[1], n[0]))
    f = lev.to_device([g], fill=np.nan)
    lev.fill_ghosts(f)
    torch.cuda.synchronize()
    got = lev.padded_boxes(f)
    want = lev.padded_boxes(lev.scatter([g], fill=np.nan))
    orc.fill_ghosts([lo + hi for lo, hi in boxes], (0, 0, 0) + n, 7, want)
    for a, b in zip(got, want):
        assert np.array_equal(a, b, equal_nan=True)


# ----------------------------------------------------------------------------
# Laplacian: polynomial exactness and oracle parity, both arithmetic forms
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("arith", [0, 1])
def test_laplacian_polynomial_exact(orc, arith):
    import torch
    from paper_1308_1343_gb300.level import Level
    nx, ny, nz = 37, 19, 13  # ragged against every tile shape
    h = 0.1
    lev = Level([((0, 0, 0), (nx, ny, nz), 0)], [dict(hi=(nx, ny, nz), h=h, periodic=0)])
    lev.set_arith(arith)
    x = h * np.arange(-2, nx + 2) - 0.3
    y = h * np.arange(-2, ny + 2) + 0.2
    z = h * np.arange(-2, nz + 2) - 0.1
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    f = X ** 5 - 2 * Y ** 4 * X + Z ** 3 * Y ** 2 + X * Y * Z + 3.0
    lap = 20 * X ** 3 - 24 * Y ** 2 * X + 2 * Z ** 3 + 6 * Z * Y ** 2
    buf = np.full(lev.field_size, np.nan)
    lev._box_view(buf, 0)[:] = f
    u = torch.from_numpy(buf).cuda()
    out = lev.new_field(np.nan)
    lev.apply_laplacian(u, out)
    lev.sync()
    got = lev.gather(out)[0]
    want = lap[2:-2, 2:-2, 2:-2]
    assert np.abs(got - want).max() <= 1e-9 * np.abs(want).max()
    # two FP64 evaluation orders of the same 13-term sum differ by at most a
    # few units of rounding of the sum of |terms|: bound 32 eps sum|w u|/(12h^2)
    ref = orc.lap_padded(f, h)
    A = np.abs(f)
    c = (slice(2, -2),) * 3
    s_abs = 90 * A[c]
    for ax in range(3):
        for off, w in ((1, 16), (2, 1)):
            for sgn in (-1, 1):
                sl = [slice(2, -2)] * 3
                sl[ax] = slice(2 + sgn * off, A.shape[ax] - 2 + sgn * off)
                s_abs = s_abs + w * A[tuple(sl)]
    bound = 32 * np.finfo(float).eps * s_abs / (12 * h * h)
    if arith == 1:
        # fixed-point form: each input is truncated to the grid 2^-S <= 2^-54 M
        # (M = max |u| over the values read), i.e. an absolute error below
        # 2^-54 M per input, 192 M 2^-54 for the weighted sum
        M = np.abs(f[2:-2, 2:-2, :]).max()
        M = max(M, np.abs(f[2:-2, :, 2:-2]).max(), np.abs(f[:, 2:-2, 2:-2]).max())
        bound = bound + 192 * 2.0 ** -54 * M / (12 * h * h)
    assert np.all(np.abs(got - ref) <= bound)


# ----------------------------------------------------------------------------
# RK4 parity
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("arith", [0, 1])
def test_plane_wave_32_twenty_steps(orc, arith):
    inst = W.plane_wave(32)
    _, u, pi = run_gpu([inst], 20, arith, 0)
    ou, op = orc.rk4_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, 20)
    assert rel_err(u[0], ou) <= TOL
    assert rel_err(pi[0], op) <= TOL
    h, dt = inst.dom.h, inst.dt
    mu = sum(_sigma(2 * np.pi * k * h) for k in (1, 2, 3)) / h ** 2
    z2 = dt * dt * mu
    a, b = 1 - z2 / 2 + z2 * z2 / 24, 1 - z2 / 6
    M = np.array([[a, b * dt], [-b * dt * mu, a]])
    ab = np.linalg.matrix_power(M, 20) @ np.array([1.0, 0.0])
    assert rel_err(u[0], ab[0] * inst.u) <= TOL
    assert rel_err(pi[0], ab[1] * inst.u) <= TOL


@pytest.mark.parametrize("arith", [0, 1])
def test_ragged_bumpy_box_all_modes(orc, arith):
    dom = W.Domain((40, 36, 28), 1.0 / 36)
    inst = W.bumpy_instance(dom, 2)
    ou, op = orc.rk4_periodic(inst.u, inst.pi, inst.c2, dom.h, inst.dt, 6)
    res = {}
    for mode in (0, 1, 2):
        _, u, pi = run_gpu([inst], 6, arith, mode)
        assert rel_err(u[0], ou) <= TOL, mode
        assert rel_err(pi[0], op) <= TOL, mode
        res[mode] = (u[0], pi[0])
    for mode in (1, 2):
        assert np.array_equal(res[mode][0], res[0][0])
        assert np.array_equal(res[mode][1], res[0][1])


@pytest.mark.parametrize("arith", [0, 1])
def test_uneven_level_matches_oracle_and_single_box(orc, arith):
    inst = W.uneven_level(n=(128, 128, 64), h=1.0 / 64, levels=6, seed=3, box_seed=30)
    assert len(inst.boxes) == 64
    ou, op = orc.rk4_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, 4)
    _, u, pi = run_gpu([inst], 4, arith, 0)
    assert rel_err(u[0], ou) <= TOL
    assert rel_err(pi[0], op) <= TOL
    one = W.Instance(inst.dom, inst.u, inst.pi, inst.c2, inst.dt)
    _, u1, p1 = run_gpu([one], 4, arith, 0)
    assert np.array_equal(u[0], u1[0]) and np.array_equal(pi[0], p1[0])
    _, u2, p2 = run_gpu([inst], 4, arith, 1)
    assert np.array_equal(u[0], u2[0]) and np.array_equal(pi[0], p2[0])


@pytest.mark.parametrize("arith", [0, 1])
def test_ensemble_per_domain_dt(orc, arith):
    insts = [W.bumpy_instance(W.Domain((n, n, n), 1.0 / n), 5000 + i)
             for i, n in enumerate((24, 32, 40, 24, 56, 48))]
    _, u, pi = run_gpu(insts, 5, arith, 0)
    for i, inst in enumerate(insts):
        ou, op = orc.rk4_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, 5)
        assert rel_err(u[i], ou) <= TOL, i
        assert rel_err(pi[i], op) <= TOL, i


def test_host_entry_point_matches_device_path():
    inst = W.bumpy_instance(W.Domain((24, 20, 16), 1.0 / 20), 8)
    lev, u, pi = run_gpu([inst], 3, 1, 0)
    hu = lev.scatter([inst.u])
    hp = lev.scatter([inst.pi])
    hc = lev.scatter([inst.c2], fill=1.0)
    ou, op = lev.rk4_step_host(hu, hp, hc, inst.dt, 3)
    assert np.array_equal(lev.gather(ou)[0], u[0])
    assert np.array_equal(lev.gather(op)[0], pi[0])


def test_autotune_keeps_results(tmp_path):
    import torch
    inst = W.uneven_level(n=(64, 64, 32), h=1.0 / 32, levels=3, seed=3, box_seed=30)
    lev, u0, p0 = run_gpu([inst], 3, 1, 0)
    cache = str(tmp_path / "tune.txt")
    lev.autotune(seed=1, budget_ms=300.0, abort_factor=2.0, cache_path=cache)
    assert os.path.getsize(cache) > 0
    _, u1, p1 = run_gpu([inst], 3, 1, 0, lev=lev)
    assert np.array_equal(u0[0], u1[0]) and np.array_equal(p0[0], p1[0])
    lev.autotune(seed=2, budget_ms=300.0, abort_factor=2.0, cache_path=cache)  # cache hit
    torch.cuda.synchronize()


def test_autotune_warm_cache_reproduces_choices(tmp_path):
    """A second level of the same boxes, tuned from the first one's cache,
    ends with the same form (stages per pass, pass kernels, staging) and the
    same tiles: whole-level timings are cached as well as per-class ones."""
    import torch
    inst = W.uneven_level(n=(64, 64, 32), h=1.0 / 32, levels=3, seed=3, box_seed=30)
    cache = str(tmp_path / "tune.txt")

    def tuned():
        lev = make_level([inst])
        lev.set_arith(1)
        lev.autotune(seed=1, budget_ms=300.0, abort_factor=2.0, cache_path=cache)
        torch.cuda.synchronize()
        tiles = [lev.get_tuning(c) for c in range(lev.size_classes()[0])]
        return (lev.get_fusion(), lev.get_pass_kernel(), lev.get_staging(), tiles)

    first = tuned()
    lines = open(cache).read().splitlines()
    assert any("|level" in ln for ln in lines)
    assert tuned() == first
    assert sorted(open(cache).read().splitlines()) == sorted(lines)


def test_nonfinite_input_is_reported(B):
    import torch
    inst = W.plane_wave(16)
    lev = make_level([inst])
    lev.set_arith(1)
    u = upload(lev, [inst.u])
    u[lev.layout[0][0] + 5] = float("nan")
    pi = upload(lev, [inst.pi])
    c2 = upload(lev, [inst.c2], fill=1.0)
    lev.rk4_step(u, pi, c2, inst.dt, 1)
    with pytest.raises(B.ScError) as e:
        lev.sync()
    assert e.value.code == B.SC_EDEVICE
    lev.sync()  # the error word was cleared
    torch.cuda.synchronize()


def test_launch_count_grows():
    inst = W.plane_wave(16)
    lev, _, _ = run_gpu([inst], 2, 1, 0)
    # a gather and a stage kernel per stage, plus the run prologue
    assert lev.launch_count() >= 2 * 8 + 2


# ----------------------------------------------------------------------------
# full-size checks in the benchmark's launch configuration
# ----------------------------------------------------------------------------

def test_full_256_plane_wave_closed_form_100_steps():
    inst = W.plane_wave(256)
    _, u, pi = run_gpu([inst], 100, 1, 0)
    h, dt = inst.dom.h, inst.dt
    mu = sum(_sigma(2 * np.pi * k * h) for k in (1, 2, 3)) / h ** 2
    z2 = dt * dt * mu
    a, b = 1 - z2 / 2 + z2 * z2 / 24, 1 - z2 / 6
    M = np.array([[a, b * dt], [-b * dt * mu, a]])
    ab = np.linalg.matrix_power(M, 100) @ np.array([1.0, 0.0])
    assert rel_err(u[0], ab[0] * inst.u) <= TOL
    assert rel_err(pi[0], ab[1] * inst.u) <= TOL


def test_full_256_bumpy_vs_oracle(orc):
    inst = W.single_box(256, seed=2)
    orc.set_threads(os.cpu_count() or 1)
    try:
        ou, op = orc.rk4_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, 2)
    finally:
        orc.set_threads(1)
    _, u, pi = run_gpu([inst], 2, 1, 0)
    assert rel_err(u[0], ou) <= TOL
    assert rel_err(pi[0], op) <= TOL


def test_full_uneven_level_vs_oracle(orc):
    inst = W.uneven_level()
    orc.set_threads(os.cpu_count() or 1)
    try:
        ou, op = orc.rk4_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, 1)
    finally:
        orc.set_threads(1)
    _, u, pi = run_gpu([inst], 1, 1, 0)
    assert rel_err(u[0], ou) <= TOL
    assert rel_err(pi[0], op) <= TOL


@pytest.mark.parametrize("arith", [0, 1])
def test_ghosts_written_by_stage_kernels(orc, arith):
    """In the taped forward with one stage per pass the stage kernels write
    the ghost copies of every value they produce; the final state's ghosts
    must equal a fresh exchange of its interior, bit for bit, on a 64-box
    level, and on a single box alone in its periodic domain for the z ghosts
    (the kernels read the owners of its x and y ghosts directly, so those
    are not written)."""
    import torch
    for inst in (W.uneven_level(n=(96, 80, 64), h=1.0 / 64, levels=6, seed=3, box_seed=30),
                 W.bumpy_instance(W.Domain((36, 28, 20), 1.0 / 28), 5)):
        lev = make_level([inst])
        lev.set_arith(arith)
        lev.set_fusion(1)
        u = upload(lev, [inst.u], fill=np.nan)
        pi = upload(lev, [inst.pi])
        c2 = upload(lev, [inst.c2], fill=1.0)
        uT = torch.full_like(u, float("nan"))
        piT = torch.empty_like(pi)
        lev.forward_tape(u, pi, c2, inst.dt, 3, 2, uT, piT)
        lev.sync()
        got = lev.padded_boxes(uT)
        want = lev.padded_boxes(lev.scatter([lev.gather(uT)[0]], fill=np.nan))
        n = inst.dom.n
        orc.fill_ghosts([lo + hi for lo, hi in inst.boxes], (0, 0, 0) + tuple(n), 7, want)
        single = len(inst.boxes) == 1
        for a, b in zip(got, want):
            m = ~np.isnan(b)
            if single:  # z ghosts and interior only
                m[:, :2, :] = False
                m[:, -2:, :] = False
                m[:, :, :2] = False
                m[:, :, -2:] = False
                assert m[:2].any() and m[-2:].any()
            assert np.array_equal(a[m], b[m])
        _, ug, _ = run_gpu([inst], 3, arith, 0)
        assert np.array_equal(lev.gather(uT)[0], ug[0])


# ----------------------------------------------------------------------------
# degenerate cases
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("arith", [0, 1])
def test_thin_and_odd_boxes(orc, arith):
    """Boxes of edge 2 and 3 and odd sizes on one periodic level."""
    n = (13, 11, 9)
    boxes = [((0, 0, 0), (2, 11, 9)), ((2, 0, 0), (5, 11, 9)), ((5, 0, 0), (13, 4, 9)),
             ((5, 4, 0), (13, 11, 2)), ((5, 4, 2), (13, 11, 9))]
    inst = W.bumpy_instance(W.Domain(n, 1.0 / 11), 7)
    inst.boxes = boxes
    ou, op = orc.rk4_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, 4)
    for mode in (0, 1):
        _, u, pi = run_gpu([inst], 4, arith, mode)
        assert rel_err(u[0], ou) <= TOL
        assert rel_err(pi[0], op) <= TOL


@pytest.mark.parametrize("fuse", [1, 2])
def test_small_self_periodic_boxes(orc, fuse):
    """A box that alone tiles its periodic domain reads the owners of its x
    and y ghosts directly (coordinates wrap by the extent), also when the
    extent is 2 or 3 so that a ghost's owner lies two periods away from the
    box's other side; an odd x extent keeps the gathered ghosts.  Every
    shape matches the oracle and, bit for bit, the same domain split into
    two boxes (which gathers every ghost)."""
    for n in ((2, 3, 5), (4, 2, 3), (6, 7, 2), (5, 6, 4), (12, 10, 3)):
        inst = W.bumpy_instance(W.Domain(n, 1.0 / 8), 11)
        ou, op = orc.rk4_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, 3)
        _, u, pi = run_gpu([inst], 3, 1, 0, fuse=fuse)
        assert rel_err(u[0], ou) <= TOL and rel_err(pi[0], op) <= TOL, n
        split = W.Instance(inst.dom, inst.u, inst.pi, inst.c2, inst.dt)
        d = int(np.argmax(n))  # halves of edge >= 2 along the longest axis
        hi0 = list(n)
        hi0[d] = n[d] // 2
        lo1 = [0, 0, 0]
        lo1[d] = n[d] // 2
        split.boxes = [((0, 0, 0), tuple(hi0)), (tuple(lo1), n)]
        _, u2, p2 = run_gpu([split], 3, 1, 0, fuse=fuse)
        assert np.array_equal(u[0], u2[0]) and np.array_equal(pi[0], p2[0]), n


def test_zero_steps_and_zero_field():
    inst = W.bumpy_instance(W.Domain((20, 16, 12), 1.0 / 16), 3)
    lev, u, pi = run_gpu([inst], 0, 1, 0)
    assert np.array_equal(u[0], inst.u) and np.array_equal(pi[0], inst.pi)
    z = W.Instance(inst.dom, np.zeros_like(inst.u), np.zeros_like(inst.u), inst.c2, inst.dt)
    _, u, pi = run_gpu([z], 3, 1, 0)
    assert not np.any(u[0]) and not np.any(pi[0])


@pytest.mark.parametrize("scale", [1e250, 1e-250])
def test_extreme_amplitudes(orc, scale):
    """The fixed-point scale follows the field's exponent: amplitudes near
    the ends of the FP64 range keep the 1e-12 bar."""
    inst = W.bumpy_instance(W.Domain((24, 20, 16), 1.0 / 20), 9)
    big = W.Instance(inst.dom, inst.u * scale, inst.pi, inst.c2, inst.dt)
    ou, op = orc.rk4_periodic(big.u, big.pi, big.c2, big.dom.h, big.dt, 3)
    for arith in (0, 1):
        _, u, pi = run_gpu([big], 3, arith, 0)
        assert rel_err(u[0], ou) <= TOL
        assert rel_err(pi[0], op) <= TOL


def test_amplitude_below_fixed_point_floor(orc):
    """Below 2^-959 the fixed form keeps an absolute resolution of 2^-1013
    (the exponent bound is clamped at 64): results stay finite and within
    that absolute bound of the oracle."""
    inst = W.bumpy_instance(W.Domain((24, 20, 16), 1.0 / 20), 9)
    tiny = W.Instance(inst.dom, inst.u * 1e-295, inst.pi, inst.c2, inst.dt)
    ou, op = orc.rk4_periodic(tiny.u, tiny.pi, tiny.c2, tiny.dom.h, tiny.dt, 2)
    _, u, pi = run_gpu([tiny], 2, 1, 0)
    assert np.all(np.isfinite(u[0])) and np.all(np.isfinite(pi[0]))
    h = tiny.dom.h
    # per stage the Laplacian is off by at most 192 2^-1013 / (12 h^2)
    bound = 8 * 192 * 2.0 ** -1013 / (12 * h * h) * (tiny.dt + 1)
    assert np.abs(pi[0] - op).max() <= bound
