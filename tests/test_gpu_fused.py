"""GPU parity of the two-stages-per-pass form (sc_level_set_fusion(2))
against the CPU oracle, through the C ABI.

The two passes evaluate the same nested RK4 step with L applied to y.u, y.pi
(pass A) and w_2.u, w_2.pi (pass B) and L w_1.u, L w_3.u formed by
linearity, so the bar is the same as for the one-stage form: u and pi
within 1e-12 relative max norm of the oracle; the launch modes and any
decomposition of the level bit-identical to each other; the two forms equal
up to rounding."""
import os

import numpy as np
import pytest

from paper_1308_1343_gb300 import workloads as W

from gpu_helpers import make_level, rel_err, run_gpu

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1308_1343_gb300 import build
    build.build()


def run_fused(instances, nsteps, arith, mode):
    lev = make_level(instances)
    lev.set_fusion(2)
    return run_gpu(instances, nsteps, arith, mode, lev=lev)


def _sigma(t):
    return (15.0 - 16.0 * np.cos(t) + np.cos(2 * t)) / 6.0


@pytest.mark.parametrize("arith", [0, 1])
def test_plane_wave_closed_form(orc, arith):
    inst = W.plane_wave(32)
    _, u, pi = run_fused([inst], 20, arith, 0)
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
def test_ragged_box_all_modes(orc, arith):
    dom = W.Domain((40, 36, 28), 1.0 / 36)
    inst = W.bumpy_instance(dom, 2)
    ou, op = orc.rk4_periodic(inst.u, inst.pi, inst.c2, dom.h, inst.dt, 6)
    res = {}
    for mode in (0, 1, 2, 3):
        _, u, pi = run_fused([inst], 6, arith, mode)
        assert rel_err(u[0], ou) <= TOL, mode
        assert rel_err(pi[0], op) <= TOL, mode
        res[mode] = (u[0], pi[0])
    for mode in (1, 2, 3):
        assert np.array_equal(res[mode][0], res[0][0]), mode
        assert np.array_equal(res[mode][1], res[0][1]), mode


@pytest.mark.parametrize("arith", [0, 1])
def test_uneven_level_decomposition_independent(orc, arith):
    inst = W.uneven_level(n=(128, 128, 64), h=1.0 / 64, levels=6, seed=3, box_seed=30)
    ou, op = orc.rk4_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, 4)
    _, u, pi = run_fused([inst], 4, arith, 0)
    assert rel_err(u[0], ou) <= TOL
    assert rel_err(pi[0], op) <= TOL
    one = W.Instance(inst.dom, inst.u, inst.pi, inst.c2, inst.dt)
    _, u1, p1 = run_fused([one], 4, arith, 0)
    assert np.array_equal(u[0], u1[0]) and np.array_equal(pi[0], p1[0])
    _, u2, p2 = run_fused([inst], 4, arith, 1)
    assert np.array_equal(u[0], u2[0]) and np.array_equal(pi[0], p2[0])


@pytest.mark.parametrize("arith", [0, 1])
def test_ensemble_per_domain_dt(orc, arith):
    insts = [W.bumpy_instance(W.Domain((n, n, n), 1.0 / n), 5000 + i)
             for i, n in enumerate((24, 32, 40, 24, 56, 48))]
    _, u, pi = run_fused(insts, 5, arith, 0)
    for i, inst in enumerate(insts):
        ou, op = orc.rk4_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, 5)
        assert rel_err(u[i], ou) <= TOL, i
        assert rel_err(pi[i], op) <= TOL, i


@pytest.mark.parametrize("arith", [0, 1])
def test_thin_and_odd_boxes(orc, arith):
    n = (13, 11, 9)
    boxes = [((0, 0, 0), (2, 11, 9)), ((2, 0, 0), (5, 11, 9)), ((5, 0, 0), (13, 4, 9)),
             ((5, 4, 0), (13, 11, 2)), ((5, 4, 2), (13, 11, 9))]
    inst = W.bumpy_instance(W.Domain(n, 1.0 / 11), 7)
    inst.boxes = boxes
    ou, op = orc.rk4_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, 4)
    for mode in (0, 1):
        _, u, pi = run_fused([inst], 4, arith, mode)
        assert rel_err(u[0], ou) <= TOL
        assert rel_err(pi[0], op) <= TOL


def test_forms_agree_to_rounding():
    inst = W.bumpy_instance(W.Domain((48, 40, 32), 1.0 / 32), 11)
    inst.boxes = W.bisect_boxes(inst.dom.n, 3, seed=7)
    _, u1, p1 = run_gpu([inst], 8, 1, 0)
    _, u2, p2 = run_fused([inst], 8, 1, 0)
    assert rel_err(u2[0], u1[0]) <= 1e-13
    assert rel_err(p2[0], p1[0]) <= 1e-13
    assert not np.array_equal(p2[0], p1[0])  # the passes really ran


@pytest.mark.parametrize("scale", [1e250, 1e-250])
def test_extreme_amplitudes(orc, scale):
    inst = W.bumpy_instance(W.Domain((24, 20, 16), 1.0 / 20), 9)
    big = W.Instance(inst.dom, inst.u * scale, inst.pi * scale + scale * 1e-3, inst.c2,
                     inst.dt)
    ou, op = orc.rk4_periodic(big.u, big.pi, big.c2, big.dom.h, big.dt, 3)
    for arith in (0, 1):
        _, u, pi = run_fused([big], 3, arith, 0)
        assert rel_err(u[0], ou) <= TOL
        assert rel_err(pi[0], op) <= TOL


def test_zero_steps_and_zero_field():
    inst = W.bumpy_instance(W.Domain((20, 16, 12), 1.0 / 16), 3)
    _, u, pi = run_fused([inst], 0, 1, 0)
    assert np.array_equal(u[0], inst.u) and np.array_equal(pi[0], inst.pi)
    z = W.Instance(inst.dom, np.zeros_like(inst.u), np.zeros_like(inst.u), inst.c2, inst.dt)
    _, u, pi = run_fused([z], 3, 1, 0)
    assert not np.any(u[0]) and not np.any(pi[0])


@pytest.mark.parametrize("kind", [0, 1])
def test_timed_mode_counts_two_passes(kind):
    """Two pass launches per step with either pass kernel, on a box that
    alone tiles its periodic domain and on a level of two boxes; two gathers
    per step, except on the single box with the warp-specialised kernels,
    which read all its ghosts from their periodic images (the one-role
    kernels read those of x and y so, and have its z ghosts gathered)."""
    from paper_1308_1343_gb300 import binding as B
    inst = W.bumpy_instance(W.Domain((32, 24, 16), 1.0 / 24), 4)
    two = W.Instance(inst.dom, inst.u, inst.pi, inst.c2, inst.dt)
    two.boxes = [((0, 0, 0), (16, 24, 16)), ((16, 0, 0), (32, 24, 16))]
    res = []
    for case in (inst, two):
        lev = make_level([case])
        lev.set_fusion(2)
        lev.set_pass_kernel(kind)
        lev, u, pi = run_gpu([case], 3, 1, B.SC_MODE_TIMED, lev=lev)
        assert lev.kernel_time(B.SC_KERNEL_PAIR_A)[1] == 3
        assert lev.kernel_time(B.SC_KERNEL_PAIR_B)[1] == 3
        want = 0 if kind == 1 and case is inst else 6
        assert lev.kernel_time(B.SC_KERNEL_GATHER)[1] == want
        assert lev.kernel_time(B.SC_KERNEL_STAGE)[1] == 0
        res.append((u[0], pi[0]))
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])


def test_full_256_bumpy_vs_oracle(orc):
    inst = W.single_box(256, seed=2)
    orc.set_threads(os.cpu_count() or 1)
    try:
        ou, op = orc.rk4_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, 2)
    finally:
        orc.set_threads(1)
    _, u, pi = run_fused([inst], 2, 1, 0)
    assert rel_err(u[0], ou) <= TOL
    assert rel_err(pi[0], op) <= TOL


def test_autotune_chooses_a_form(orc, tmp_path):
    """Without a fixed form the tuner picks one; the result still matches the
    oracle and equals that form's run with default tiles bit for bit."""
    inst = W.uneven_level(n=(64, 64, 32), h=1.0 / 32, levels=3, seed=3, box_seed=30)
    lev = make_level([inst])
    lev.set_arith(1)
    lev.autotune(seed=1, budget_ms=400.0, abort_factor=2.0, cache_path=str(tmp_path / "t.txt"))
    form = lev.get_fusion()
    assert form in (1, 2)
    _, u, pi = run_gpu([inst], 3, 1, 0, lev=lev)
    ou, op = orc.rk4_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, 3)
    assert rel_err(u[0], ou) <= TOL
    assert rel_err(pi[0], op) <= TOL
    _, u1, p1 = run_gpu([inst], 3, 1, 0, fuse=form)
    assert np.array_equal(u[0], u1[0]) and np.array_equal(pi[0], p1[0])


@pytest.mark.parametrize("fuse", [1, 2])
def test_tiles_and_z_runs_change_no_bit(orc, fuse):
    """Tile widths 16, 32, 64 and z-run lengths that do or do not divide
    the box (runs of near-equal length: 37 on 75 planes gives 38 + 37, 5
    gives fifteen runs of 5, 100 one run), on a ragged box: every setting
    gives the same bits, and the oracle's values within the bar."""
    dom = W.Domain((44, 38, 75), 1.0 / 40)
    inst = W.bumpy_instance(dom, 12)
    ou, op = orc.rk4_periodic(inst.u, inst.pi, inst.c2, dom.h, inst.dt, 3)
    lev = make_level([inst])
    lev.set_fusion(fuse)
    ref = None
    for tx, tz in ((32, 32), (32, 37), (16, 5), (64, 100), (16, 74), (64, 3)):
        lev.set_tuning(0, tx, tz)
        assert lev.get_tuning(0) == (tx, 512 // tx, tz)
        _, u, pi = run_gpu([inst], 3, 1, 0, lev=lev)
        if ref is None:
            ref = (u[0], pi[0])
            assert rel_err(u[0], ou) <= TOL and rel_err(pi[0], op) <= TOL
        assert np.array_equal(u[0], ref[0]) and np.array_equal(pi[0], ref[1]), (tx, tz)


def test_full_ensemble_vs_oracle(orc):
    """The benchmark's ensemble (256 periodic cubes of edge 24-96, each with
    its own fields and step size, one level, default tiles and form), two RK4
    steps: every instance within the bar of the oracle."""
    insts = W.ensemble()
    lev = make_level(insts)
    _, u, pi = run_gpu(insts, 2, 1, 0, lev=lev)
    orc.set_threads(os.cpu_count() or 1)
    try:
        for k, inst in enumerate(insts):
            ou, op = orc.rk4_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, 2)
            assert rel_err(u[k], ou) <= TOL, k
            assert rel_err(pi[k], op) <= TOL, k
    finally:
        orc.set_threads(1)


def test_stagings_change_no_bit(orc):
    """One stage per pass with the raw stencil inputs staged in registers or
    in shared memory by cp.async: the same bits, on a ragged multi-box level
    and on a self-periodic box, in every launch mode; and the autotuner,
    free to choose the staging, keeps the bits too."""
    from paper_1308_1343_gb300 import binding as B
    uneven = W.uneven_level(n=(96, 80, 64), h=1.0 / 64, levels=4, seed=3, box_seed=30)
    single = W.bumpy_instance(W.Domain((44, 38, 30), 1.0 / 38), 6)
    for inst in (uneven, single):
        ou, op = orc.rk4_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, 3)
        ref = None
        for staging in (B.SC_STAGING_REGISTERS, B.SC_STAGING_SHARED):
            for mode in (0, 1, 2):
                lev = make_level([inst])
                lev.set_fusion(1)
                lev.set_staging(staging)
                _, u, pi = run_gpu([inst], 3, 1, mode, lev=lev)
                if ref is None:
                    ref = (u[0], pi[0])
                    assert rel_err(u[0], ou) <= TOL and rel_err(pi[0], op) <= TOL
                assert np.array_equal(u[0], ref[0]) and np.array_equal(pi[0], ref[1]), \
                    (staging, mode)
        lev = make_level([inst])
        lev.set_fusion(1)
        lev.autotune(seed=3, budget_ms=200.0)
        assert lev.get_staging() in (B.SC_STAGING_REGISTERS, B.SC_STAGING_SHARED)
        _, u, pi = run_gpu([inst], 3, 1, 0, lev=lev)
        assert np.array_equal(u[0], ref[0]) and np.array_equal(pi[0], ref[1])
