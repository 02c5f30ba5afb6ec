"""Pins of the oracle's tangent-linear and adjoint codes.

The adjoint is checked against the independently written tangent-linear
code (dot-product identity, one step and a checkpointed trajectory), and
both are checked against central finite differences of the plain forward
RK4.  The loss is quadratic in u0 (the step is linear in the state), so its
u0-gradient must match a central difference to rounding for any step.
"""
import numpy as np
import pytest

from paper_1308_1343_gb300 import workloads as W


def _small(n=12, seed=4):
    inst = W.gradient_problem(n, seed)
    return inst


def _rand(shape, seed):
    return np.random.default_rng(seed).normal(size=shape)


def test_one_step_dot_identity(orc):
    inst = _small()
    h, dt = inst.dom.h, inst.dt
    sh = inst.dom.shape
    du, dpi, dc2 = _rand(sh, 1), _rand(sh, 2), _rand(sh, 3)
    bu, bpi = _rand(sh, 4), _rand(sh, 5)
    pi0 = 0.3 * _rand(sh, 6)
    _, _, tu, tp = orc.tlm_periodic(inst.u, pi0, inst.c2, du, dpi, dc2, h, dt, 1)
    au, ap, ac2 = orc.adj_step_periodic(inst.u, pi0, inst.c2, bu, bpi, np.zeros(sh), h, dt)
    lhs = np.sum(tu * bu) + np.sum(tp * bpi)
    rhs = np.sum(du * au) + np.sum(dpi * ap) + np.sum(dc2 * ac2)
    assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + 1e-300) + 1e-14 * np.sum(np.abs(tu * bu))


def test_trajectory_dot_identity_with_checkpoints(orc):
    inst = _small()
    h, dt = inst.dom.h, inst.dt
    sh = inst.dom.shape
    du, dc2 = _rand(sh, 11), _rand(sh, 12)
    dpi = np.zeros(sh)
    bu, bpi = _rand(sh, 13), _rand(sh, 14)
    nsteps = 9
    _, _, tu, tp = orc.tlm_periodic(inst.u, inst.pi, inst.c2, du, dpi, dc2, h, dt, nsteps)
    gu, gp, gc2 = orc.grad_periodic(inst.u, inst.pi, inst.c2, h, dt, nsteps, 4, bu, bpi)
    lhs = np.sum(tu * bu) + np.sum(tp * bpi)
    rhs = np.sum(du * gu) + np.sum(dpi * gp) + np.sum(dc2 * gc2)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_checkpoint_interval_does_not_change_gradient(orc):
    inst = _small(10)
    h, dt = inst.dom.h, inst.dt
    sh = inst.dom.shape
    bu, bpi = _rand(sh, 21), _rand(sh, 22)
    res = [orc.grad_periodic(inst.u, inst.pi, inst.c2, h, dt, 7, k, bu, bpi)
           for k in (1, 3, 7, 100)]
    for r in res[1:]:
        for a, b in zip(res[0], r):
            assert np.array_equal(a, b)


def test_tlm_matches_central_difference(orc):
    inst = _small()
    h, dt = inst.dom.h, inst.dt
    sh = inst.dom.shape
    dc2 = W.random_direction(sh, 40)
    du = W.random_direction(sh, 41)
    eps = 1e-5
    nsteps = 6
    _, _, tu, tp = orc.tlm_periodic(inst.u, inst.pi, inst.c2, du, np.zeros(sh), dc2, h, dt,
                                     nsteps)
    up, pp = orc.rk4_periodic(inst.u + eps * du, inst.pi, inst.c2 + eps * dc2, h, dt, nsteps)
    um, pm = orc.rk4_periodic(inst.u - eps * du, inst.pi, inst.c2 - eps * dc2, h, dt, nsteps)
    fu = (up - um) / (2 * eps)
    fp = (pp - pm) / (2 * eps)
    assert np.abs(fu - tu).max() <= 1e-6 * np.abs(tu).max()
    assert np.abs(fp - tp).max() <= 1e-6 * np.abs(tp).max()


def _loss_and_grad(orc, inst, c2, u0, nsteps, ckpt):
    h, dt = inst.dom.h, inst.dt
    uT, _ = orc.rk4_periodic(u0, inst.pi, c2, h, dt, nsteps)
    uo, _ = orc.rk4_periodic(inst.u, inst.pi, inst.c2_obs, h, dt, nsteps)
    loss = orc.misfit_loss(uT, uo, h)
    seed = orc.misfit_seed(uT, uo, h)
    g = orc.grad_periodic(u0, inst.pi, c2, h, dt, nsteps, ckpt, seed, np.zeros_like(seed))
    return loss, g, uo


@pytest.mark.parametrize("which", ["c2", "u0"])
def test_gradient_matches_central_difference(orc, which):
    inst = _small(12)
    nsteps, ckpt = 20, 5
    h, dt = inst.dom.h, inst.dt
    loss, (gu, _, gc2), uo = _loss_and_grad(orc, inst, inst.c2, inst.u, nsteps, ckpt)
    assert loss > 0
    for s in (40, 41):
        d = W.random_direction(inst.dom.shape, s)
        eps = 1e-6
        if which == "c2":
            lp = orc.misfit_loss(orc.rk4_periodic(inst.u, inst.pi, inst.c2 + eps * d, h, dt,
                                                  nsteps)[0], uo, h)
            lm = orc.misfit_loss(orc.rk4_periodic(inst.u, inst.pi, inst.c2 - eps * d, h, dt,
                                                  nsteps)[0], uo, h)
            g = gc2
        else:
            lp = orc.misfit_loss(orc.rk4_periodic(inst.u + eps * d, inst.pi, inst.c2, h, dt,
                                                  nsteps)[0], uo, h)
            lm = orc.misfit_loss(orc.rk4_periodic(inst.u - eps * d, inst.pi, inst.c2, h, dt,
                                                  nsteps)[0], uo, h)
            g = gu
        fd = (lp - lm) / (2 * eps)
        ad = np.sum(g * d)
        assert abs(fd - ad) <= 1e-5 * abs(ad), (which, fd, ad)


def test_u0_gradient_exact_for_quadratic_loss(orc):
    # u_T is linear in u0, so the loss is an exact quadratic in u0 and the
    # central difference equals <g, d> for any step size (up to rounding).
    inst = _small(10)
    nsteps = 8
    h, dt = inst.dom.h, inst.dt
    _, (gu, _, _), uo = _loss_and_grad(orc, inst, inst.c2, inst.u, nsteps, 3)
    d = W.random_direction(inst.dom.shape, 42)
    eps = 0.1
    lp = orc.misfit_loss(orc.rk4_periodic(inst.u + eps * d, inst.pi, inst.c2, h, dt, nsteps)[0],
                         uo, h)
    lm = orc.misfit_loss(orc.rk4_periodic(inst.u - eps * d, inst.pi, inst.c2, h, dt, nsteps)[0],
                         uo, h)
    fd = (lp - lm) / (2 * eps)
    ad = np.sum(gu * d)
    assert abs(fd - ad) <= 1e-10 * abs(ad)
