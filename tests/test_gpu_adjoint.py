"""GPU adjoint: parity with the oracle's checkpointed gradient (1e-10), the
dot-product identity against the GPU forward (the step is linear in the
state), central finite differences of the GPU forward (1e-5), the misfit
kernel against the oracle, and the autograd Function."""
import numpy as np
import pytest

from paper_1308_1343_gb300 import workloads as W

from gpu_helpers import make_level, rel_err, upload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1308_1343_gb300 import build
    build.build()


def _setup(inst, arith, fuse=1):
    lev = make_level([inst])
    lev.set_arith(arith)
    lev.set_fusion(fuse)
    t = lambda a, fill=0.0: upload(lev, [a], fill)
    return lev, t


def _gpu_forward(lev, t, inst, u0, c2, nsteps):
    import torch
    u = t(u0)
    pi = t(inst.pi)
    lev.rk4_step(u, pi, t(c2, 1.0), inst.dt, nsteps, 0)
    lev.sync()
    torch.cuda.synchronize()
    return u, pi


@pytest.mark.parametrize("fuse", [1, 2])
@pytest.mark.parametrize("arith", [0, 1])
def test_gradient_matches_oracle(orc, arith, fuse):
    import torch
    inst = W.gradient_problem(20, 4)
    nsteps, ckpt = 16, 5
    h, dt = inst.dom.h, inst.dt
    lev, t = _setup(inst, arith, fuse)
    u_obs, _ = _gpu_forward(lev, t, inst, inst.u, inst.c2_obs, nsteps)
    u0, pi0, c2 = t(inst.u), t(inst.pi), t(inst.c2, 1.0)
    uT, piT = torch.empty_like(u0), torch.empty_like(u0)
    lev.forward_tape(u0, pi0, c2, dt, nsteps, ckpt, uT, piT)
    seed = torch.zeros_like(u0)
    loss, _ = lev.misfit(uT, u_obs, seed)
    g_u0, g_pi0, g_c2 = (torch.empty_like(u0) for _ in range(3))
    lev.backward_tape(c2, seed, None, g_u0, g_pi0, g_c2)
    lev.sync()
    # oracle
    ouT, _ = orc.rk4_periodic(inst.u, inst.pi, inst.c2, h, dt, nsteps)
    ouo, _ = orc.rk4_periodic(inst.u, inst.pi, inst.c2_obs, h, dt, nsteps)
    oseed = orc.misfit_seed(ouT, ouo, h)
    assert abs(loss.item() - orc.misfit_loss(ouT, ouo, h)) <= 1e-11 * orc.misfit_loss(ouT, ouo, h)
    ou, op, oc = orc.grad_periodic(inst.u, inst.pi, inst.c2, h, dt, nsteps, ckpt, oseed,
                                   np.zeros_like(oseed))
    assert rel_err(lev.gather(g_u0)[0], ou) <= 1e-10
    assert rel_err(lev.gather(g_pi0)[0], op) <= 1e-10
    assert rel_err(lev.gather(g_c2)[0], oc) <= 1e-10


def test_misfit_matches_oracle(orc):
    import torch
    inst = W.gradient_problem(24, 9)
    lev, t = _setup(inst, 1)
    seed = torch.zeros(lev.field_size, dtype=torch.float64, device="cuda")
    loss, _ = lev.misfit(t(inst.u), t(inst.c2_obs), seed)
    want = orc.misfit_loss(inst.u, inst.c2_obs, inst.dom.h)
    assert abs(loss.item() - want) <= 1e-13 * abs(want)
    assert rel_err(lev.gather(seed)[0], orc.misfit_seed(inst.u, inst.c2_obs, inst.dom.h)) <= 1e-15


@pytest.mark.parametrize("fuse", [1, 2])
@pytest.mark.parametrize("n,nsteps,ckpt", [(20, 12, 5), (128, 200, 20)])
def test_dot_identity_and_finite_differences(n, nsteps, ckpt, fuse):
    """Linear in u0: <u_T(d), a> + <pi_T(d), b> = <d, g_u0(a, b)>; and central
    differences of the misfit along c2 and u0 directions (the 128^3 case is
    the differentiation workload's full size)."""
    import torch
    inst = W.gradient_problem(n, 4)
    h, dt = inst.dom.h, inst.dt
    lev, t = _setup(inst, 1, fuse)
    sh = inst.dom.shape
    d = W.random_direction(sh, 41)
    a = W.random_direction(sh, 43)
    b = W.random_direction(sh, 44)
    zero = np.zeros(sh)
    # tangent of the state along u0 is the forward applied to (d, 0)
    ud, pd = _gpu_forward(lev, t, W.Instance(inst.dom, d, zero, inst.c2, dt), d, inst.c2, nsteps)
    lhs = float(np.sum(lev.gather(ud)[0] * a) + np.sum(lev.gather(pd)[0] * b))
    c2 = t(inst.c2, 1.0)
    g = [torch.empty(lev.field_size, dtype=torch.float64, device="cuda") for _ in range(3)]
    lev.grad(t(inst.u), t(zero), c2, dt, nsteps, ckpt, t(a), t(b), g[0], g[1], g[2])
    lev.sync()
    rhs = float(np.sum(lev.gather(g[0])[0] * d))
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)

    # misfit gradient vs central differences
    u_obs, _ = _gpu_forward(lev, t, inst, inst.u, inst.c2_obs, nsteps)
    u0 = t(inst.u)
    uT = torch.empty_like(u0)
    lev.forward_tape(u0, t(zero), c2, dt, nsteps, ckpt, uT, None)
    seed = torch.zeros_like(u0)
    lev.misfit(uT, u_obs, seed)
    lev.backward_tape(c2, seed, None, g[0], g[1], g[2])
    lev.sync()
    gu, gc = lev.gather(g[0])[0], lev.gather(g[2])[0]

    def loss_at(uu, cc):
        uT_, _ = _gpu_forward(lev, t, inst, uu, cc, nsteps)
        l, _ = lev.misfit(uT_, u_obs)
        return l.item()

    eps = 1e-6
    for seed_dir in (40, 42):
        dc = W.random_direction(sh, seed_dir)
        fd = (loss_at(inst.u, inst.c2 + eps * dc) - loss_at(inst.u, inst.c2 - eps * dc)) / (2 * eps)
        ad = float(np.sum(gc * dc))
        assert abs(fd - ad) <= 1e-5 * abs(ad), (fd, ad)
    du = W.random_direction(sh, 45)
    fd = (loss_at(inst.u + eps * du, inst.c2) - loss_at(inst.u - eps * du, inst.c2)) / (2 * eps)
    ad = float(np.sum(gu * du))
    assert abs(fd - ad) <= 1e-5 * abs(ad), (fd, ad)


def test_autograd_function():
    import torch
    from paper_1308_1343_gb300.level import wave_rk4
    inst = W.gradient_problem(16, 4)
    lev, t = _setup(inst, 1)
    u_obs, _ = _gpu_forward(lev, t, inst, inst.u, inst.c2_obs, 8)
    u0 = t(inst.u).requires_grad_(True)
    c2 = t(inst.c2, 1.0).requires_grad_(True)
    pi0 = t(inst.pi)
    uT, piT = wave_rk4(lev, u0, pi0, c2, inst.dt, 8, ckpt_every=3)
    # misfit through the library kernel, seeded into autograd
    seed = torch.zeros_like(uT)
    loss, _ = lev.misfit(uT.detach(), u_obs, seed)
    uT.backward(seed)
    g = [torch.empty_like(seed) for _ in range(3)]
    lev.grad(t(inst.u), pi0, c2.detach(), inst.dt, 8, 3, seed, None, *g)
    lev.sync()
    assert torch.equal(u0.grad, g[0]) or rel_err(lev.gather(u0.grad)[0], lev.gather(g[0])[0]) == 0
    assert rel_err(lev.gather(c2.grad)[0], lev.gather(g[2])[0]) == 0


@pytest.mark.parametrize("fuse", [1, 2])
def test_autograd_function_vs_oracle(orc, fuse):
    """wave_rk4 under torch autograd, with a loss built in torch on both
    outputs -- the misfit of u_T against an oracle observation plus a
    linear functional of pi_T, so that autograd hands the Function non-zero
    seeds for both -- against the oracle's checkpointed adjoint seeded with
    the same derivatives: u0.grad, pi0.grad and c2.grad within 1e-10, and
    the loss itself within 1e-11."""
    import torch
    from paper_1308_1343_gb300.level import wave_rk4
    inst = W.gradient_problem(20, 4)
    nsteps, ckpt = 12, 5
    h, dt = inst.dom.h, inst.dt
    lev, t = _setup(inst, 1, fuse)
    ouo, _ = orc.rk4_periodic(inst.u, inst.pi, inst.c2_obs, h, dt, nsteps)
    b = W.random_direction(inst.dom.shape, 47)
    interior = t(np.ones(inst.dom.shape)) != 0.0
    u_obs, b_dev = t(ouo), t(b)
    u0 = t(inst.u).requires_grad_(True)
    pi0 = t(inst.pi).requires_grad_(True)
    c2 = t(inst.c2, 1.0).requires_grad_(True)
    uT, piT = wave_rk4(lev, u0, pi0, c2, dt, nsteps, ckpt_every=ckpt)
    m = interior
    loss = 0.5 * h ** 3 * ((uT[m] - u_obs[m]) ** 2).sum() + (b_dev[m] * piT[m]).sum()
    loss.backward()
    lev.sync()
    ouT, opT = orc.rk4_periodic(inst.u, inst.pi, inst.c2, h, dt, nsteps)
    want_loss = 0.5 * h ** 3 * float(np.sum((ouT - ouo) ** 2)) + float(np.sum(b * opT))
    assert abs(loss.item() - want_loss) <= 1e-11 * abs(want_loss)
    ou, op, oc = orc.grad_periodic(inst.u, inst.pi, inst.c2, h, dt, nsteps, ckpt,
                                   orc.misfit_seed(ouT, ouo, h), b)
    assert rel_err(lev.gather(u0.grad)[0], ou) <= 1e-10
    assert rel_err(lev.gather(pi0.grad)[0], op) <= 1e-10
    assert rel_err(lev.gather(c2.grad)[0], oc) <= 1e-10


@pytest.mark.parametrize("fuse", [1, 2])
@pytest.mark.parametrize("arith", [0, 1])
def test_gradient_on_uneven_level(orc, arith, fuse):
    """Adjoint on an uneven multi-box level: equal to the one-box level's
    gradient bit for bit (decomposition independence) and to the oracle."""
    import torch
    inst = W.uneven_level(n=(64, 48, 40), h=1.0 / 48, levels=4, seed=6, box_seed=31)
    assert len(inst.boxes) == 16
    nsteps, ckpt = 9, 4
    res = []
    for insts in ([inst], [W.Instance(inst.dom, inst.u, inst.pi, inst.c2, inst.dt)]):
        lev = make_level(insts)
        lev.set_arith(arith)
        lev.set_fusion(fuse)
        t = lambda a, fill=0.0: upload(lev, [a], fill)
        seed_u = W.random_direction(inst.dom.shape, 43)
        g = [torch.empty(lev.field_size, dtype=torch.float64, device="cuda") for _ in range(3)]
        lev.grad(t(inst.u), t(inst.pi), t(inst.c2, 1.0), inst.dt, nsteps, ckpt, t(seed_u), None,
                 *g)
        lev.sync()
        res.append([lev.gather(x)[0] for x in g])
    for a, b in zip(res[0], res[1]):
        assert np.array_equal(a, b)
    ou, op, oc = orc.grad_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, nsteps, ckpt,
                                   seed_u, np.zeros_like(seed_u))
    assert rel_err(res[0][0], ou) <= 1e-10
    assert rel_err(res[0][1], op) <= 1e-10
    assert rel_err(res[0][2], oc) <= 1e-10


@pytest.mark.parametrize("fuse", [1, 2])
def test_gradient_of_an_ensemble(orc, fuse):
    """One level of several periodic domains with their own sizes, wave
    speeds, seeds and step sizes (the ensemble workload's structure): every
    instance's gradient matches the oracle's."""
    import torch
    insts = [W.bumpy_instance(W.Domain((n, n, n), 1.0 / n), 5000 + i)
             for i, n in enumerate((24, 32, 16, 40))]
    nsteps, ckpt = 7, 3
    lev = make_level(insts)
    lev.set_arith(1)
    lev.set_fusion(fuse)
    up = lambda arrs, fill=0.0: upload(lev, arrs, fill)
    seeds_u = [W.random_direction(i.dom.shape, 60 + k) for k, i in enumerate(insts)]
    seeds_p = [W.random_direction(i.dom.shape, 70 + k) for k, i in enumerate(insts)]
    g = [torch.empty(lev.field_size, dtype=torch.float64, device="cuda") for _ in range(3)]
    lev.grad(up([i.u for i in insts]), up([i.pi for i in insts]),
             up([i.c2 for i in insts], 1.0), [i.dt for i in insts], nsteps, ckpt,
             up(seeds_u), up(seeds_p), *g)
    lev.sync()
    got = [lev.gather(x) for x in g]
    for k, inst in enumerate(insts):
        ou, op, oc = orc.grad_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, nsteps,
                                       ckpt, seeds_u[k], seeds_p[k])
        assert rel_err(got[0][k], ou) <= 1e-10, k
        assert rel_err(got[1][k], op) <= 1e-10, k
        assert rel_err(got[2][k], oc) <= 1e-10, k


def test_gradient_of_the_full_ensemble(orc):
    """The benchmark's ensemble (256 cubes, own sizes, fields and step sizes)
    through the checkpointed adjoint, two steps with a checkpoint each: every
    instance's gradient within 1e-10 of the oracle's."""
    import os
    import torch
    insts = W.ensemble()
    nsteps, ckpt = 2, 1
    lev = make_level(insts)
    lev.set_arith(1)
    up = lambda arrs, fill=0.0: upload(lev, arrs, fill)
    seeds_u = [W.random_direction(i.dom.shape, 900 + k) for k, i in enumerate(insts)]
    seeds_p = [W.random_direction(i.dom.shape, 1900 + k) for k, i in enumerate(insts)]
    g = [torch.empty(lev.field_size, dtype=torch.float64, device="cuda") for _ in range(3)]
    lev.grad(up([i.u for i in insts]), up([i.pi for i in insts]),
             up([i.c2 for i in insts], 1.0), [i.dt for i in insts], nsteps, ckpt,
             up(seeds_u), up(seeds_p), *g)
    lev.sync()
    got = [lev.gather(x) for x in g]
    orc.set_threads(os.cpu_count() or 1)
    try:
        for k, inst in enumerate(insts):
            ou, op, oc = orc.grad_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt,
                                           nsteps, ckpt, seeds_u[k], seeds_p[k])
            assert rel_err(got[0][k], ou) <= 1e-10, k
            assert rel_err(got[1][k], op) <= 1e-10, k
            assert rel_err(got[2][k], oc) <= 1e-10, k
    finally:
        orc.set_threads(1)
