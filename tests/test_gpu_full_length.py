"""Parity at the benchmarked configurations, at their full sizes and step
counts, against the CPU oracle (OpenMP over z-planes, bit-identical to one
thread), through the C ABI:

* the 256^3 bumpy box in the form the benchmark runs: two RK4 stages per
  pass, fixed-point Laplacian sums, CUDA graph per step, tuned tiles, 100
  steps -- u and pi within 1e-12 relative max norm;
* the 512 x 512 x 256 level of 64 uneven boxes in the same form, 50 steps;
* the 128^3 gradient problem, 200 steps with checkpoints every 20, misfit
  loss: g_u0, g_pi0 and g_c2 within 1e-10 of the oracle's checkpointed
  adjoint;
* the 512 x 512 x 256 level's gradient (a short run: the oracle's adjoint
  takes about a second per step at this size);
* what the fixed-point form gives up: its error is bounded relative to the
  domain's largest value, not to each value, so where |u| is 1e-8 of the
  maximum a point keeps fewer correct digits than in the FP64 form.

Tiles come from the benchmark's tuning cache when it holds them (tuning
changes no bit: test_gpu_fused.py)."""
import os

import numpy as np
import pytest

from paper_1308_1343_gb300 import workloads as W

from gpu_helpers import make_level, rel_err, upload

pytestmark = pytest.mark.gpu

TOL = 1e-12
GRAD_TOL = 1e-10
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TUNE_CACHE = os.path.join(ROOT, "paper_1308_1343_gb300", "_build", "tune_cache.txt")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1308_1343_gb300 import build
    build.build()


@pytest.fixture()
def all_cores(orc):
    orc.set_threads(os.cpu_count() or 1)
    yield orc
    orc.set_threads(1)


def _bench_level(insts, seed, budget_ms, fuse=2, arith=1):
    """A level set up as the benchmark sets up its workloads: fixed-point
    arithmetic, the given form, tiles tuned (or read from the cache)."""
    import torch
    lev = make_level(insts)
    lev.set_arith(arith)
    lev.set_fusion(fuse)
    os.makedirs(os.path.dirname(TUNE_CACHE), exist_ok=True)
    lev.autotune(seed=seed, budget_ms=budget_ms, abort_factor=2.0, cache_path=TUNE_CACHE,
                 stream=torch.cuda.current_stream())
    return lev


def _evolve(lev, inst, nsteps, mode=0):
    import torch
    u = upload(lev, [inst.u])
    pi = upload(lev, [inst.pi])
    c2 = upload(lev, [inst.c2], fill=1.0)
    lev.rk4_step(u, pi, c2, inst.dt, nsteps, mode)
    lev.sync()
    torch.cuda.synchronize()
    return lev.gather(u)[0], lev.gather(pi)[0]


def test_headline_256_two_stage_fixed_graph_100_steps(all_cores):
    inst = W.single_box(256, seed=2)
    lev = _bench_level([inst], seed=2, budget_ms=2000.0)
    assert lev.get_fusion() == 2
    u, pi = _evolve(lev, inst, 100)
    lev.close()
    ou, op = all_cores.rk4_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, 100)
    assert rel_err(u, ou) <= TOL
    assert rel_err(pi, op) <= TOL


def test_uneven_level_two_stage_fixed_graph_50_steps(all_cores):
    inst = W.uneven_level()
    assert len(inst.boxes) == 64 and inst.u.shape == (256, 512, 512)
    lev = _bench_level([inst], seed=3, budget_ms=3000.0)
    u, pi = _evolve(lev, inst, 50)
    lev.close()
    ou, op = all_cores.rk4_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, 50)
    assert rel_err(u, ou) <= TOL
    assert rel_err(pi, op) <= TOL


def _misfit_gradient(lev, inst, nsteps, ckpt):
    """GPU gradient of the misfit against the observation made with
    c2_obs, seeded by the library's misfit kernel."""
    import torch
    t = lambda a, fill=0.0: upload(lev, [a], fill)
    u_obs = t(inst.u)
    p_obs = t(inst.pi)
    lev.rk4_step(u_obs, p_obs, t(inst.c2_obs, 1.0), inst.dt, nsteps, 0)
    u0, pi0, c2 = t(inst.u), t(inst.pi), t(inst.c2, 1.0)
    uT = torch.empty_like(u0)
    lev.forward_tape(u0, pi0, c2, inst.dt, nsteps, ckpt, uT, None)
    seed = torch.zeros_like(u0)
    lev.misfit(uT, u_obs, seed)
    g = [torch.empty_like(u0) for _ in range(3)]
    lev.backward_tape(c2, seed, None, *g)
    lev.sync()
    torch.cuda.synchronize()
    return [lev.gather(x)[0] for x in g]


def _oracle_misfit_gradient(orc, inst, nsteps, ckpt):
    h, dt = inst.dom.h, inst.dt
    ouT, _ = orc.rk4_periodic(inst.u, inst.pi, inst.c2, h, dt, nsteps)
    ouo, _ = orc.rk4_periodic(inst.u, inst.pi, inst.c2_obs, h, dt, nsteps)
    seed = orc.misfit_seed(ouT, ouo, h)
    return orc.grad_periodic(inst.u, inst.pi, inst.c2, h, dt, nsteps, ckpt, seed,
                             np.zeros_like(seed))


def test_gradient_128_200_steps_checkpoint_20(all_cores):
    inst = W.gradient_problem(128, 4)
    lev = _bench_level([inst], seed=4, budget_ms=2000.0)
    got = _misfit_gradient(lev, inst, 200, 20)
    lev.close()
    want = _oracle_misfit_gradient(all_cores, inst, 200, 20)
    for name, g, w in zip(("g_u0", "g_pi0", "g_c2"), got, want):
        assert rel_err(g, w) <= GRAD_TOL, name


def test_gradient_of_the_full_uneven_level(all_cores):
    """The adjoint on the 64-box 512 x 512 x 256 level (the differentiated
    form of the uneven workload), 4 steps with checkpoints every 2, a seed
    on u and one on pi."""
    import torch
    inst = W.uneven_level()
    lev = _bench_level([inst], seed=3, budget_ms=3000.0)
    t = lambda a, fill=0.0: upload(lev, [a], fill)
    su = W.random_direction(inst.dom.shape, 81)
    sp = W.random_direction(inst.dom.shape, 82)
    g = [torch.empty(lev.field_size, dtype=torch.float64, device="cuda") for _ in range(3)]
    lev.grad(t(inst.u), t(inst.pi), t(inst.c2, 1.0), inst.dt, 4, 2, t(su), t(sp), *g)
    lev.sync()
    got = [lev.gather(x)[0] for x in g]
    lev.close()
    want = all_cores.grad_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, 4, 2, su, sp)
    for name, a, b in zip(("g_u0", "g_pi0", "g_c2"), got, want):
        assert rel_err(a, b) <= GRAD_TOL, name


def test_fixed_point_error_is_domain_relative(orc):
    """What the fixed-point form gives up.  Each input of a fixed-point sum
    is off by < 2^-54 max|x| of its field: the error is bounded relative to
    the domain's largest value, not to each value.  After n steps both forms
    stay within 4 n 2^-52 max|u| of the oracle everywhere (and so within the
    1e-12 max-norm bar), but in the Gaussian pulse's far field, where
    1e-10 <= |u| / max|u| <= 1e-8, the fixed form's error relative to each
    value is larger than the FP64 form's, which rounds every value relative
    to itself.  (Below about 2^-55 max|u| an input truncates to zero, so far
    enough out the fixed form keeps no correct digit of u's change.)"""
    inst = W.bumpy_instance(W.Domain((64, 64, 64), 1.0 / 64), 21)
    nsteps = 20
    ou, op = orc.rk4_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, nsteps)
    umax = np.abs(ou).max()
    a = np.abs(ou) / umax
    band = (a >= 1e-10) & (a <= 1e-8)
    assert band.sum() > 100
    res = {}
    for arith in (0, 1):
        lev = make_level([inst])
        lev.set_arith(arith)
        lev.set_fusion(2)
        u, pi = _evolve(lev, inst, nsteps)
        lev.close()
        assert rel_err(u, ou) <= TOL and rel_err(pi, op) <= TOL
        err = np.abs(u - ou)
        assert err.max() <= 4 * nsteps * 2.0 ** -52 * umax, arith
        res[arith] = (err.max() / umax, (err[band] / np.abs(ou[band])).max())
    (fp_abs, fp_rel), (fx_abs, fx_rel) = res[0], res[1]
    print("max error / max|u|: fp64 %.2e, fixed %.2e; in the band 1e-10..1e-8 of max|u|, "
          "max error / |u|: fp64 %.2e, fixed %.2e (%d points)"
          % (fp_abs, fx_abs, fp_rel, fx_rel, int(band.sum())))
    assert fp_rel < fx_rel
