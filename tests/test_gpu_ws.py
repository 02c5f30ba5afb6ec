"""The warp-specialised pass kernels (sc_level_set_pass_kernel,
SC_PASS_WARP_SPECIALISED) and adjoint passes against the one-role pass
kernels and adjoint passes with their combination kernel, through the C
ABI: bit-identical states and gradients on every layout the one-role
kernels are tested on (ragged, thin and odd boxes, an uneven level, an
ensemble with per-domain step sizes, self-periodic boxes, every tile width
and z-run, every launch mode, both arithmetic forms, the taped forward and
the adjoint's recomputation), the oracle's values within the bar, and the
bounded wait: a wait test makes the producers' wait for a free ring slot
run out, the kernel returns, sc_level_sync reports SC_EDEVICE, and the
level works again afterwards."""
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


def _both(inst_list, nsteps, arith, mode, tiles=None):
    out = []
    for kind in (0, 1):
        lev = make_level(inst_list)
        lev.set_fusion(2)
        lev.set_pass_kernel(kind)
        if tiles:
            for cls, (tx, tz) in tiles.items():
                lev.set_tuning(cls, tx, tz)
        _, u, pi = run_gpu(inst_list, nsteps, arith, mode, lev=lev)
        assert lev.get_pass_kernel() == kind
        out.append((u, pi))
        lev.close()
    return out


def _same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a[0] + a[1], b[0] + b[1]))


@pytest.mark.parametrize("arith", [0, 1])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_ragged_box_every_mode(orc, arith, mode):
    dom = W.Domain((40, 36, 28), 1.0 / 36)
    inst = W.bumpy_instance(dom, 2)
    one, ws = _both([inst], 6, arith, mode)
    assert _same(one, ws)
    ou, op = orc.rk4_periodic(inst.u, inst.pi, inst.c2, dom.h, inst.dt, 6)
    assert rel_err(ws[0][0], ou) <= TOL and rel_err(ws[1][0], op) <= TOL


@pytest.mark.parametrize("arith", [0, 1])
def test_uneven_level_and_thin_boxes(orc, arith):
    inst = W.uneven_level(n=(128, 128, 64), h=1.0 / 64, levels=6, seed=3, box_seed=30)
    one, ws = _both([inst], 4, arith, 0)
    assert _same(one, ws)
    ou, op = orc.rk4_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, 4)
    assert rel_err(ws[0][0], ou) <= TOL and rel_err(ws[1][0], op) <= TOL
    n = (13, 11, 9)
    thin = W.bumpy_instance(W.Domain(n, 1.0 / 11), 7)
    thin.boxes = [((0, 0, 0), (2, 11, 9)), ((2, 0, 0), (5, 11, 9)), ((5, 0, 0), (13, 4, 9)),
                  ((5, 4, 0), (13, 11, 2)), ((5, 4, 2), (13, 11, 9))]
    one, ws = _both([thin], 4, arith, 0)
    assert _same(one, ws)


@pytest.mark.parametrize("arith", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_boundary_tile_shapes(orc, arith, mode):
    """Two boxes whose extents leave remainders under 32 x 16 tiles: a band of
    64 x 8 tiles under the first box's full tiles and an 8-wide column of
    8 x 64 tiles at its high x end (whose x-face ghosts come from the second
    box); both pass kernels bit-identical, the oracle's values within the
    bar."""
    dom = W.Domain((104, 40, 20), 1.0 / 40)
    inst = W.bumpy_instance(dom, 9)
    inst.boxes = [((0, 0, 0), (72, 40, 20)), ((72, 0, 0), (104, 40, 20))]
    lev = make_level([inst])
    ncls = lev.size_classes()[0]
    for c in range(ncls):
        lev.set_tuning(c, 32, 8)
    shapes = {(int(r[0]), int(r[5])) for r in lev.work_items()}
    assert (0, 64) in shapes and (0, 8) in shapes
    lev.close()
    one, ws = _both([inst], 4, arith, mode, tiles={c: (32, 8) for c in range(ncls)})
    assert _same(one, ws)
    ou, op = orc.rk4_periodic(inst.u, inst.pi, inst.c2, dom.h, inst.dt, 4)
    assert rel_err(ws[0][0], ou) <= TOL and rel_err(ws[1][0], op) <= TOL


def _owner_change_level():
    """Four boxes of a 64 x 24 x 40 periodic domain: across both x faces of
    box 0 the owner of the ghosts changes along y (box 1 below y = 10) and,
    inside a z-run, along z (boxes 2 and 3 above y = 10, split at z = 17);
    box widths 26 and 38 leave ragged tiles at the x faces."""
    dom = W.Domain((64, 24, 40), 1.0 / 24)
    inst = W.bumpy_instance(dom, 11)
    inst.boxes = [((0, 0, 0), (26, 24, 40)), ((26, 0, 0), (64, 10, 40)),
                  ((26, 10, 0), (64, 24, 17)), ((26, 10, 17), (64, 24, 40))]
    return inst


@pytest.mark.parametrize("arith", [0, 1])
@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("tx,tz", [(16, 40), (32, 8), (64, 13)])
def test_x_face_ghosts_read_from_their_owners(orc, arith, mode, tx, tz):
    """The warp-specialised producers read x-face ghosts from the boxes that
    own them (those rows are not gathered), with work items at an x face
    ending their z-run where the owner changes: bit-identical to the
    one-role kernels, which gather every ghost, in every launch mode and for
    z-runs that the owner change cuts, and within the bar of the oracle."""
    inst = _owner_change_level()
    one, ws = _both([inst], 5, arith, mode, tiles={c: (tx, tz) for c in range(3)})
    assert _same(one, ws)
    ou, op = orc.rk4_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, 5)
    assert rel_err(ws[0][0], ou) <= TOL and rel_err(ws[1][0], op) <= TOL


def test_ensemble_per_domain_dt_and_self_periodic_boxes():
    insts = [W.bumpy_instance(W.Domain((n, n, n), 1.0 / n), 5000 + i)
             for i, n in enumerate((24, 32, 40, 24, 56, 48))]
    insts.append(W.bumpy_instance(W.Domain((3, 2, 5), 0.2), 9))   # odd x: gathered
    insts.append(W.bumpy_instance(W.Domain((2, 2, 2), 0.5), 10))  # extent 2
    one, ws = _both(insts, 5, 1, 0)
    assert _same(one, ws)


@pytest.mark.parametrize("tx,tz", [(16, 5), (32, 37), (64, 100), (64, 3), (16, 74)])
def test_every_tile_and_z_run(tx, tz):
    dom = W.Domain((44, 38, 75), 1.0 / 40)
    inst = W.bumpy_instance(dom, 12)
    one, ws = _both([inst], 3, 1, 0, tiles={0: (tx, tz)})
    assert _same(one, ws)


def test_256_box_bit_identical():
    inst = W.single_box(256, seed=2)
    one, ws = _both([inst], 3, 1, 0)
    assert _same(one, ws)


@pytest.mark.parametrize("arith", [0, 1])
def test_taped_gradient_bit_identical(orc, arith):
    import torch
    inst = W.gradient_problem(20, 4)
    res = []
    for kind in (0, 1):
        lev = make_level([inst])
        lev.set_arith(arith)
        lev.set_fusion(2)
        lev.set_pass_kernel(kind)
        t = lambda a, fill=0.0: upload(lev, [a], fill)
        su = W.random_direction(inst.dom.shape, 43)
        g = [torch.empty(lev.field_size, dtype=torch.float64, device="cuda") for _ in range(3)]
        uT = torch.empty_like(g[0])
        lev.grad(t(inst.u), t(inst.pi), t(inst.c2, 1.0), inst.dt, 11, 4, t(su), None, *g,
                 u_T=uT)
        lev.sync()
        res.append([lev.gather(x)[0] for x in g + [uT]])
        lev.close()
    for a, b in zip(res[0], res[1]):
        assert np.array_equal(a, b)
    ou, op, oc = orc.grad_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, 11, 4, su,
                                   np.zeros_like(su))
    assert rel_err(res[1][0], ou) <= 1e-10 and rel_err(res[1][2], oc) <= 1e-10


@pytest.mark.parametrize("arith", [0, 1])
def test_adjoint_passes_bit_identical_on_uneven_level_and_ensemble(orc, arith):
    """The warp-specialised adjoint passes (which also form the adjoint
    combination) against the one-role adjoint passes and combination kernel:
    the same gradients bit for bit on an uneven 16-box level (ghosts of
    every stencil input gathered) and on an ensemble with per-domain step
    sizes; and the oracle's within 1e-10."""
    import torch
    uneven = W.uneven_level(n=(64, 48, 40), h=1.0 / 48, levels=4, seed=6, box_seed=31)
    ens = [W.bumpy_instance(W.Domain((n, n, n), 1.0 / n), 5000 + i)
           for i, n in enumerate((24, 32, 16))]
    for insts, nsteps, ckpt in (([uneven], 7, 3), (ens, 5, 2)):
        res = []
        for kind in (0, 1):
            lev = make_level(insts)
            lev.set_arith(arith)
            lev.set_fusion(2)
            lev.set_pass_kernel(kind)
            up = lambda arrs, fill=0.0: upload(lev, arrs, fill)
            su = [W.random_direction(i.dom.shape, 60 + k) for k, i in enumerate(insts)]
            sp = [W.random_direction(i.dom.shape, 70 + k) for k, i in enumerate(insts)]
            g = [torch.empty(lev.field_size, dtype=torch.float64, device="cuda")
                 for _ in range(3)]
            lev.grad(up([i.u for i in insts]), up([i.pi for i in insts]),
                     up([i.c2 for i in insts], 1.0), [i.dt for i in insts], nsteps, ckpt,
                     up(su), up(sp), *g)
            lev.sync()
            res.append([lev.gather(x) for x in g])
            lev.close()
        for a, b in zip(res[0], res[1]):
            for x, y in zip(a, b):
                assert np.array_equal(x, y)
        for k, inst in enumerate(insts):
            ou, op, oc = orc.grad_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt,
                                           nsteps, ckpt, su[k], sp[k])
            assert rel_err(res[1][0][k], ou) <= 1e-10
            assert rel_err(res[1][1][k], op) <= 1e-10
            assert rel_err(res[1][2][k], oc) <= 1e-10


def test_bounded_wait_runs_out_and_is_reported():
    """A wait test withholds the consumers' release of the ring slots: the
    producers' wait gives up after its limit, the kernel ends, sc_level_sync
    reports SC_EDEVICE; the next steps run normally and match a fresh run."""
    import torch
    from paper_1308_1343_gb300 import binding as B
    inst = W.bumpy_instance(W.Domain((48, 40, 36), 1.0 / 40), 3)
    lev = make_level([inst])
    lev.set_fusion(2)
    lev.set_pass_kernel(1)
    u, pi = upload(lev, [inst.u]), upload(lev, [inst.pi])
    c2 = upload(lev, [inst.c2], fill=1.0)
    lev.arm_wait_test()
    lev.rk4_step(u, pi, c2, inst.dt, 1, B.SC_MODE_BATCHED)
    with pytest.raises(B.ScError) as e:
        lev.sync()
    assert e.value.code == B.SC_EDEVICE and "bounded wait" in str(e.value)
    # the context and the level are usable: a normal run from fresh inputs
    u, pi = upload(lev, [inst.u]), upload(lev, [inst.pi])
    lev.rk4_step(u, pi, c2, inst.dt, 3, B.SC_MODE_GRAPH)
    lev.sync()
    torch.cuda.synchronize()
    _, u1, p1 = run_gpu([inst], 3, 1, 0, fuse=2)
    assert np.array_equal(lev.gather(u)[0], u1[0]) and np.array_equal(lev.gather(pi)[0], p1[0])
    lev.close()
