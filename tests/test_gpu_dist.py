"""GPU tests of the distributed level (include/sc_dist.h) through the C ABI,
with every rank's part held in this one process on one GPU: the ranks
advance pass by pass and their send blocks are copied into the peers'
receive blocks between passes (dist.step_ranks), so no launch waits on
another rank.

* the exchange kernels: after pack, block copies, unpack and the local
  gather, every ghost of every box equals the oracle's ghost fill of the
  whole level, bit for bit;
* RK4 steps: in SC_ARITH_FP64 bit-identical to the one-level run of the
  same form; in the fixed-point form within 1e-12 of the oracle, including
  a spike in one rank's boundary data that another rank only sees through
  the exchange (the unpack raises that rank's exponent bound);
* the loss: the ranks' shares sum to the whole level's misfit;
* a non-finite value that arrives through the exchange is reported;
* the full 512 x 512 x 256 level of 64 boxes over 2 and 4 ranks."""
import os

import numpy as np
import pytest

from paper_1308_1343_gb300 import workloads as W

from gpu_helpers import rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1308_1343_gb300 import build
    build.build()


def _ranks(inst, nranks, method=1, arith=1):
    from paper_1308_1343_gb300.dist import DistLevel, partition
    boxes = [(lo, hi, 0) for lo, hi in inst.boxes]
    doms = [dict(hi=inst.dom.n, h=inst.dom.h, periodic=7)]
    owner = partition(boxes, nranks, method)
    levs = [DistLevel(boxes, doms, nranks, r, owner) for r in range(nranks)]
    for L in levs:
        L.set_arith(arith)
    return levs


def _gather_all(levs, fields, shape):
    """Whole-domain array from every rank's part."""
    out = np.full(shape, np.nan)
    for L, f in zip(levs, fields):
        buf = f.cpu().numpy()
        for b, (lo, hi, _) in enumerate(L.boxes):
            v = L._box_view(buf, b)
            out[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = v[2:-2, 2:-2, 2:-2]
    return out


@pytest.mark.parametrize("nranks,method", [(2, 1), (3, 0), (5, 1)])
def test_exchange_fills_every_ghost_like_the_oracle(orc, nranks, method):
    import torch
    from paper_1308_1343_gb300 import binding as B
    from paper_1308_1343_gb300.dist import copy_blocks
    inst = W.uneven_level(n=(64, 48, 40), h=1.0 / 48, levels=4, seed=6, box_seed=31)
    levs = _ranks(inst, nranks, method)
    rng = np.random.default_rng(3)
    u_h, p_h = rng.normal(size=(2,) + inst.dom.shape)
    us = [L.to_device([u_h], fill=np.nan) for L in levs]
    ps = [L.to_device([p_h], fill=np.nan) for L in levs]
    for L, u, p in zip(levs, us, ps):
        L.pack(B.SC_DIST_STATE, u, p, L.buffers()[0])
    copy_blocks(levs)
    for L, u, p in zip(levs, us, ps):
        L.unpack(B.SC_DIST_STATE, L.buffers()[1], u, p)
        L.fill_ghosts(u)
        L.fill_ghosts(p)
    torch.cuda.synchronize()
    boxes = [lo + hi for lo, hi in inst.boxes]
    for w, fs in ((u_h, us), (p_h, ps)):
        want = []
        for lo, hi in inst.boxes:
            a = np.full((hi[2] - lo[2] + 4, hi[1] - lo[1] + 4, hi[0] - lo[0] + 4), np.nan)
            a[2:-2, 2:-2, 2:-2] = w[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
            want.append(a)
        orc.fill_ghosts(boxes, (0, 0, 0) + inst.dom.n, 7, want)
        for L, f in zip(levs, fs):
            got = L.padded_boxes(f)
            for b, g in enumerate(L.global_box):
                assert np.array_equal(got[b], want[g], equal_nan=True), (L.rank, b)


def _single(inst, nsteps, arith):
    import torch
    from gpu_helpers import make_level, upload
    lev = make_level([inst])
    lev.set_arith(arith)
    lev.set_fusion(2)
    u, p = upload(lev, [inst.u]), upload(lev, [inst.pi])
    c2 = upload(lev, [inst.c2], fill=1.0)
    lev.rk4_step(u, p, c2, inst.dt, nsteps, 2)
    lev.sync()
    torch.cuda.synchronize()
    out = lev.gather(u)[0], lev.gather(p)[0]
    lev.close()
    return out


def _dist_run(inst, nranks, nsteps, arith, method=1):
    import torch
    from paper_1308_1343_gb300.dist import step_ranks
    levs = _ranks(inst, nranks, method, arith)
    us = [L.to_device([inst.u]) for L in levs]
    ps = [L.to_device([inst.pi]) for L in levs]
    cs = [L.to_device([inst.c2], fill=1.0) for L in levs]
    step_ranks(levs, us, ps, cs, inst.dt, nsteps)
    for L in levs:
        L.sync()
    torch.cuda.synchronize()
    shape = inst.dom.shape
    return levs, _gather_all(levs, us, shape), _gather_all(levs, ps, shape), us, ps


@pytest.mark.parametrize("nranks", [2, 3, 4])
def test_fp64_steps_bit_identical_to_one_level(nranks):
    inst = W.uneven_level(n=(64, 48, 40), h=1.0 / 48, levels=4, seed=6, box_seed=31)
    u1, p1 = _single(inst, 5, 0)
    _, u, p, _, _ = _dist_run(inst, nranks, 5, 0)
    assert np.array_equal(u, u1) and np.array_equal(p, p1)


@pytest.mark.parametrize("nranks,method", [(2, 1), (4, 0)])
def test_fixed_point_steps_vs_oracle(orc, nranks, method):
    inst = W.uneven_level(n=(64, 48, 40), h=1.0 / 48, levels=4, seed=6, box_seed=31)
    _, u, p, _, _ = _dist_run(inst, nranks, 6, 1, method)
    ou, op = orc.rk4_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, 6)
    assert rel_err(u, ou) <= TOL and rel_err(p, op) <= TOL


def test_spike_seen_only_through_the_exchange(orc):
    """A spike 1e6 times the pulse in the interior of one rank's box, two
    points from a face whose neighbour belongs to another rank: that rank's
    own data stay far below the spike, so only the raised exponent bound of
    the unpacked ghosts keeps its fixed-point conversion in range (no scale
    error) and its values within the bar."""
    from paper_1308_1343_gb300.dist import partition
    inst = W.uneven_level(n=(64, 48, 40), h=1.0 / 48, levels=4, seed=6, box_seed=31)
    boxes = [(lo, hi, 0) for lo, hi in inst.boxes]
    owner = partition(boxes, 2, 1)
    # a face of a rank-0 box whose neighbour across it is a rank-1 box
    spike = None
    for b, (lo, hi, _) in enumerate(boxes):
        if owner[b] != 0:
            continue
        for o, (lo2, hi2, _) in enumerate(boxes):
            if owner[o] == 1 and lo2[0] == hi[0] and lo2[1] < hi[1] and hi2[1] > lo[1] and \
                    lo2[2] < hi[2] and hi2[2] > lo[2]:
                y = (max(lo[1], lo2[1]) + min(hi[1], hi2[1])) // 2
                z = (max(lo[2], lo2[2]) + min(hi[2], hi2[2])) // 2
                spike = (hi[0] - 1, y, z)
                break
        if spike:
            break
    assert spike is not None
    u0 = inst.u.copy()
    u0[spike[2], spike[1], spike[0]] += 1e6 * np.abs(inst.u).max()
    big = W.Instance(inst.dom, u0, inst.pi, inst.c2, inst.dt)
    big.boxes = inst.boxes
    _, u, p, _, _ = _dist_run(big, 2, 3, 1)
    ou, op = orc.rk4_periodic(big.u, big.pi, big.c2, big.dom.h, big.dt, 3)
    assert rel_err(u, ou) <= TOL and rel_err(p, op) <= TOL


def test_loss_shares_sum_to_the_whole_level(orc):
    import torch
    inst = W.uneven_level(n=(64, 48, 40), h=1.0 / 48, levels=4, seed=6, box_seed=31)
    levs = _ranks(inst, 3)
    rng = np.random.default_rng(5)
    obs = rng.normal(size=inst.dom.shape)
    total = 0.0
    for L in levs:
        loss, _ = L.misfit(L.to_device([inst.u]), L.to_device([obs]))
        total += loss.item()
    want = orc.misfit_loss(inst.u, obs, inst.dom.h)
    assert abs(total - want) <= 1e-13 * abs(want)


def test_non_finite_value_through_the_exchange_is_reported():
    import torch
    from paper_1308_1343_gb300 import binding as B
    from paper_1308_1343_gb300.dist import step_ranks
    inst = W.uneven_level(n=(64, 48, 40), h=1.0 / 48, levels=4, seed=6, box_seed=31)
    levs = _ranks(inst, 2)
    L0 = levs[0]
    rows = L0.peer_list(0, False)  # a point rank 0 sends to rank 1
    b, lo = rows[0][0], rows[0][2:5]
    u = inst.u.copy()
    u[lo[2], lo[1], lo[0]] = np.nan
    us = [L.to_device([u]) for L in levs]
    ps = [L.to_device([inst.pi]) for L in levs]
    cs = [L.to_device([inst.c2], fill=1.0) for L in levs]
    step_ranks(levs, us, ps, cs, inst.dt, 1)
    torch.cuda.synchronize()
    with pytest.raises(B.ScError, match="non-finite"):
        levs[1].sync()
    for L in levs:
        try:
            L.sync()
        except B.ScError:
            pass


def test_passes_out_of_order_are_refused():
    from paper_1308_1343_gb300 import binding as B
    inst = W.uneven_level(n=(64, 48, 40), h=1.0 / 48, levels=4, seed=6, box_seed=31)
    L = _ranks(inst, 2)[0]
    u, p = L.to_device([inst.u]), L.to_device([inst.pi])
    c = L.to_device([inst.c2], fill=1.0)
    L.rk4_begin(u, p, c, inst.dt)
    with pytest.raises(B.ScError, match="pass 0 of the step first"):
        L.rk4_pass(u, p, 1)
    q = u.clone()
    with pytest.raises(B.ScError, match="given to sc_dist_rk4_begin"):
        L.rk4_pass(q, p, 0)
    L.rk4_pass(u, p, 0)
    with pytest.raises(B.ScError, match="previous step's pass 1"):
        L.rk4_pass(u, p, 0)
    L.sync()


@pytest.mark.parametrize("nranks", [2, 4])
def test_full_uneven_level_over_ranks(orc, nranks):
    """The benchmark's 512 x 512 x 256 level of 64 uneven boxes over 2 and
    4 ranks, 4 steps: FP64 bit-identical to the one-level run, fixed point
    within the bar of the oracle."""
    inst = W.uneven_level()
    u1, p1 = _single(inst, 4, 0)
    _, u, p, _, _ = _dist_run(inst, nranks, 4, 0)
    assert np.array_equal(u, u1) and np.array_equal(p, p1)
    del u1, p1, u, p
    _, u, p, _, _ = _dist_run(inst, nranks, 4, 1)
    orc.set_threads(os.cpu_count() or 1)
    try:
        ou, op = orc.rk4_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, 4)
    finally:
        orc.set_threads(1)
    assert rel_err(u, ou) <= TOL and rel_err(p, op) <= TOL
