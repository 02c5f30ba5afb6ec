"""GPU parity of the two-level hierarchy against the oracle
(oracle/hierarchy.py), through the C ABI: prolongation and restriction bit
for bit; hierarchy steps within 1e-12 relative max norm on the coarse level
and on the fine trusted region T (the buffer band is boundary-influenced by
design and refilled before every fine step); decomposition of either level
into several boxes changes no bit."""
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


def _fields(n, seed, lo, hi):
    """Fine-grid (2n)^3 inputs with the pulse in the refined region, and
    their coarse n^3 subsample."""
    fine = W.refined_pair(n, seed, lo, hi)
    sub = (slice(None, None, 2),) * 3
    return fine, fine.u[sub].copy(), fine.pi[sub].copy(), fine.c2[sub].copy()


def _region(a, lo, hi, pad=0):
    return a[lo[2] - pad:hi[2] + pad, lo[1] - pad:hi[1] + pad, lo[0] - pad:hi[0] + pad].copy()


def _setup(n, lo, hi, fine_boxes=None, coarse_boxes=None, arith=1, fuse=2, buffer=4):
    from paper_1308_1343_gb300.level import Hierarchy, Level
    c = Level(coarse_boxes or [((0, 0, 0), (n, n, n), 0)],
              [dict(hi=(n, n, n), h=1.0 / n, periodic=7)])
    f = Level([(a, b, 0) for a, b in (fine_boxes or [(lo, hi)])],
              [dict(lo=lo, hi=hi, h=0.5 / n, periodic=0)])
    for lev in (c, f):
        lev.set_arith(arith)
        lev.set_fusion(fuse)
    return c, f, Hierarchy(c, f, buffer=buffer)


def test_prolongation_vs_oracle():
    """Every prolongated point of both fields against the oracle: equal bit
    for bit on dyadic data (integers below 2^20: every product with the
    weights (-1, 9, 9, -1)/16 and every partial sum is exact, so the value is
    the interpolant itself in any evaluation order), and within 4 ulps of
    the data's scale on random data (the kernel chains fused multiply-adds,
    the oracle rounds each product and sum), at alpha = 0, 1/2 and 0.3."""
    import torch
    from oracle import hierarchy as H
    n, lo, hi = 24, (8, 6, 10), (38, 36, 36)
    c, f, h = _setup(n, lo, hi)
    rng = np.random.default_rng(4)
    eps = np.finfo(float).eps
    pts = h.prolongation_points()
    fu = torch.zeros(f.field_size, dtype=torch.float64, device="cuda")
    fp = torch.zeros_like(fu)
    dyadic = [rng.integers(-2 ** 20, 2 ** 20, size=(n, n, n)).astype(np.float64)
              for _ in range(4)]
    normal = [rng.normal(size=(n, n, n)) for _ in range(4)]
    for data, alphas, exact in ((dyadic, (0.0, 0.5), True), (normal, (0.0, 0.5, 0.3), False)):
        a0, a1, b0, b1 = data
        d = [c.to_device([x]) for x in data]
        for alpha in alphas:
            h.prolongate(d[0], d[1], d[2], d[3], alpha, fu, fp)
            torch.cuda.synchronize()
            for got, (x0, x1) in ((_read_points(f, fu, pts, lo), (a0, a1)),
                                  (_read_points(f, fp, pts, lo), (b0, b1))):
                want = H.prolongate(x0, x1, alpha, pts)
                if exact:
                    assert np.array_equal(got, want), alpha
                else:
                    scale = np.abs((1.0 - alpha) * x0 + alpha * x1).max()
                    assert np.abs(got - want).max() <= 4 * eps * scale, alpha


def test_prolongation_vs_order_free_tensor_sum():
    """The GPU prolongation against the tensor-product sum rounded once
    (exact_sums.tensor_sum_exact), which shares no evaluation order with
    the kernel or the oracle: equal bit for bit on dyadic data (every
    product and partial sum is then exact, in any order), and within 4 ulps
    of the data's scale on random data, at alpha = 0, 1/2 and 0.3."""
    import torch
    from exact_sums import tensor_sum_exact
    n, lo, hi = 24, (8, 6, 10), (38, 36, 36)
    c, f, h = _setup(n, lo, hi)
    rng = np.random.default_rng(8)
    pts = h.prolongation_points()
    sample = pts[::5]
    fu = torch.zeros(f.field_size, dtype=torch.float64, device="cuda")
    fp = torch.zeros_like(fu)
    eps = np.finfo(float).eps
    dyadic = [rng.integers(-2 ** 20, 2 ** 20, size=(n, n, n)).astype(np.float64)
              for _ in range(2)]
    normal = [rng.normal(size=(n, n, n)) for _ in range(2)]
    for (a0, a1), alphas, exact in ((dyadic, (0.0, 0.5), True), (normal, (0.0, 0.3), False)):
        d0, d1 = c.to_device([a0]), c.to_device([a1])
        for alpha in alphas:
            h.prolongate(d0, d1, d0, d1, alpha, fu, fp)
            torch.cuda.synchronize()
            got = _read_points(f, fu, sample, lo)
            data = (1.0 - alpha) * a0 + alpha * a1
            want = np.array([tensor_sum_exact(data, p) for p in sample])
            if exact:
                assert np.array_equal(got, want), alpha
            else:
                assert np.abs(got - want).max() <= 4 * eps * np.abs(data).max(), alpha


def _read_points(lev, t, pts, lo):
    """Values of a level field at level points (interior or ghost shell)."""
    buf = t.cpu().numpy()
    out = np.empty(len(pts))
    for k, p in enumerate(pts):
        for b, (blo, bhi, _) in enumerate(lev.boxes):
            inside = all(blo[d] - 2 <= p[d] < bhi[d] + 2 for d in range(3))
            nout = sum(not (blo[d] <= p[d] < bhi[d]) for d in range(3))
            if inside and nout <= 1:
                off, _, (_, py, pz) = lev.layout[b]
                out[k] = buf[off + (p[0] - blo[0]) + (p[1] - blo[1]) * py + (p[2] - blo[2]) * pz]
                break
    return out


def test_restriction_bit_exact():
    import torch
    n, lo, hi = 24, (8, 8, 8), (40, 40, 40)
    c, f, h = _setup(n, lo, hi, fine_boxes=[((8, 8, 8), (24, 40, 40)), ((24, 8, 8), (40, 40, 40))])
    rng = np.random.default_rng(5)
    fu_h, fp_h = rng.normal(size=(2, 32, 32, 32))
    cu_h, cp_h = rng.normal(size=(2, n, n, n))
    fu, fp = f.to_device([fu_h]), f.to_device([fp_h])
    cu, cp = c.to_device([cu_h]), c.to_device([cp_h])
    h.restrict(fu, fp, cu, cp)
    torch.cuda.synchronize()
    gu, gp = c.gather(cu)[0], c.gather(cp)[0]
    covered = np.zeros((n,) * 3, bool)
    for x, y, z in h.restriction_points():
        covered[z, y, x] = True
        assert gu[z, y, x] == fu_h[2 * z - lo[2], 2 * y - lo[1], 2 * x - lo[0]]
        assert gp[z, y, x] == fp_h[2 * z - lo[2], 2 * y - lo[1], 2 * x - lo[0]]
    assert covered.sum() == 12 ** 3
    assert np.array_equal(gu[~covered], cu_h[~covered])


def _run_both(n, lo, hi, nsteps, seed, arith, fuse, fine_boxes=None, coarse_boxes=None):
    import torch
    from oracle import hierarchy as H
    fine, cu_h, cp_h, cc_h = _fields(n, seed, lo, hi)
    hgrid = 1.0 / n
    dt = 0.25 * hgrid
    c, f, h = _setup(n, lo, hi, fine_boxes, coarse_boxes, arith, fuse)
    cu, cp, cc = c.to_device([cu_h]), c.to_device([cp_h]), c.to_device([cc_h], fill=1.0)
    fu = f.to_device([_region(fine.u, lo, hi)])
    fp = f.to_device([_region(fine.pi, lo, hi)])
    fc = f.to_device([_region(fine.c2, lo, hi)], fill=1.0)
    h.step(cu, cp, cc, fu, fp, fc, dt, nsteps)
    c.sync()
    f.sync()
    torch.cuda.synchronize()
    ou, op = cu_h, cp_h
    fu_p = _region(fine.u, lo, hi, 2)
    fp_p = _region(fine.pi, lo, hi, 2)
    fc_p = _region(fine.c2, lo, hi, 2)
    for _ in range(nsteps):
        ou, op, fu_p, fp_p = H.bo_step(ou, op, cc_h, hgrid, dt, fu_p, fp_p, fc_p, lo, hi, 4)
    return (c.gather(cu)[0], c.gather(cp)[0], f.gather(fu)[0], f.gather(fp)[0]), \
        (ou, op, fu_p[2:-2, 2:-2, 2:-2], fp_p[2:-2, 2:-2, 2:-2])


def _trusted(a, buffer=4):
    return a[buffer:-buffer, buffer:-buffer, buffer:-buffer]


def _t_err(got, want, buffer=4):
    """Max difference on T relative to the oracle field's max over the fine
    level R: the relative max norm of the level, taken where the two sides
    compute the same values (the fixed-point bound is level-relative)."""
    d = np.abs(_trusted(got, buffer) - _trusted(want, buffer)).max()
    return float(d / np.abs(want).max())


@pytest.mark.parametrize("fuse", [1, 2])
@pytest.mark.parametrize("arith", [0, 1])
def test_hierarchy_steps_match_oracle(arith, fuse):
    n, lo, hi = 24, (8, 8, 8), (40, 40, 40)
    gpu, ora = _run_both(n, lo, hi, 3, 21, arith, fuse)
    assert rel_err(gpu[0], ora[0]) <= TOL
    assert rel_err(gpu[1], ora[1]) <= TOL
    assert _t_err(gpu[2], ora[2]) <= TOL
    assert _t_err(gpu[3], ora[3]) <= TOL
    # and on T's own scale, with the pulse inside T
    assert rel_err(_trusted(gpu[2]), _trusted(ora[2])) <= 1e-11


def test_hierarchy_ragged_region_and_buffer_values_finite():
    n, lo, hi = 24, (7, 9, 6), (39, 35, 41)
    gpu, ora = _run_both(n, lo, hi, 2, 22, 1, 2)
    assert rel_err(gpu[0], ora[0]) <= TOL
    assert _t_err(gpu[2], ora[2]) <= TOL
    assert np.all(np.isfinite(gpu[2])) and np.all(np.isfinite(gpu[3]))


@pytest.mark.parametrize("fuse", [1, 2])
def test_decomposition_of_either_level_changes_no_bit(fuse):
    """Four fine boxes instead of one, and a coarse level of two boxes (cut
    away from the refined region's stencils) instead of one."""
    n, lo, hi = 32, (8, 8, 8), (40, 40, 40)
    one, _ = _run_both(n, lo, hi, 2, 23, 1, fuse)
    fb = [((8, 8, 8), (19, 40, 40)), ((19, 8, 8), (40, 25, 40)), ((19, 25, 8), (40, 40, 22)),
          ((19, 25, 22), (40, 40, 40))]
    cb = [((0, 0, 0), (26, n, n), 0), ((26, 0, 0), (n, n, n), 0)]
    many, _ = _run_both(n, lo, hi, 2, 23, 1, fuse, fine_boxes=fb, coarse_boxes=cb)
    assert np.array_equal(one[0], many[0]) and np.array_equal(one[1], many[1])
    assert np.array_equal(_trusted(one[2]), _trusted(many[2]))
    assert np.array_equal(_trusted(one[3]), _trusted(many[3]))


def test_non_periodic_level_takes_one_step_per_call():
    import torch
    from paper_1308_1343_gb300 import binding as B
    n, lo, hi = 24, (8, 8, 8), (40, 40, 40)
    c, f, h = _setup(n, lo, hi)
    z = torch.zeros(f.field_size, dtype=torch.float64, device="cuda")
    with pytest.raises(B.ScError, match="one step per call"):
        f.rk4_step(z, z.clone(), z.clone() + 1.0, 0.01, 2)


def test_full_size_step_vs_oracle(orc):
    """The benchmark's configuration (coarse 256^3, fine region of 256^3
    points, buffer 4, default launch form), one hierarchy step."""
    import os
    import torch
    from oracle import hierarchy as H
    n = 256
    lo, hi = (n // 2,) * 3, (3 * n // 2,) * 3
    coarse, (fu_h, fp_h, fc_h) = W.refined_fields(n, 7, lo, hi)
    from paper_1308_1343_gb300.level import Hierarchy, Level
    c = Level.from_instances([coarse])
    f = Level([(lo, hi, 0)], [dict(lo=lo, hi=hi, h=0.5 / n, periodic=0)])
    h = Hierarchy(c, f)
    cu, cp = c.to_device([coarse.u]), c.to_device([coarse.pi])
    cc = c.to_device([coarse.c2], fill=1.0)
    fu, fp, fc = f.to_device([fu_h]), f.to_device([fp_h]), f.to_device([fc_h], fill=1.0)
    h.step(cu, cp, cc, fu, fp, fc, coarse.dt, 1)
    c.sync()
    f.sync()
    torch.cuda.synchronize()
    gcu, gfu, gfp = c.gather(cu)[0], f.gather(fu)[0], f.gather(fp)[0]
    h.close()

    def pad(a):
        return np.pad(a, 2)  # ghosts: filled by prolongation before use
    orc.set_threads(os.cpu_count() or 1)
    try:
        ou, op, fu_p, fp_p = H.bo_step(coarse.u, coarse.pi, coarse.c2, 1.0 / n, coarse.dt,
                                       pad(fu_h), pad(fp_h), pad(fc_h), lo, hi, 4)
    finally:
        orc.set_threads(1)
    assert rel_err(gcu, ou) <= TOL
    assert _t_err(gfu, fu_p[2:-2, 2:-2, 2:-2]) <= TOL
    assert _t_err(gfp, fp_p[2:-2, 2:-2, 2:-2]) <= TOL


@pytest.mark.parametrize("fuse", [1, 2])
def test_bounds_follow_prolongated_and_restricted_values(fuse):
    """After the first step of a call each level reuses the exponent bounds
    of its last pass, raised by what prolongation or restriction wrote into
    it since.  A spike 1e6 times the pulse in the coarse data just outside
    the fine region reaches the fine level only through prolongation (band
    and ghost shell): four hierarchy steps in one call must still match the
    oracle, with no scale error raised."""
    import torch
    from oracle import hierarchy as H
    n, lo, hi = 24, (8, 8, 8), (40, 40, 40)
    fine = W.refined_pair(n, 31, lo, hi)
    rng = np.random.default_rng(8)
    # coarse points 1..2 outside R's low x face, on the coarse grid (even fine indices)
    for cz, cy in ((12, 12), (14, 10)):
        for cx in (2, 3):
            fine.u[2 * cz, 2 * cy, 2 * cx] += 1e6 * rng.normal()
    sub = (slice(None, None, 2),) * 3
    cu_h, cp_h, cc_h = fine.u[sub].copy(), fine.pi[sub].copy(), fine.c2[sub].copy()
    hgrid = 1.0 / n
    dt = 0.25 * hgrid
    c, f, h = _setup(n, lo, hi, fuse=fuse)
    cu, cp, cc = c.to_device([cu_h]), c.to_device([cp_h]), c.to_device([cc_h], fill=1.0)
    fu = f.to_device([_region(fine.u, lo, hi)])
    fp = f.to_device([_region(fine.pi, lo, hi)])
    fc = f.to_device([_region(fine.c2, lo, hi)], fill=1.0)
    h.step(cu, cp, cc, fu, fp, fc, dt, 4)
    c.sync()
    f.sync()  # raises if a value exceeded its level's exponent bound
    torch.cuda.synchronize()
    ou, op = cu_h, cp_h
    fu_p, fp_p = _region(fine.u, lo, hi, 2), _region(fine.pi, lo, hi, 2)
    fc_p = _region(fine.c2, lo, hi, 2)
    for _ in range(4):
        ou, op, fu_p, fp_p = H.bo_step(ou, op, cc_h, hgrid, dt, fu_p, fp_p, fc_p, lo, hi, 4)
    assert rel_err(c.gather(cu)[0], ou) <= TOL
    assert rel_err(c.gather(cp)[0], op) <= TOL
    assert _t_err(f.gather(fu)[0], fu_p[2:-2, 2:-2, 2:-2]) <= TOL
    assert _t_err(f.gather(fp)[0], fp_p[2:-2, 2:-2, 2:-2]) <= TOL
