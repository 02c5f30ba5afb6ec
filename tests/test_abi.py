"""CPU tests of the C-ABI library: it builds, loads and exports every symbol
its headers declare; the host-side bboxset algebra equals brute-force point
enumeration; levels are validated; the layout follows its documented rule;
and the ghost-exchange lists equal the oracle's brute-force owner map
exactly.  No test here launches a kernel."""
import ctypes
import os
import random
import re

import numpy as np
import pytest

from oracle import pointset as P
from paper_1308_1343_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def B():
    from paper_1308_1343_gb300 import binding, build
    build.build()
    binding.lib()
    return binding


def _declared_functions():
    names = []
    for h in ("sc_level.h", "sc_bboxset.h", "sc_hierarchy.h", "sc_dist.h"):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"\b(sc_\w+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(B):
    names = _declared_functions()
    assert len(names) >= 25
    lib = B.lib()
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(B.declared_symbols()) == names


# ----------------------------------------------------------------------------
# bboxset algebra vs brute force
# ----------------------------------------------------------------------------

def _arr(boxes):
    a = np.ascontiguousarray(np.array([list(lo) + list(hi) for lo, hi in boxes],
                                      dtype=np.int64).reshape(-1, 6))
    return a


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _lib_op(B, op, A, Bx):
    a, b = _arr(A), _arr(Bx)
    n = ctypes.c_int64()
    B.check(B.lib().sc_bboxset_op(op, _p(a), len(A), _p(b), len(Bx), None, 0, ctypes.byref(n)))
    out = np.zeros((max(n.value, 1), 6), dtype=np.int64)
    B.check(B.lib().sc_bboxset_op(op, _p(a), len(A), _p(b), len(Bx), _p(out), n.value,
                                  ctypes.byref(n)))
    return out[:n.value]


def _points_of(rows):
    s = set()
    total = 0
    for r in rows:
        pts = P.box_points(r[:3], r[3:])
        total += len(pts)
        s |= pts
    return s, total


def _rand_boxes(rng, k, n=8):
    out = []
    for _ in range(k):
        lo = [rng.randrange(0, n) for _ in range(3)]
        hi = [rng.randrange(l, n + 1) for l in lo]
        out.append((lo, hi))
    return out


OPS = {0: lambda a, b: a | b, 1: lambda a, b: a & b, 2: lambda a, b: a - b,
       3: lambda a, b: a ^ b}


@pytest.mark.parametrize("seed", range(40))
def test_set_operations_match_point_enumeration(B, seed):
    rng = random.Random(seed)
    A = _rand_boxes(rng, rng.randrange(1, 5))
    C = _rand_boxes(rng, rng.randrange(1, 5))
    pa, pc = P.union_of_boxes(A), P.union_of_boxes(C)
    for op, f in OPS.items():
        rows = _lib_op(B, op, A, C)
        pts, total = _points_of(rows)
        assert pts == f(pa, pc), (op, A, C)
        assert total == len(pts)  # the normalized boxes are disjoint
        assert all((r[3:] > r[:3]).all() for r in rows)


@pytest.mark.parametrize("seed", range(20))
def test_derivative_expand_shift_size(B, seed):
    rng = random.Random(100 + seed)
    A = _rand_boxes(rng, rng.randrange(1, 5))
    pa = P.union_of_boxes(A)
    a = _arr(A)
    n = ctypes.c_int64()
    B.check(B.lib().sc_bboxset_derivative(_p(a), len(A), None, 0, ctypes.byref(n)))
    pts = np.zeros((max(n.value, 1), 3), dtype=np.int64)
    B.check(B.lib().sc_bboxset_derivative(_p(a), len(A), _p(pts), n.value, ctypes.byref(n)))
    assert {tuple(int(v) for v in p) for p in pts[:n.value]} == P.full_derivative(pa, 3)
    B.check(B.lib().sc_bboxset_size(_p(a), len(A), ctypes.byref(n)))
    assert n.value == len(pa)
    lo_by = [rng.randrange(0, 3) for _ in range(3)]
    hi_by = [rng.randrange(0, 3) for _ in range(3)]
    v = [rng.randrange(-5, 6) for _ in range(3)]
    L3 = ctypes.c_int64 * 3
    B.check(B.lib().sc_bboxset_expand_shift(_p(a), len(A), L3(*lo_by), L3(*hi_by), L3(*v), None,
                                            0, ctypes.byref(n)))
    out = np.zeros((max(n.value, 1), 6), dtype=np.int64)
    B.check(B.lib().sc_bboxset_expand_shift(_p(a), len(A), L3(*lo_by), L3(*hi_by), L3(*v),
                                            _p(out), n.value, ctypes.byref(n)))
    got, _ = _points_of(out[:n.value])
    assert got == P.shift(P.expand(pa, lo_by, hi_by), v)


def test_paper_examples_through_library(B):
    # cuboid: 8 corner points (Sec. 2.2); L-shape extruded over one z-layer:
    # the 6 key points of the 2D shape on both faces z = 0 and z = 1
    cub = _arr([((1, 2, 3), (5, 7, 4))])
    n = ctypes.c_int64()
    pts = np.zeros((16, 3), dtype=np.int64)
    B.check(B.lib().sc_bboxset_derivative(_p(cub), 1, _p(pts), 16, ctypes.byref(n)))
    assert n.value == 8
    ell = _arr([((0, 0, 0), (4, 2, 1)), ((0, 2, 0), (2, 5, 1))])
    B.check(B.lib().sc_bboxset_derivative(_p(ell), 2, _p(pts), 16, ctypes.byref(n)))
    assert n.value == 12
    assert sorted({int(p[2]) for p in pts[:12]}) == [0, 1]


# ----------------------------------------------------------------------------
# level creation, validation, layout
# ----------------------------------------------------------------------------

def _level(boxes, doms):
    from paper_1308_1343_gb300.level import Level
    return Level(boxes, doms)


def test_invalid_levels_are_rejected(B):
    from paper_1308_1343_gb300.level import Level
    dom = [dict(hi=(16, 16, 16), h=0.1)]
    with pytest.raises(B.ScError, match="overlaps"):
        Level([((0, 0, 0), (10, 16, 16), 0), ((8, 0, 0), (16, 16, 16), 0)], dom)
    with pytest.raises(B.ScError, match="do not tile"):
        Level([((0, 0, 0), (8, 16, 16), 0)], dom)
    with pytest.raises(B.ScError, match="not inside"):
        Level([((0, 0, 0), (17, 16, 16), 0)], dom)
    with pytest.raises(B.ScError, match="edge < 2"):
        Level([((0, 0, 0), (1, 16, 16), 0), ((1, 0, 0), (16, 16, 16), 0)], dom)
    with pytest.raises(B.ScError, match="ghost"):
        Level([((0, 0, 0), (16, 16, 16), 0)], dom, ghost=3)
    with pytest.raises(B.ScError, match="bad domain"):
        Level([((0, 0, 0), (16, 16, 16), 1)], dom)


def test_layout_rule(B):
    inst = W.uneven_level(n=(64, 48, 32), h=1 / 32, levels=3, seed=3, box_seed=7)
    from paper_1308_1343_gb300.level import Level
    lev = Level.from_instances([inst])
    prev_end = 0
    for (off, dims, pitch), (lo, hi, d) in zip(lev.layout, lev.boxes):
        nx, ny, nz = dims
        assert dims == tuple(h - l for l, h in zip(lo, hi))
        assert off % 16 == 0
        assert pitch[0] == 1 and pitch[1] == -(-(nx + 4) // 16) * 16
        assert pitch[2] == pitch[1] * (ny + 4)
        start = off - 2 - 2 * pitch[1] - 2 * pitch[2]
        assert start >= prev_end
        prev_end = start + pitch[2] * (nz + 4)
    assert lev.field_size >= prev_end


# ----------------------------------------------------------------------------
# exchange lists vs the oracle's brute-force owner map (bit-exact)
# ----------------------------------------------------------------------------

def _rows_from_copies(copies):
    out = []
    for c in copies:
        sb, db = c[0], c[1]
        slo, dlo, ext = c[2:5], c[5:8], c[8:11]
        zz, yy, xx = np.meshgrid(np.arange(ext[2]), np.arange(ext[1]), np.arange(ext[0]),
                                 indexing="ij")
        o = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)
        n = len(o)
        rows = np.empty((n, 8), dtype=np.int64)
        rows[:, 0] = db
        rows[:, 1:4] = o + dlo
        rows[:, 4] = sb
        rows[:, 5:8] = o + slo
        out.append(rows)
    return np.concatenate(out) if out else np.zeros((0, 8), dtype=np.int64)


def _sorted_rows(r):
    return r[np.lexsort(r.T[::-1])]


def _check_level_exchange(orc, boxes_per_dom, doms):
    boxes = []
    for d, bl in enumerate(boxes_per_dom):
        boxes += [(lo, hi, d) for lo, hi in bl]
    lev = _level(boxes, doms)
    copies = lev.exchange_list()
    got = _rows_from_copies(copies)
    # no ghost point is written twice
    assert len(np.unique(got[:, :4], axis=0)) == len(got)
    want = []
    base = 0
    for d, bl in enumerate(boxes_per_dom):
        D = doms[d]
        rows = orc.ghost_owners([lo + hi for lo, hi in bl], tuple(D.get("lo", (0, 0, 0))) +
                                tuple(D["hi"]), D.get("periodic", 7))
        rows[:, 0] += base
        rows[:, 4] += base
        want.append(rows)
        base += len(bl)
    want = np.concatenate(want)
    assert np.array_equal(_sorted_rows(got), _sorted_rows(want))


def test_exchange_single_periodic_box(B, orc):
    _check_level_exchange(orc, [[((0, 0, 0), (12, 10, 8))]], [dict(hi=(12, 10, 8), h=0.1)])


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_exchange_bisected_level(B, orc, seed):
    n = (64, 48, 40)
    boxes = W.bisect_boxes(n, 4, seed)
    _check_level_exchange(orc, [boxes], [dict(hi=n, h=0.1)])


def test_exchange_uneven_64_box_level_reduced(B, orc):
    # the 64-box recipe of the uneven level on a smaller domain
    n = (128, 128, 64)
    boxes = W.bisect_boxes(n, 6, 30)
    assert len(boxes) == 64
    _check_level_exchange(orc, [boxes], [dict(hi=n, h=0.1)])


def test_exchange_thin_boxes_and_partial_periodicity(B, orc):
    n = (12, 9, 10)
    boxes = [((0, 0, 0), (2, 9, 10)), ((2, 0, 0), (5, 9, 10)), ((5, 0, 0), (12, 4, 10)),
             ((5, 4, 0), (12, 9, 10))]
    for per in (0, 1, 3, 5, 7):
        _check_level_exchange(orc, [boxes], [dict(hi=n, h=0.1, periodic=per)])


def test_exchange_multi_domain(B, orc):
    doms = [dict(hi=(8, 8, 8), h=0.1), dict(hi=(16, 8, 12), h=0.05),
            dict(lo=(3, 4, 5), hi=(13, 14, 15), h=0.2)]
    per = [[((0, 0, 0), (8, 8, 8))],
           W.bisect_boxes((16, 8, 12), 2, 5, quantum=2, min_edge=2),
           [((3, 4, 5), (8, 14, 15)), ((8, 4, 5), (13, 14, 15))]]
    _check_level_exchange(orc, per, doms)


def test_exchange_full_uneven_level_counts(B):
    # the full 512 x 512 x 256, 64-box level: every star ghost point of every
    # box is written exactly once, from an interior point of its owner
    inst = W.uneven_level()
    from paper_1308_1343_gb300.level import Level
    lev = Level.from_instances([inst])
    c = lev.exchange_list()
    ext = c[:, 8:11]
    total = int(np.prod(ext, axis=1).sum())
    want = sum(4 * ((h[0] - l[0]) * (h[1] - l[1]) + (h[1] - l[1]) * (h[2] - l[2]) +
                    (h[0] - l[0]) * (h[2] - l[2])) for l, h in inst.boxes)
    assert total == want
    N = np.array(inst.dom.n)
    for row in c:
        sb, db = row[0], row[1]
        slo, dlo, e = row[2:5], row[5:8], row[8:11]
        lo, hi = np.array(inst.boxes[sb][0]), np.array(inst.boxes[sb][1])
        assert (slo >= lo).all() and (slo + e <= hi).all()
        assert ((dlo - slo) % N == 0).all()


def test_level_too_large_is_rejected(B):
    from paper_1308_1343_gb300.level import Level
    n = (2048, 2048, 520)  # (2048+16) * (2048+4) * (520+4) > 2^31 doubles
    with pytest.raises(B.ScError, match="too large"):
        Level([((0, 0, 0), n, 0)], [dict(hi=n, h=0.1)])


def test_fusion_setting_and_tile_query(B):
    from paper_1308_1343_gb300.level import Level
    n = (32, 24, 16)
    lev = Level([((0, 0, 0), n, 0)], [dict(hi=n, h=0.1)])
    assert lev.get_fusion() == 2
    lev.set_fusion(1)
    assert lev.get_fusion() == 1
    lev.set_fusion(2)
    assert lev.get_fusion() == 2
    for bad in (0, 3, -1):
        with pytest.raises(B.ScError, match="stages_per_pass"):
            lev.set_fusion(bad)
    assert lev.get_fusion() == 2
    assert lev.get_staging() == B.SC_STAGING_REGISTERS
    lev.set_staging(B.SC_STAGING_SHARED)
    assert lev.get_staging() == B.SC_STAGING_SHARED
    for bad in (2, -1):
        with pytest.raises(B.ScError, match="staging"):
            lev.set_staging(bad)
    assert lev.get_staging() == B.SC_STAGING_SHARED
    tx, ty, tz = lev.get_tuning(0)
    assert tx in (16, 32, 64) and tx * ty == 512 and tz >= 1
    lev.set_tuning(0, 32, 12)
    assert lev.get_tuning(0) == (32, 16, 12)
    with pytest.raises(B.ScError, match="bad class"):
        lev.get_tuning(1)


def test_missing_library_fails_loudly(tmp_path):
    """Without the compiled library the Python API raises at the first call:
    there is no CPU path to fall back to."""
    import subprocess
    import sys
    code = (
        "from paper_1308_1343_gb300 import binding as B\n"
        "B.LIB_PATH = %r\n"
        "from paper_1308_1343_gb300.level import Level\n"
        "Level([((0, 0, 0), (8, 8, 8), 0)],\n"
        "      [dict(lo=(0, 0, 0), hi=(8, 8, 8), h=1 / 8, periodic=7)])\n"
    ) % str(tmp_path / "libsc_level.so")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode != 0
    assert "libsc_level.so is missing" in r.stderr
    assert "no CPU fallback" in r.stderr


def test_field_tensors_are_checked_before_any_call(B):
    """The Python layer checks what the C ABI cannot see behind a pointer:
    dtype, contiguity, element count and device of every field tensor, and
    the host buffers of the end-to-end call.  Each wrong argument raises
    before the library is called (no GPU is needed to see it)."""
    import torch
    from paper_1308_1343_gb300.level import Level
    lev = Level([((0, 0, 0), (8, 8, 8), 0)], [dict(lo=(0, 0, 0), hi=(8, 8, 8), h=1 / 8,
                                                  periodic=7)])
    n = lev.field_size
    good = torch.zeros(n, dtype=torch.float64)
    cases = [
        (torch.zeros(n, dtype=torch.float32), "dtype"),
        (torch.zeros(n - 1, dtype=torch.float64), "elements"),
        (torch.zeros(2 * n, dtype=torch.float64)[::2], "contiguous"),
        (good, "CUDA device"),
    ]
    for bad, why in cases:
        with pytest.raises(ValueError, match=why):
            lev.rk4_step(bad, good, good, 0.01, 1)
    with pytest.raises(TypeError):
        lev.fill_ghosts(np.zeros(n))
    with pytest.raises(ValueError, match="required"):
        lev.apply_laplacian(None, good)
    h = np.zeros(n)
    with pytest.raises(ValueError, match="u_out"):
        lev.rk4_step_host(h, h, h, 0.01, 1, u_out=np.zeros(n - 1), pi_out=np.zeros(n))
    with pytest.raises(ValueError, match="c2"):
        lev.rk4_step_host(h, h, h[::1].astype(np.float32), 0.01, 1)


def test_checked_build_compiles_and_exports_every_symbol(B):
    """The checked build (SC_BOUNDS_CHECK: traversal indices verified against
    their box on the device) compiles from the same sources and exports the
    same C ABI; the GPU test runs it."""
    from paper_1308_1343_gb300 import build
    path = build.build(checked=True)
    assert path.endswith("libsc_level_checked.so") and os.path.exists(path)
    lib = ctypes.CDLL(path)
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_bad_calls_fail_with_einval_before_any_device_work(B):
    """Host-side failure injection through the raw C ABI: a NULL level,
    NULL or misaligned field pointers, a bad mode or step count, aliasing
    fields and a missing tape all return SC_EINVAL with a message, without
    touching a GPU (none is present here)."""
    from paper_1308_1343_gb300.level import Level
    lev = Level([((0, 0, 0), (8, 8, 8), 0)], [dict(lo=(0, 0, 0), hi=(8, 8, 8), h=1 / 8,
                                                  periodic=7)])
    lib, h = B.lib(), lev._h
    ok = ctypes.c_void_p(1 << 20)    # aligned, never dereferenced here
    mis = ctypes.c_void_p((1 << 20) + 8)
    dt = (ctypes.c_double * 1)(0.01)

    def einval(rc, text):
        assert rc == B.SC_EINVAL
        assert text in lib.sc_last_error().decode()

    einval(lib.sc_level_rk4_step(None, ok, ok, ok, dt, 1, 1, 0, None), "NULL level")
    einval(lib.sc_level_rk4_step(h, mis, ok, ok, dt, 1, 1, 0, None), "aligned")
    einval(lib.sc_level_rk4_step(h, ok, None, ok, dt, 1, 1, 0, None), "aligned")
    einval(lib.sc_level_rk4_step(h, ok, ok, ok, dt, 1, -1, 0, None), "nsteps")
    einval(lib.sc_level_rk4_step(h, ok, ok, ok, dt, 1, 1, 9, None), "mode")
    einval(lib.sc_level_fill_ghosts(h, mis, None), "aligned")
    einval(lib.sc_level_apply_laplacian(h, ok, ok, None), "overlap")
    einval(lib.sc_level_misfit(h, mis, ok, ok, None, None), "pointer")
    einval(lib.sc_level_rk4_step_host(h, None, ok, ok, ok, ok, dt, 1, 1, None), "NULL")
    einval(lib.sc_level_backward_tape(h, ok, None, None, ok, ok, ok, None), "tape")
    bad = B.ScTile(24, 20, 8, 0)
    einval(lib.sc_level_set_tuning(h, 0, ctypes.byref(bad), 0), "tile_x")
    bad = B.ScTile(32, 16, 0, 0)
    einval(lib.sc_level_set_tuning(h, 0, ctypes.byref(bad), 0), "tile_z")


def test_noalloc_rejects_huge_extents_before_any_device_work(B):
    """The entry point without device allocation checks the box size in 64
    bits: extents near INT32_MAX, whose padded size would wrap a 32-bit
    product, and a padded box just over the static scratch return SC_EINVAL
    ('too large') before any CUDA call (none can succeed here: no GPU)."""
    lib = B.lib()
    ok = ctypes.c_void_p(1 << 20)    # aligned, never dereferenced
    big = 2147483644
    for n in ((2, big, 2), (big, 2, 2), (2, 2, big), (big, big, big), (65536, 65536, 2)):
        rc = lib.sc_box_rk4_step_noalloc(ok, ok, ok, n[0], n[1], n[2], 0.01, 0.0025, 1, None)
        assert rc == B.SC_EINVAL, n
        assert "too large" in lib.sc_last_error().decode(), n
    # padded size 16 * 64 * 516 = 528384 > 2^19 doubles: one plane too many
    rc = lib.sc_box_rk4_step_noalloc(ok, ok, ok, 12, 60, 512, 0.01, 0.0025, 1, None)
    assert rc == B.SC_EINVAL and "too large" in lib.sc_last_error().decode()
    rc = lib.sc_box_rk4_step_noalloc(ok, ok, ok, 1, 8, 8, 0.01, 0.0025, 1, None)
    assert rc == B.SC_EINVAL and "bad argument" in lib.sc_last_error().decode()
