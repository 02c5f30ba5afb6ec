"""Host logic of the work items (sc_level_work_items, no GPU): the items of
the batched launches tile every box exactly once; tiles are the size
class's width where a whole one fits and narrower ones (same thread count,
taller) for the rest of a box's width; a column of tiles at an x face whose
ghosts the warp-specialised passes read from the box that owns them never
runs a z-run across a change of that owner (the copies are re-derived here
from the exchange list and the layout); z-runs keep at most tile_z planes;
the order is the place of the tile in its domain."""
import numpy as np
import pytest

from paper_1308_1343_gb300 import workloads as W


def _level(inst):
    from paper_1308_1343_gb300.level import Level
    return Level.from_instances([inst])


def _owner_change():
    dom = W.Domain((64, 24, 40), 1.0 / 24)
    inst = W.bumpy_instance(dom, 11)
    inst.boxes = [((0, 0, 0), (26, 24, 40)), ((26, 0, 0), (64, 10, 40)),
                  ((26, 10, 0), (64, 24, 17)), ((26, 10, 17), (64, 24, 40))]
    return inst


def _owner_reads(lev):
    """(box, side) -> list of (y0, y1, z0, z1) of the x-face copies that are
    read from their owners: two ghost columns of an even-wide box that does
    not tile its domain alone, both ends 16-byte aligned, rows and planes
    inside the box."""
    out = {}
    boxes = lev.boxes
    for c in lev.exchange_list():
        sb, db = int(c[0]), int(c[1])
        slo, dlo, ext = c[2:5], c[5:8], c[8:11]
        lo, hi, _ = boxes[db]
        side = 0 if dlo[0] == lo[0] - 2 else (1 if dlo[0] == hi[0] else -1)
        if side < 0 or ext[0] != 2 or (hi[0] - lo[0]) % 2:
            continue
        dom = lev.domains[boxes[db][2]]
        alone = tuple(lo) == tuple(dom["lo"]) and tuple(hi) == tuple(dom["hi"])
        if alone and dom.get("periodic", 7) == 7:
            continue  # a box alone in its periodic domain wraps its ghosts
        soff, _, (_, spy, spz) = lev.layout[sb]
        doff, _, (_, dpy, dpz) = lev.layout[db]
        slo_b = boxes[sb][0]
        src = soff + (slo[0] - slo_b[0]) + (slo[1] - slo_b[1]) * spy + (slo[2] - slo_b[2]) * spz
        dst = doff + (dlo[0] - lo[0]) + (dlo[1] - lo[1]) * dpy + (dlo[2] - lo[2]) * dpz
        if src % 2 or dst % 2:
            continue
        if not (lo[1] <= dlo[1] and dlo[1] + ext[1] <= hi[1] and
                lo[2] <= dlo[2] and dlo[2] + ext[2] <= hi[2]):
            continue
        out.setdefault((db, side), []).append(
            (dlo[1] - lo[1], dlo[1] - lo[1] + ext[1], dlo[2] - lo[2], dlo[2] - lo[2] + ext[2]))
    return out


def _check(lev, tiles):
    items = lev.work_items()
    assert items.dtype == np.int32 and items.shape[1] == 6
    boxes = lev.boxes
    ncls, cls_of = lev.size_classes()
    reads = _owner_reads(lev)
    seen = {}
    cols = {b: set() for b in range(len(boxes))}  # tile columns (x0, y0, width, rows)
    for box, x0, y0, z0, nz_run, w in items.tolist():
        lo, hi, _ = boxes[box]
        n = [hi[d] - lo[d] for d in range(3)]
        t = lev.get_tuning(cls_of[box])
        # the class's tile (512 threads' worth of points per plane), a
        # narrower and taller one only where a tile twice as wide would not
        # fit, a wider and flatter one only over the last band of rows when
        # that band is at most half a tile tall
        assert w in (8, 16, 32, 64) and x0 % 8 == 0
        rows = t[1] * t[0] // w
        if w < t[0]:
            assert x0 + 2 * w > n[0], (box, x0, w, n[0])
            assert y0 % rows == 0
        elif w > t[0]:
            full = n[1] // t[1] * t[1]
            assert y0 == full and 0 < n[1] - full <= rows < t[1], (box, y0, w, n[1])
        else:
            assert y0 % rows == 0
        assert 0 <= x0 < n[0] and 0 <= y0 < n[1] and 0 <= z0 and z0 + nz_run <= n[2]
        assert 1 <= nz_run <= t[2]
        cols[box].add((x0, y0, w, rows))
        for z in range(z0, z0 + nz_run):
            key = (box, x0, y0, z)
            assert key not in seen, key
            seen[key] = True
        # no owner change of a read x-face row inside the run
        for side, at_face in ((0, x0 == 0), (1, x0 + w >= n[0])):
            if not at_face:
                continue
            for (ya, yb, za, zb) in reads.get((box, side), []):
                for zc in (za, zb):
                    assert not (z0 < zc < z0 + nz_run), (box, side, z0, nz_run, zc)
    # the tile columns cover every box's (x, y) extent exactly once, each over
    # all of its planes
    for b, (lo, hi, _) in enumerate(boxes):
        n = [hi[d] - lo[d] for d in range(3)]
        cover = np.zeros((n[1], n[0]), dtype=np.int32)
        for (x0, y0, w, rows) in cols[b]:
            cover[y0:y0 + rows, x0:x0 + w] += 1
            for z in range(n[2]):
                assert (b, x0, y0, z) in seen, (b, x0, y0, z)
        assert (cover == 1).all(), b
    assert len(seen) == sum(len(cols[b]) * (hi[2] - lo[2])
                            for b, (lo, hi, _) in enumerate(boxes))
    # launch order: domain, then z, y, x of the tile's first point
    keys = []
    for box, x0, y0, z0, _, _ in items.tolist():
        lo, _, d = boxes[box]
        keys.append((d, lo[2] + z0, lo[1] + y0, lo[0] + x0))
    assert keys == sorted(keys)
    return items, reads


@pytest.mark.parametrize("tiles", [None, (16, 40), (32, 8), (64, 13), (32, 5)])
def test_owner_change_level(tiles):
    inst = _owner_change()
    lev = _level(inst)
    if tiles:
        for c in range(lev.size_classes()[0]):
            lev.set_tuning(c, *tiles)
    items, reads = _check(lev, tiles)
    # box 0's faces are read from boxes 1-3, whose owner changes at z = 17:
    # its edge columns have a run boundary there
    assert reads.get((0, 1)) and any(z0 == 17 for b, x0, _, z0, _, _ in items.tolist()
                                     if b == 0)


@pytest.mark.parametrize("tiles", [None, (32, 32), (16, 64)])
def test_uneven_levels(tiles):
    for inst in (W.uneven_level(n=(64, 48, 40), h=1.0 / 48, levels=4, seed=6, box_seed=31),
                 W.uneven_level()):
        lev = _level(inst)
        if tiles:
            for c in range(lev.size_classes()[0]):
                lev.set_tuning(c, *tiles)
        items, reads = _check(lev, tiles)
        assert reads  # the level has x faces read from their owners


@pytest.mark.parametrize("nranks,method", [(2, 1), (3, 0)])
def test_distributed_ranks(nranks, method):
    """Every rank's part of a distributed uneven level: its own items and
    its own x-face reads (copies from boxes of other ranks arrive through
    the exchange and are not among them)."""
    from paper_1308_1343_gb300.dist import DistLevel, partition
    inst = W.uneven_level(n=(64, 48, 40), h=1.0 / 48, levels=4, seed=6, box_seed=31)
    boxes = [(lo, hi, 0) for lo, hi in inst.boxes]
    doms = [dict(hi=inst.dom.n, h=inst.dom.h, periodic=7)]
    owner = partition(boxes, nranks, method)
    total = 0
    for r in range(nranks):
        lev = DistLevel(boxes, doms, nranks, r, owner)
        for c in range(lev.size_classes()[0]):
            lev.set_tuning(c, 32, 8)
        items, _ = _check(lev, (32, 8))
        total += len(items)
    assert total > 0


def test_single_box_and_ensemble():
    lev = _level(W.single_box(64, 2))
    items, reads = _check(lev, None)
    assert not reads
    insts = [W.bumpy_instance(W.Domain((n, n, n), 1.0 / n), 5000 + i)
             for i, n in enumerate((24, 40, 32))]
    from paper_1308_1343_gb300.level import Level
    lev = Level.from_instances(insts)
    items, reads = _check(lev, None)
    assert not reads
    assert sorted(set(items[:, 0].tolist())) == [0, 1, 2]


@pytest.mark.parametrize("nx,ny,tx,want", [
    (40, 64, 32, [(0, 32), (32, 8)]),
    (104, 64, 32, [(0, 32), (32, 32), (64, 32), (96, 8)]),
    (56, 64, 32, [(0, 32), (32, 16), (48, 8)]),
    (120, 64, 64, [(0, 64), (64, 32), (96, 16), (112, 8)]),
    (64, 64, 32, [(0, 32), (32, 32)]),
    (5, 64, 16, [(0, 8)]),
    (21, 64, 16, [(0, 16), (16, 8)]),
    # few rows: one tile of the narrowest width that holds the rest takes
    # fewer tiles than the halved widths (1 against 2)
    (56, 16, 32, [(0, 32), (32, 32)]),
    (24, 16, 32, [(0, 32)]),
    (88, 8, 64, [(0, 64), (64, 32)]),
    # a tie keeps the halved widths
    (56, 32, 32, [(0, 32), (32, 16), (48, 8)]),
])
def test_tile_columns(nx, ny, tx, want):
    """The tile columns of one box: whole tiles of the class's width, then
    for the rest the halved widths down to 8 or one tile of the narrowest
    width that holds it, whichever takes fewer tiles over the box's rows."""
    inst = W.bumpy_instance(W.Domain((nx, ny, 6), 1.0 / ny), 3)
    lev = _level(inst)
    lev.set_tuning(0, tx, 8)
    items, _ = _check(lev, (tx, 8))
    got = sorted({(x0, w) for _, x0, _, _, _, w in items.tolist()})
    assert got == want
    # rows: 512 threads' worth of points per tile plane (no short last band here)
    for _, x0, y0, _, _, w in items.tolist():
        assert y0 % (512 // w) == 0


@pytest.mark.parametrize("nx,ny,tx,want", [
    (64, 24, 32, [(0, 0, 32), (0, 16, 64), (32, 0, 32)]),
    (96, 40, 32, [(0, 0, 32), (0, 16, 32), (0, 32, 64), (32, 0, 32), (32, 16, 32),
                  (64, 0, 32), (64, 16, 32), (64, 32, 32)]),
    (40, 24, 32, [(0, 0, 32), (0, 16, 32), (32, 0, 8)]),
    (48, 36, 16, [(0, 0, 16), (0, 32, 32), (16, 0, 16), (32, 0, 16), (32, 32, 16)]),
    (128, 36, 16, [(0, 0, 16), (0, 32, 64), (16, 0, 16), (32, 0, 16), (48, 0, 16), (64, 0, 16),
                   (64, 32, 64), (80, 0, 16), (96, 0, 16), (112, 0, 16)]),
    (48, 44, 16, [(0, 0, 16), (0, 32, 32), (16, 0, 16), (32, 0, 16), (32, 32, 16)]),
    (64, 28, 32, [(0, 0, 32), (0, 16, 32), (32, 0, 32), (32, 16, 32)]),
])
def test_last_row_band(nx, ny, tx, want):
    """The last band of rows under the full-width columns, when at most half
    a tile tall: the flattest tiles that hold it (up to 64 wide), each as
    wide as fits, down to the class's tile (tile_y = 512 / tile_x)."""
    inst = W.bumpy_instance(W.Domain((nx, ny, 6), 1.0 / ny), 3)
    lev = _level(inst)
    lev.set_tuning(0, tx, 8)
    items, _ = _check(lev, (tx, 8))
    assert sorted({(x0, y0, w) for _, x0, y0, _, _, w in items.tolist()}) == want


def test_item_shapes_fit_the_kernels():
    """Every item's tile fits what the traversal kernels hold: a (TX + 4) x
    (TY + 4) halo tile of at most 816 elements (the 64 x 8 tile's, the size of
    their shared-memory tile buffers) and at most one halo pair per thread
    (4 TX/2 + 2 TY <= 256), with TY = 512 / TX."""
    insts = [W.uneven_level(), W.uneven_level(n=(64, 48, 40), h=1.0 / 48, levels=4, seed=6,
                                              box_seed=31)]
    thin = W.bumpy_instance(W.Domain((13, 11, 9), 1.0 / 11), 7)
    thin.boxes = [((0, 0, 0), (2, 11, 9)), ((2, 0, 0), (5, 11, 9)), ((5, 0, 0), (13, 4, 9)),
                  ((5, 4, 0), (13, 11, 2)), ((5, 4, 2), (13, 11, 9))]
    insts.append(thin)
    levels = [[i] for i in insts] + [W.ensemble(count=12)]
    for group in levels:
        from paper_1308_1343_gb300.level import Level
        lev = Level.from_instances(group)
        for tiles in (None, (16, 32), (32, 32), (64, 32)):
            if tiles:
                for c in range(lev.size_classes()[0]):
                    lev.set_tuning(c, *tiles)
            shapes = {int(w) for w in lev.work_items()[:, 5]}
            for w in shapes:
                ty = 512 // w
                assert w in (8, 16, 32, 64)
                assert (w + 4) * (ty + 4) <= 816 and 4 * (w // 2) + 2 * ty <= 256


@pytest.mark.parametrize("tx,floor_unev,floor_ens", [(16, 0.96, 0.93), (32, 0.97, 0.95),
                                                     (64, 0.97, 0.95)])
def test_tile_slots_hold_points(tx, floor_unev, floor_ens):
    """The share of tile slots (512 points per tile plane) that hold points of
    a box, on the benchmark's 64-box level and 256-cube ensemble: with one
    ragged tile per remainder it was 0.87 on the level (32-wide tiles); the
    boundary tile shapes keep it near 0.98."""
    from paper_1308_1343_gb300.level import Level
    for insts, floor in (([W.uneven_level()], floor_unev), (W.ensemble(count=256), floor_ens)):
        lev = Level.from_instances(insts)
        for c in range(lev.size_classes()[0]):
            lev.set_tuning(c, tx, 32)
        items = lev.work_items()
        slots = 512 * int(items[:, 4].astype(np.int64).sum())
        pts = sum((hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]) for lo, hi, _ in lev.boxes)
        assert pts / slots >= floor, (tx, pts / slots)
        lev.close()


def test_work_items_errors():
    import ctypes
    from paper_1308_1343_gb300 import binding as B
    lev = _level(_owner_change())
    n = ctypes.c_int64()
    with pytest.raises(B.ScError):
        B.check(B.lib().sc_level_work_items(lev._h, None, 4, ctypes.byref(n)))
    with pytest.raises(B.ScError):
        B.check(B.lib().sc_level_work_items(lev._h, None, 0, None))
