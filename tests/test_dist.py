"""CPU tests of the distributed level (include/sc_dist.h), no GPU:

* the partition: every rank gets boxes, the greedy split is balanced within
  one box, the spatial bisection moves fewer ghost points across ranks;
* the schedule: over all ranks, the local exchange lists plus the received
  copies are exactly the oracle's brute-force owner map of the whole level,
  and what rank r sends to p is, copy for copy and in order, what p
  receives from r;
* the exchange itself on two gloo ranks (separate processes): each packs
  its send blocks from host copies of its boxes in the buffer layout the
  header states, torch.distributed moves them (the library's transport
  class), each unpacks and applies its local copies, and then every ghost
  of every box equals the oracle's ghost fill of the whole level, bit for
  bit;
* calls the one-GPU entry points refuse for a distributed level fail with
  SC_EINVAL before any device work."""
import ctypes
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1308_1343_gb300 import workloads as W


@pytest.fixture(scope="session")
def B():
    from paper_1308_1343_gb300 import binding, build
    build.build()
    binding.lib()
    return binding


def _spec(n=(64, 48, 40), levels=4, seed=6):
    boxes = [(lo, hi, 0) for lo, hi in W.bisect_boxes(n, levels, seed)]
    return boxes, [dict(hi=n, h=1.0 / n[1], periodic=7)]


def _points(b):
    return int(np.prod(np.array(b[1]) - np.array(b[0])))


def _cross_points(boxes, doms, ranks):
    from paper_1308_1343_gb300.level import Level
    ex = Level(boxes, doms).exchange_list()
    return int(sum(np.prod(r[8:11]) for r in ex if ranks[r[0]] != ranks[r[1]]))


@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("nranks", [1, 2, 3, 4, 8, 16])
def test_partition_is_valid_balanced_and_deterministic(B, method, nranks):
    from paper_1308_1343_gb300.dist import partition
    boxes, _ = _spec()
    r = partition(boxes, nranks, method)
    assert r == partition(boxes, nranks, method)
    assert sorted(set(r)) == list(range(nranks))
    load = np.zeros(nranks)
    for b, k in zip(boxes, r):
        load[k] += _points(b)
    if method == B.SC_DIST_GREEDY:
        assert load.max() <= load.mean() + max(_points(b) for b in boxes)
    # the whole level is assigned
    assert load.sum() == sum(_points(b) for b in boxes)


def test_bisection_moves_fewer_ghost_points_than_greedy(B):
    from paper_1308_1343_gb300.dist import partition
    inst = W.uneven_level(n=(128, 128, 64), h=1.0 / 64, levels=6, seed=3, box_seed=30)
    boxes = [(lo, hi, 0) for lo, hi in inst.boxes]
    doms = [dict(hi=inst.dom.n, h=inst.dom.h, periodic=7)]
    for n in (2, 4, 8):
        g = _cross_points(boxes, doms, partition(boxes, n, B.SC_DIST_GREEDY))
        s = _cross_points(boxes, doms, partition(boxes, n, B.SC_DIST_BISECT))
        assert s < g, n


def test_partition_and_create_reject_bad_requests(B):
    from paper_1308_1343_gb300.dist import DistLevel, partition
    boxes, doms = _spec()
    with pytest.raises(B.ScError, match="fewer boxes than ranks"):
        partition(boxes, len(boxes) + 1)
    with pytest.raises(B.ScError, match="nranks"):
        partition(boxes, 0)
    with pytest.raises(B.ScError, match="method"):
        partition(boxes, 2, 7)
    with pytest.raises(B.ScError, match="owns no box"):
        DistLevel(boxes, doms, 2, 0, [0] * len(boxes))
    with pytest.raises(B.ScError, match="rank out of range"):
        DistLevel(boxes, doms, 2, 0, [0, 5] + [1] * (len(boxes) - 2))
    with pytest.raises(B.ScError, match="bad rank"):
        DistLevel(boxes, doms, 2, 2)
    nonper = [dict(doms[0], periodic=3)]
    with pytest.raises(B.ScError, match="periodic"):
        DistLevel(boxes, nonper, 2, 0)


def _rows(copies, src_map, dst_map):
    """Point rows (dst_box, p, src_box, q) of copy rows, boxes mapped to
    whole-level indices."""
    out = []
    for c in copies:
        sb, db = src_map(c[0]), dst_map(c[1])
        slo, dlo, ext = c[2:5], c[5:8], c[8:11]
        zz, yy, xx = np.meshgrid(np.arange(ext[2]), np.arange(ext[1]), np.arange(ext[0]),
                                 indexing="ij")
        o = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)
        rows = np.empty((len(o), 8), dtype=np.int64)
        rows[:, 0] = db
        rows[:, 1:4] = o + dlo
        rows[:, 4] = sb
        rows[:, 5:8] = o + slo
        out.append(rows)
    return np.concatenate(out) if out else np.zeros((0, 8), dtype=np.int64)


def _sorted(r):
    return r[np.lexsort(r.T[::-1])]


@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("nranks", [2, 3, 5])
def test_schedule_is_the_whole_exchange_split_by_rank(B, orc, method, nranks):
    from paper_1308_1343_gb300.dist import DistLevel, partition
    boxes, doms = _spec()
    ranks = partition(boxes, nranks, method)
    levs = [DistLevel(boxes, doms, nranks, r, ranks) for r in range(nranks)]
    got = []
    for L in levs:
        g = L.global_box
        assert g == [b for b in range(len(boxes)) if ranks[b] == L.rank]
        got.append(_rows(L.exchange_list(), lambda b: g[b], lambda b: g[b]))
        total_send = total_recv = 0
        for i, p in enumerate(L.peers):
            assert p.send_offset == total_send and p.recv_offset == total_recv
            total_send += 2 * p.send_points
            total_recv += 2 * p.recv_points
            recv = L.peer_list(i, True)
            assert int(np.prod(recv[:, 8:11], axis=1).sum()) == p.recv_points
            got.append(_rows(recv, lambda b: b, lambda b: g[b]))
            # what p receives from L is what L sends to p, copy for copy
            P = levs[p.peer]
            j = [q.peer for q in P.peers].index(L.rank)
            sent = L.peer_list(i, False)
            theirs = P.peer_list(j, True)
            assert len(sent) == len(theirs)
            assert np.array_equal(_rows(sent, lambda b: g[b], lambda b: b),
                                  _rows(theirs, lambda b: b, lambda b: P.global_box[b]))
        assert (L.send_doubles, L.recv_doubles) == (total_send, total_recv)
        assert L.peers == sorted(L.peers, key=lambda p: p.peer)
    got = np.concatenate(got)
    assert len(np.unique(got[:, :4], axis=0)) == len(got)  # no ghost written twice
    D = doms[0]
    want = orc.ghost_owners([lo + hi for lo, hi, _ in boxes], (0, 0, 0) + tuple(D["hi"]), 7)
    assert np.array_equal(_sorted(got), _sorted(want))


def test_one_gpu_calls_refuse_a_distributed_level(B):
    """rk4_step, the taped forward and a hierarchy refuse a distributed
    level, and the split step refuses a plain one: SC_EINVAL with a message,
    before any device work (no GPU here)."""
    from paper_1308_1343_gb300.dist import DistLevel
    from paper_1308_1343_gb300.level import Level
    boxes, doms = _spec()
    L = DistLevel(boxes, doms, 2, 0)
    plain = Level(boxes, doms)
    lib, h = B.lib(), L.handle
    ok = ctypes.c_void_p(1 << 20)
    ok2 = ctypes.c_void_p(1 << 21)
    dt = (ctypes.c_double * 1)(0.01)

    def einval(rc, text):
        assert rc == B.SC_EINVAL
        assert text in lib.sc_last_error().decode()

    einval(lib.sc_level_rk4_step(h, ok, ok2, ok, dt, 1, 1, 0, None), "distributed level")
    einval(lib.sc_level_forward_tape(h, ok, ok2, ok, dt, 1, 2, 1, None, None, None),
           "distributed")
    hh = ctypes.c_void_p()
    einval(lib.sc_hierarchy_create(h, plain.handle, 2, 4, ctypes.byref(hh)), "distributed")
    einval(lib.sc_dist_rk4_begin(plain.handle, ok, ok2, ok, dt, 1, None), "not a distributed")
    einval(lib.sc_dist_pack(plain.handle, 0, ok, ok2, ok, None), "not a distributed")
    einval(lib.sc_dist_rk4_pass(h, ok, ok2, 0, None), "sc_dist_rk4_begin first")
    einval(lib.sc_dist_rk4_begin(h, ok, ok, ok, dt, 1, None), "different buffers")
    einval(lib.sc_dist_pack(h, 0, ok, ok2, None, None), "exchange buffer")


# ---- two gloo ranks ---------------------------------------------------------------

def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _box_view(L, buf, b):
    off, (nx, ny, nz), (_, py, pz) = L.layout[b]
    start = off - 2 - 2 * py - 2 * pz
    it = buf.itemsize
    return np.lib.stride_tricks.as_strided(buf[start:], shape=(nz + 4, ny + 4, nx + 4),
                                           strides=(pz * it, py * it, it))


def _rect(L, buf, b, lo, ext):
    """View of the points lo .. lo + ext of local box b (level coordinates)."""
    blo = L.boxes[b][0]
    v = _box_view(L, buf, b)
    x, y, z = (int(lo[d] - blo[d] + 2) for d in range(3))
    return v[z:z + ext[2], y:y + ext[1], x:x + ext[0]]


def _exchange_rank(rank, world, port, out):
    """One rank: pack, move by gloo, unpack, local copies; compare with the
    oracle's fill of the whole level."""
    import torch
    import torch.distributed as dist
    from oracle import oracle as orc
    from paper_1308_1343_gb300.dist import DistLevel, TorchTransport, partition
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = (64, 48, 40)
        boxes, doms = _spec(n)
        ranks = partition(boxes, world)
        L = DistLevel(boxes, doms, world, rank, ranks)
        rng = np.random.default_rng(11)
        whole = [rng.normal(size=(n[2], n[1], n[0])) for _ in range(2)]  # u, pi
        bufs = [L.scatter([w], fill=np.nan) for w in whole]
        send = np.zeros(max(L.send_doubles, 1))
        recv = np.zeros(max(L.recv_doubles, 1))
        for i, p in enumerate(L.peers):
            pos = p.send_offset
            for c in L.peer_list(i, False):
                vals = [_rect(L, f, c[0], c[2:5], c[8:11]).ravel() for f in bufs]
                k = len(vals[0])
                send[pos:pos + k] = vals[0]
                send[pos + p.send_points:pos + p.send_points + k] = vals[1]
                pos += k
        TorchTransport()(L.peers, torch.from_numpy(send), torch.from_numpy(recv))
        for i, p in enumerate(L.peers):
            pos = p.recv_offset
            for c in L.peer_list(i, True):
                ext = c[8:11]
                k = int(np.prod(ext))
                for f, shift in ((bufs[0], 0), (bufs[1], p.recv_points)):
                    _rect(L, f, c[1], c[5:8], ext)[...] = \
                        recv[pos + shift:pos + shift + k].reshape(ext[2], ext[1], ext[0])
                pos += k
        for c in L.exchange_list():
            for f in bufs:
                _rect(L, f, c[1], c[5:8], c[8:11])[...] = _rect(L, f, c[0], c[2:5], c[8:11])
        ok = True
        D = doms[0]
        for w, f in zip(whole, bufs):
            fields = []
            for lo, hi, _ in boxes:
                a = np.full((hi[2] - lo[2] + 4, hi[1] - lo[1] + 4, hi[0] - lo[0] + 4), np.nan)
                a[2:-2, 2:-2, 2:-2] = w[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
                fields.append(a)
            orc.fill_ghosts([lo + hi for lo, hi, _ in boxes], (0, 0, 0) + tuple(D["hi"]), 7,
                            fields)
            for b, g in enumerate(L.global_box):
                ok = ok and np.array_equal(np.array(_box_view(L, f, b)), fields[g],
                                           equal_nan=True)
        out[rank] = (bool(ok), len(L.peers), L.send_doubles)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_exchange_ghosts_bit_exact():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_exchange_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] and res[1][0], res
    assert res[0][1] == res[1][1] == 1 and res[0][2] > 0
