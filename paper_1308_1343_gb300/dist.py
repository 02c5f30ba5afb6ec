"""A level distributed over ranks, one GPU per rank (include/sc_dist.h).

The boxes of a level are assigned to ranks (``partition``); each rank holds
a ``DistLevel``: the part of the level made of its own boxes, whose ghost
copies between local boxes are a local gather and whose ghost copies across
ranks form per-peer send and receive lists -- the communication schedule
that the paper derives from bboxset intersections (arXiv 1308.1343, Sec. 2).

Per RK4 step there are two exchanges, each of two fields: the state (u, pi)
before pass A and the stage fields w_2 before pass B.  An exchange is

    sc_dist_pack (kernel)  ->  transport  ->  sc_dist_unpack (kernel)

where the transport moves each peer's block of the send buffer into that
peer's receive buffer.  ``TorchTransport`` does it with torch.distributed
point-to-point operations, one batch per exchange (NCCL between GPUs, gloo
between CPU processes).  ``step_ranks`` runs several ranks' parts in one
process on one device, copying the blocks between their buffers: the same
schedule with sequential launches and no rank waiting for another.

Python marshals arguments and moves buffers; packing, unpacking and every
step of the method run in libsc_level.so.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

from . import binding as B
from .level import Level, _field, _stream, _torch


def partition(boxes: Sequence, nranks: int, method: int = B.SC_DIST_BISECT) -> List[int]:
    """Rank of each box (``sc_dist_partition``): boxes are (lo, hi, domain)."""
    cb, _ = Level._c_arrays(boxes, [dict(hi=(1, 1, 1), h=1.0)])
    out = (ctypes.c_int32 * max(len(boxes), 1))()
    B.check(B.lib().sc_dist_partition(cb, len(boxes), int(nranks), int(method), out))
    return [int(out[i]) for i in range(len(boxes))]


@dataclass
class Peer:
    peer: int            # the peer's rank
    send_points: int     # points of one field sent to it
    recv_points: int     # points of one field received from it
    send_offset: int     # offset (doubles) of its block in the send buffer
    recv_offset: int     # ... in the receive buffer


class DistLevel(Level):
    """Rank `rank`'s part of a level of `boxes` over `domains` distributed
    over `nranks` ranks by `rank_of_box` (default: ``partition``).  Field
    buffers, layout, ``boxes`` and ``gather`` cover this rank's boxes only;
    ``global_box[b]`` is the whole-level index of local box b."""

    def __init__(self, boxes, domains, nranks: int, rank: int,
                 rank_of_box: Optional[Sequence[int]] = None,
                 method: int = B.SC_DIST_BISECT, ghost: int = 2):
        lib = B.lib()
        if rank_of_box is None:
            rank_of_box = partition(boxes, nranks, method)
        self.rank_of_box = [int(r) for r in rank_of_box]
        cb, cd = self._c_arrays(boxes, domains)
        ranks = (ctypes.c_int32 * max(len(boxes), 1))(*self.rank_of_box)
        h = ctypes.c_void_p()
        B.check(lib.sc_dist_create(cb, len(boxes), cd, len(domains), int(ghost), ranks,
                                   int(nranks), int(rank), ctypes.byref(h)))
        mine = [b for b in range(len(boxes)) if self.rank_of_box[b] == rank]
        self._adopt(h, [boxes[b] for b in mine], domains)
        self.rank, self.nranks = int(rank), int(nranks)
        g = ctypes.c_int32()
        self.global_box = []
        for b in range(len(mine)):
            B.check(lib.sc_dist_global_box(h, b, ctypes.byref(g)))
            self.global_box.append(g.value)
        r, n, npeers = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        B.check(lib.sc_dist_info(h, ctypes.byref(r), ctypes.byref(n), ctypes.byref(npeers)))
        self.peers: List[Peer] = []
        for i in range(npeers.value):
            vals = [ctypes.c_int32()] + [ctypes.c_int64() for _ in range(4)]
            B.check(lib.sc_dist_peer(h, i, *[ctypes.byref(v) for v in vals]))
            self.peers.append(Peer(*[v.value for v in vals]))
        sd, rd = ctypes.c_int64(), ctypes.c_int64()
        B.check(lib.sc_dist_buffer_sizes(h, ctypes.byref(sd), ctypes.byref(rd)))
        self.send_doubles, self.recv_doubles = sd.value, rd.value
        self._send = self._recv = None

    # ---- schedule (host) ------------------------------------------------------

    def peer_list(self, i: int, recv: bool) -> np.ndarray:
        """(n, 11) int64 rows (src_box, dst_box, src_lo, dst_lo, ext) of peer
        i's copies: sent (src_box local, dst_box whole-level) or received
        (dst_box local, src_box whole-level)."""
        lib = B.lib()
        n = ctypes.c_int64()
        B.check(lib.sc_dist_list(self._h, int(i), int(recv), None, 0, ctypes.byref(n)))
        arr = (B.ScCopy * max(n.value, 1))()
        B.check(lib.sc_dist_list(self._h, int(i), int(recv), arr, n.value, ctypes.byref(n)))
        rows = np.zeros((n.value, 11), dtype=np.int64)
        for k in range(n.value):
            c = arr[k]
            rows[k] = [c.src_box, c.dst_box, *c.src_lo, *c.dst_lo, *c.ext]
        return rows

    # ---- exchange and step ------------------------------------------------------

    def buffers(self, device="cuda"):
        """The level's send and receive buffers (allocated once)."""
        torch = _torch()
        if self._send is None:
            self._send = torch.zeros(max(self.send_doubles, 2), dtype=torch.float64,
                                     device=device)
            self._recv = torch.zeros(max(self.recv_doubles, 2), dtype=torch.float64,
                                     device=device)
        return self._send, self._recv

    def _buf(self, t, n, name):
        return _field(t, n, name) if n > 0 else (t.data_ptr() if t is not None else None)

    def pack(self, which: int, u, pi, send, stream=None):
        f = self._f
        pu = f(u, "u") if which == B.SC_DIST_STATE else None
        pp = f(pi, "pi") if which == B.SC_DIST_STATE else None
        B.check(B.lib().sc_dist_pack(self._h, int(which), pu, pp,
                                     self._buf(send, self.send_doubles, "send"),
                                     _stream(stream)))

    def unpack(self, which: int, recv, u, pi, stream=None):
        f = self._f
        pu = f(u, "u") if which == B.SC_DIST_STATE else None
        pp = f(pi, "pi") if which == B.SC_DIST_STATE else None
        B.check(B.lib().sc_dist_unpack(self._h, int(which),
                                       self._buf(recv, self.recv_doubles, "recv"), pu, pp,
                                       _stream(stream)))

    def rk4_begin(self, u, pi, c2, dt, stream=None):
        d, nd = self._dt(dt)
        f = self._f
        B.check(B.lib().sc_dist_rk4_begin(self._h, f(u, "u"), f(pi, "pi"), f(c2, "c2"), d, nd,
                                          _stream(stream)))

    def rk4_pass(self, u, pi, which_pass: int, stream=None):
        f = self._f
        B.check(B.lib().sc_dist_rk4_pass(self._h, f(u, "u"), f(pi, "pi"), int(which_pass),
                                         _stream(stream)))

    def exchange(self, which: int, u, pi, transport, stream=None):
        send, recv = self.buffers()
        self.pack(which, u, pi, send, stream)
        transport(self.peers, send, recv)
        self.unpack(which, recv, u, pi, stream)

    def rk4_step(self, u, pi, c2, dt, nsteps: int, transport=None, stream=None, mode=None):
        """nsteps RK4 steps of this rank's part, exchanging with the other
        ranks through `transport` (default: TorchTransport on the default
        process group).  Every rank must make the same calls."""
        transport = transport or TorchTransport()
        self.rk4_begin(u, pi, c2, dt, stream)
        for _ in range(int(nsteps)):
            self.exchange(B.SC_DIST_STATE, u, pi, transport, stream)
            self.rk4_pass(u, pi, 0, stream)
            self.exchange(B.SC_DIST_STAGE, None, None, transport, stream)
            self.rk4_pass(u, pi, 1, stream)

    def misfit_total(self, u, u_obs, seed=None, group=None, stream=None):
        """The whole level's misfit loss: this rank's share (sc_level_misfit)
        summed over ranks by one all-reduce; seed is this rank's dL/du."""
        import torch.distributed as dist
        loss, seed = self.misfit(u, u_obs, seed, stream)
        total = loss.reshape(1).clone()
        dist.all_reduce(total, op=dist.ReduceOp.SUM, group=group)
        return total[0], seed


class TorchTransport:
    """Moves every peer's block with torch.distributed point-to-point
    operations, all of one exchange in one batch (NCCL between GPUs, gloo
    between CPU processes).  Block i of `send` goes to peer i's rank, which
    receives it into its own block for this rank; the layouts match by
    construction (include/sc_dist.h)."""

    def __init__(self, group=None):
        self.group = group

    def __call__(self, peers: Sequence[Peer], send, recv):
        import torch.distributed as dist
        ops = []
        for p in peers:
            if p.send_points:
                ops.append(dist.P2POp(dist.isend,
                                      send[p.send_offset:p.send_offset + 2 * p.send_points],
                                      p.peer, self.group))
            if p.recv_points:
                ops.append(dist.P2POp(dist.irecv,
                                      recv[p.recv_offset:p.recv_offset + 2 * p.recv_points],
                                      p.peer, self.group))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()


def copy_blocks(levels: Sequence[DistLevel]):
    """Loopback transport of ranks held in one process: every rank's
    receive block for peer p is copied from p's send block for it."""
    by_rank = {L.rank: L for L in levels}
    for L in levels:
        _, recv = L.buffers()
        for p in L.peers:
            src = by_rank[p.peer]
            q = next(x for x in src.peers if x.peer == L.rank)
            n = 2 * p.recv_points
            assert n == 2 * q.send_points
            send, _ = src.buffers()
            recv[p.recv_offset:p.recv_offset + n].copy_(send[q.send_offset:q.send_offset + n])


def step_ranks(levels: Sequence[DistLevel], us, pis, c2s, dt, nsteps: int, stream=None):
    """nsteps RK4 steps of every rank's part held in this process (one
    device): the ranks advance pass by pass, packing, copying blocks and
    unpacking between passes; no launch waits on another rank."""
    for L, u, pi, c2 in zip(levels, us, pis, c2s):
        L.rk4_begin(u, pi, c2, dt, stream)
    for _ in range(int(nsteps)):
        for which in (B.SC_DIST_STATE, B.SC_DIST_STAGE):
            for L, u, pi in zip(levels, us, pis):
                send, _ = L.buffers()
                L.pack(which, u, pi, send, stream)
            copy_blocks(levels)
            for L, u, pi in zip(levels, us, pis):
                _, recv = L.buffers()
                L.unpack(which, recv, u, pi, stream)
                L.rk4_pass(u, pi, 0 if which == B.SC_DIST_STATE else 1, stream)
