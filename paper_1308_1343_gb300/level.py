"""Python API over the C ABI: ``Level`` and the ``WaveRK4`` autograd Function.

PyTorch provides device memory and streams only; every step of the path
runs in libsc_level.so.  Field buffers are flat float64 tensors of
``level.field_size`` entries in the level layout (see include/sc_level.h).
``scatter`` / ``gather`` move whole-domain numpy arrays into and out of that
layout on the host (data marshalling, no arithmetic).
"""
from __future__ import annotations

import ctypes
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import binding as B

Box3 = Tuple[Tuple[int, int, int], Tuple[int, int, int]]


def _torch():
    import torch
    return torch


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return t.data_ptr()


def _field(t, n: int, name: str, optional: bool = False) -> Optional[int]:
    """Device pointer of a field tensor after the checks the C ABI cannot
    make (it sees only a pointer): a contiguous float64 CUDA tensor on the
    current device holding at least n elements.  Raises ValueError or
    TypeError otherwise, before any kernel could read or write past it."""
    if t is None:
        if optional:
            return None
        raise ValueError("%s: a field tensor is required" % name)
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s: expected a torch tensor, got %s" % (name, type(t).__name__))
    if t.dtype != torch.float64:
        raise ValueError("%s: dtype %s, fields are float64" % (name, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s: not contiguous" % name)
    if t.numel() < n:
        raise ValueError("%s: %d elements, the level's fields hold %d" % (name, t.numel(), n))
    if not t.is_cuda or t.device.index != torch.cuda.current_device():
        raise ValueError("%s: on %s, not on the current CUDA device" % (name, t.device))
    return t.data_ptr()


def _host_field(a, n: int, name: str) -> int:
    """Address of a host field buffer: a C-contiguous float64 numpy array of
    exactly n elements."""
    if not isinstance(a, np.ndarray) or a.dtype != np.float64:
        raise ValueError("%s: expected a float64 numpy array" % name)
    if not a.flags.c_contiguous or a.size != n:
        raise ValueError("%s: expected a contiguous array of %d elements" % (name, n))
    if name.endswith("_out") and not a.flags.writeable:
        raise ValueError("%s: not writeable" % name)
    return a.ctypes.data


def _stream(stream) -> Optional[int]:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class Level:
    """A level: boxes tiling one or more domains, ghost width 2."""

    def __init__(self, boxes: Sequence[Tuple[Sequence[int], Sequence[int], int]],
                 domains: Sequence[dict], ghost: int = 2):
        lib = B.lib()
        nb, nd = len(boxes), len(domains)
        cb, cd = self._c_arrays(boxes, domains)
        h = ctypes.c_void_p()
        B.check(lib.sc_level_create(cb, nb, cd, nd, int(ghost), ctypes.byref(h)))
        self._adopt(h, boxes, domains)

    @staticmethod
    def _c_arrays(boxes, domains):
        """ctypes arrays of sc_box and sc_domain."""
        nb, nd = len(boxes), len(domains)
        cb = (B.ScBox * max(nb, 1))()
        for i, (lo, hi, d) in enumerate(boxes):
            cb[i].lo[:] = [int(v) for v in lo]
            cb[i].hi[:] = [int(v) for v in hi]
            cb[i].domain = int(d)
        cd = (B.ScDomain * max(nd, 1))()
        for i, D in enumerate(domains):
            cd[i].lo[:] = [int(v) for v in D.get("lo", (0, 0, 0))]
            cd[i].hi[:] = [int(v) for v in D["hi"]]
            cd[i].h = float(D["h"])
            cd[i].periodic = int(D.get("periodic", 7))
        return cb, cd

    def _adopt(self, h, boxes, domains):
        """Take ownership of level handle h whose stored boxes are `boxes`."""
        lib = B.lib()
        self._h = h
        self.boxes = [(tuple(int(v) for v in lo), tuple(int(v) for v in hi), int(d))
                      for lo, hi, d in boxes]
        self.domains = [dict(lo=tuple(D.get("lo", (0, 0, 0))), hi=tuple(D["hi"]),
                             h=float(D["h"]), periodic=int(D.get("periodic", 7)))
                        for D in domains]
        nb = len(self.boxes)
        n = ctypes.c_int64()
        B.check(lib.sc_level_field_size(h, ctypes.byref(n)))
        self.field_size = n.value
        self.layout = []
        for b in range(nb):
            off = ctypes.c_int64()
            dims = (ctypes.c_int64 * 3)()
            pitch = (ctypes.c_int64 * 3)()
            B.check(lib.sc_level_box_layout(h, b, ctypes.byref(off), dims, pitch))
            self.layout.append((off.value, tuple(dims), tuple(pitch)))

    # ---- construction helpers --------------------------------------------

    @classmethod
    def from_instances(cls, instances) -> "Level":
        """One domain per workloads.Instance, tiled by its boxes."""
        boxes, doms = [], []
        for d, inst in enumerate(instances):
            doms.append(dict(hi=inst.dom.n, h=inst.dom.h, periodic=7))
            for lo, hi in inst.boxes:
                boxes.append((lo, hi, d))
        return cls(boxes, doms)

    def close(self):
        if getattr(self, "_h", None):
            B.lib().sc_level_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # ---- host-side layout marshalling -------------------------------------

    def _box_view(self, buf: np.ndarray, b: int) -> np.ndarray:
        off, (nx, ny, nz), (_, py, pz) = self.layout[b]
        start = off - 2 - 2 * py - 2 * pz
        it = buf.itemsize
        return np.lib.stride_tricks.as_strided(buf[start:], shape=(nz + 4, ny + 4, nx + 4),
                                               strides=(pz * it, py * it, it))

    def scatter(self, arrays: Sequence[np.ndarray], fill: float = 0.0) -> np.ndarray:
        """Whole-domain arrays (one per domain, shape (nz, ny, nx)) -> a host
        field buffer; ghosts and padding get `fill`."""
        buf = np.full(self.field_size, fill, dtype=np.float64)
        for b, (lo, hi, d) in enumerate(self.boxes):
            dlo = self.domains[d]["lo"]
            a = arrays[d]
            v = self._box_view(buf, b)
            v[2:-2, 2:-2, 2:-2] = a[lo[2] - dlo[2]:hi[2] - dlo[2], lo[1] - dlo[1]:hi[1] - dlo[1],
                                    lo[0] - dlo[0]:hi[0] - dlo[0]]
        return buf

    def gather(self, buf) -> List[np.ndarray]:
        """Field buffer (numpy or tensor) -> whole-domain arrays."""
        if not isinstance(buf, np.ndarray):
            buf = buf.detach().cpu().numpy()
        out = []
        for D in self.domains:
            n = [D["hi"][i] - D["lo"][i] for i in range(3)]
            out.append(np.empty((n[2], n[1], n[0])))
        for b, (lo, hi, d) in enumerate(self.boxes):
            dlo = self.domains[d]["lo"]
            v = self._box_view(buf, b)
            out[d][lo[2] - dlo[2]:hi[2] - dlo[2], lo[1] - dlo[1]:hi[1] - dlo[1],
                   lo[0] - dlo[0]:hi[0] - dlo[0]] = v[2:-2, 2:-2, 2:-2]
        return out

    def padded_boxes(self, buf) -> List[np.ndarray]:
        """Copies of every box's padded (nz+4, ny+4, nx+4) array."""
        if not isinstance(buf, np.ndarray):
            buf = buf.detach().cpu().numpy()
        return [np.array(self._box_view(buf, b)) for b in range(len(self.boxes))]

    def to_device(self, arrays_or_buf, fill: float = 0.0, device="cuda"):
        torch = _torch()
        buf = arrays_or_buf
        if not isinstance(buf, np.ndarray) or buf.ndim != 1:
            buf = self.scatter(arrays_or_buf, fill)
        return torch.from_numpy(buf).to(device)

    def new_field(self, fill: float = 0.0, device="cuda"):
        torch = _torch()
        return torch.full((self.field_size,), fill, dtype=torch.float64, device=device)

    # ---- queries ------------------------------------------------------------

    def exchange_list(self) -> np.ndarray:
        """(n, 11) int64 rows: src_box, dst_box, src_lo[3], dst_lo[3], ext[3]."""
        lib = B.lib()
        n = ctypes.c_int64()
        B.check(lib.sc_level_exchange_list(self._h, None, 0, ctypes.byref(n)))
        arr = (B.ScCopy * max(n.value, 1))()
        B.check(lib.sc_level_exchange_list(self._h, arr, n.value, ctypes.byref(n)))
        rows = np.zeros((n.value, 11), dtype=np.int64)
        for i in range(n.value):
            c = arr[i]
            rows[i] = [c.src_box, c.dst_box, *c.src_lo, *c.dst_lo, *c.ext]
        return rows

    def work_items(self) -> np.ndarray:
        """(n, 6) int32 rows of the batched launches' work items in launch
        order: box, x0, y0, z0, planes of the z-run, tile_x (the item's tile
        is tile_x x 512 / tile_x points: the size class's tile, or a
        narrower or flatter one at a box's remainder)."""
        lib = B.lib()
        n = ctypes.c_int64()
        B.check(lib.sc_level_work_items(self._h, None, 0, ctypes.byref(n)))
        arr = np.zeros((max(n.value, 1), 6), dtype=np.int32)
        B.check(lib.sc_level_work_items(
            self._h, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), n.value,
            ctypes.byref(n)))
        return arr[:n.value]

    def size_classes(self):
        lib = B.lib()
        n = ctypes.c_int32()
        cls = (ctypes.c_int32 * len(self.boxes))()
        B.check(lib.sc_level_size_classes(self._h, ctypes.byref(n), cls))
        return n.value, list(cls)

    def launch_count(self) -> int:
        n = ctypes.c_int64()
        B.check(B.lib().sc_level_launch_count(self._h, ctypes.byref(n)))
        return n.value

    # ---- configuration --------------------------------------------------------

    def set_arith(self, arith: int):
        B.check(B.lib().sc_level_set_arith(self._h, int(arith)))

    def set_tuning(self, cls: int, tile_x: int, tile_z: int, ctas_per_sm: int = 0):
        t = B.ScTile(int(tile_x), 512 // int(tile_x), int(tile_z), 0)
        B.check(B.lib().sc_level_set_tuning(self._h, int(cls), ctypes.byref(t), int(ctas_per_sm)))

    def get_tuning(self, cls: int):
        """(tile_x, tile_y, tile_z) of size class `cls`."""
        t = B.ScTile()
        B.check(B.lib().sc_level_get_tuning(self._h, int(cls), ctypes.byref(t)))
        return t.tile_x, t.tile_y, t.tile_z

    def set_fusion(self, stages_per_pass: int):
        """RK4 stages per stencil pass of rk4_step (1 or 2)."""
        B.check(B.lib().sc_level_set_fusion(self._h, int(stages_per_pass)))

    def get_fusion(self) -> int:
        n = ctypes.c_int32()
        B.check(B.lib().sc_level_get_fusion(self._h, ctypes.byref(n)))
        return n.value

    def set_pass_kernel(self, kind: int):
        """Kernels of the two-stage passes: binding.SC_PASS_ONE_ROLE or
        binding.SC_PASS_WARP_SPECIALISED."""
        B.check(B.lib().sc_level_set_pass_kernel(self._h, int(kind)))

    def get_pass_kernel(self) -> int:
        n = ctypes.c_int32()
        B.check(B.lib().sc_level_get_pass_kernel(self._h, ctypes.byref(n)))
        return n.value

    def arm_wait_test(self):
        """Failure-detection tests: the next warp-specialised pass launch
        withholds its ring slots so that its bounded wait runs out."""
        B.check(B.lib().sc_level_arm_wait_test(self._h))

    def set_staging(self, staging: int):
        """Staging of the one-stage kernel's raw inputs: 0 registers, 1 shared
        memory by cp.async (binding.SC_STAGING_*)."""
        B.check(B.lib().sc_level_set_staging(self._h, int(staging)))

    def get_staging(self) -> int:
        n = ctypes.c_int32()
        B.check(B.lib().sc_level_get_staging(self._h, ctypes.byref(n)))
        return n.value

    def autotune(self, seed: int = 0, budget_ms: float = 2000.0, abort_factor: float = 2.0,
                 cache_path: Optional[str] = None, stream=None):
        cp = cache_path.encode() if cache_path else None
        B.check(B.lib().sc_level_autotune(self._h, int(seed), float(budget_ms),
                                          float(abort_factor), cp, _stream(stream)))

    # ---- kernels ----------------------------------------------------------------

    def _dt(self, dt):
        a = np.atleast_1d(np.asarray(dt, dtype=np.float64))
        return (ctypes.c_double * len(a))(*a), len(a)

    def _f(self, t, name, optional=False):
        return _field(t, self.field_size, name, optional)

    def fill_ghosts(self, field, stream=None):
        B.check(B.lib().sc_level_fill_ghosts(self._h, self._f(field, "field"), _stream(stream)))

    def apply_laplacian(self, u, out, stream=None):
        B.check(B.lib().sc_level_apply_laplacian(self._h, self._f(u, "u"), self._f(out, "out"),
                                                 _stream(stream)))

    def rk4_step(self, u, pi, c2, dt, nsteps: int, mode: int = B.SC_MODE_GRAPH, stream=None):
        d, nd = self._dt(dt)
        B.check(B.lib().sc_level_rk4_step(self._h, self._f(u, "u"), self._f(pi, "pi"),
                                          self._f(c2, "c2"), d, nd, int(nsteps), int(mode),
                                          _stream(stream)))

    def rk4_step_host(self, u: np.ndarray, pi: np.ndarray, c2: np.ndarray, dt, nsteps: int,
                      u_out: Optional[np.ndarray] = None, pi_out: Optional[np.ndarray] = None,
                      stream=None):
        """End to end from host buffers (ideally pinned); returns (u, pi)."""
        n = self.field_size
        u_out = np.empty_like(u) if u_out is None else u_out
        pi_out = np.empty_like(pi) if pi_out is None else pi_out
        vp = ctypes.c_void_p
        ptrs = [vp(_host_field(a, n, name)) for a, name in
                ((u, "u"), (pi, "pi"), (c2, "c2"), (u_out, "u_out"), (pi_out, "pi_out"))]
        d, nd = self._dt(dt)
        B.check(B.lib().sc_level_rk4_step_host(self._h, *ptrs, d, nd, int(nsteps),
                                               _stream(stream)))
        return u_out, pi_out

    def misfit(self, u, u_obs, seed=None, stream=None):
        """(loss device scalar, seed) with seed = h^3 (u - u_obs)."""
        torch = _torch()
        pu, po = self._f(u, "u"), self._f(u_obs, "u_obs")
        ps = self._f(seed, "seed", optional=True)
        loss = torch.zeros(2, dtype=torch.float64, device=u.device)[:1]
        B.check(B.lib().sc_level_misfit(self._h, pu, po, _ptr(loss), ps, _stream(stream)))
        return loss[0], seed

    def forward_tape(self, u0, pi0, c2, dt, nsteps: int, ckpt_every: int, u_T=None, pi_T=None,
                     stream=None):
        d, nd = self._dt(dt)
        f = self._f
        B.check(B.lib().sc_level_forward_tape(
            self._h, f(u0, "u0"), f(pi0, "pi0"), f(c2, "c2"), d, nd, int(nsteps),
            int(ckpt_every), f(u_T, "u_T", True), f(pi_T, "pi_T", True), _stream(stream)))

    def backward_tape(self, c2, gu_T, gpi_T, g_u0, g_pi0, g_c2, stream=None):
        f = self._f
        B.check(B.lib().sc_level_backward_tape(
            self._h, f(c2, "c2"), f(gu_T, "gu_T", True), f(gpi_T, "gpi_T", True),
            f(g_u0, "g_u0"), f(g_pi0, "g_pi0"), f(g_c2, "g_c2"), _stream(stream)))

    def grad(self, u0, pi0, c2, dt, nsteps, ckpt_every, gu_T, gpi_T, g_u0, g_pi0, g_c2,
             u_T=None, pi_T=None, stream=None):
        d, nd = self._dt(dt)
        f = self._f
        B.check(B.lib().sc_level_grad(
            self._h, f(u0, "u0"), f(pi0, "pi0"), f(c2, "c2"), d, nd, int(nsteps),
            int(ckpt_every), f(gu_T, "gu_T", True), f(gpi_T, "gpi_T", True),
            f(g_u0, "g_u0"), f(g_pi0, "g_pi0"), f(g_c2, "g_c2"),
            f(u_T, "u_T", True), f(pi_T, "pi_T", True), _stream(stream)))

    def kernel_times(self):
        """(stage_ms, stage_launches, gather_ms, gather_launches) of the last
        rk4_step in SC_MODE_TIMED."""
        sm, gm = ctypes.c_double(), ctypes.c_double()
        sl, gl = ctypes.c_int64(), ctypes.c_int64()
        B.check(B.lib().sc_level_kernel_times(self._h, ctypes.byref(sm), ctypes.byref(sl),
                                              ctypes.byref(gm), ctypes.byref(gl)))
        return sm.value, sl.value, gm.value, gl.value

    def kernel_time(self, kind: int):
        """(ms, launches) of one kernel kind (binding.SC_KERNEL_*) in the
        last timed call."""
        ms, n = ctypes.c_double(), ctypes.c_int64()
        B.check(B.lib().sc_level_kernel_time(self._h, int(kind), ctypes.byref(ms),
                                             ctypes.byref(n)))
        return ms.value, n.value

    def set_profiling(self, on: bool):
        B.check(B.lib().sc_level_set_profiling(self._h, 1 if on else 0))

    def sync(self, stream=None):
        B.check(B.lib().sc_level_sync(self._h, _stream(stream)))


def wave_rk4(level: Level, u0, pi0, c2, dt, nsteps: int, ckpt_every: int = 20):
    """Differentiable RK4 evolution: returns (u_T, pi_T); gradients flow to
    u0, pi0 and c2 through the library's adjoint (checkpointed)."""
    torch = _torch()

    class WaveRK4(torch.autograd.Function):
        @staticmethod
        def forward(ctx, u0_, pi0_, c2_):
            uT = torch.empty_like(u0_)
            piT = torch.empty_like(pi0_)
            level.forward_tape(u0_, pi0_, c2_, dt, nsteps, ckpt_every, uT, piT)
            ctx.save_for_backward(c2_)
            return uT, piT

        @staticmethod
        def backward(ctx, guT, gpiT):
            (c2_,) = ctx.saved_tensors
            g_u0 = torch.empty_like(c2_)
            g_pi0 = torch.empty_like(c2_)
            g_c2 = torch.empty_like(c2_)
            guT = None if guT is None else guT.contiguous()
            gpiT = None if gpiT is None else gpiT.contiguous()
            level.backward_tape(c2_, guT, gpiT, g_u0, g_pi0, g_c2)
            return g_u0, g_pi0, g_c2

    return WaveRK4.apply(u0, pi0, c2)


class Hierarchy:
    """Two-level refinement hierarchy over a coarse periodic level and a fine
    level of half the spacing (see include/sc_hierarchy.h)."""

    def __init__(self, coarse: Level, fine: Level, ratio: int = 2, buffer: int = 4):
        h = ctypes.c_void_p()
        B.check(B.lib().sc_hierarchy_create(coarse.handle, fine.handle, int(ratio), int(buffer),
                                            ctypes.byref(h)))
        self._h = h
        self.coarse, self.fine, self.buffer = coarse, fine, int(buffer)

    def close(self):
        if getattr(self, "_h", None):
            B.lib().sc_hierarchy_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def counts(self):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        B.check(B.lib().sc_hierarchy_counts(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def _points(self, fn) -> np.ndarray:
        n = ctypes.c_int64()
        B.check(fn(self._h, None, 0, ctypes.byref(n)))
        out = np.zeros((max(n.value, 1), 3), dtype=np.int64)
        B.check(fn(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), n.value,
                   ctypes.byref(n)))
        return out[:n.value]

    def prolongation_points(self) -> np.ndarray:
        """Fine (x, y, z) points that prolongation fills."""
        return self._points(B.lib().sc_hierarchy_prolongation_points)

    def restriction_points(self) -> np.ndarray:
        """Coarse (x, y, z) points that restriction sets."""
        return self._points(B.lib().sc_hierarchy_restriction_points)

    def _c(self, t, name):
        return _field(t, self.coarse.field_size, name)

    def _fn(self, t, name):
        return _field(t, self.fine.field_size, name)

    def prolongate(self, u0, u1, p0, p1, alpha: float, fu, fpi, stream=None):
        c, f = self._c, self._fn
        B.check(B.lib().sc_hierarchy_prolongate(self._h, c(u0, "u0"), c(u1, "u1"), c(p0, "p0"),
                                                c(p1, "p1"), float(alpha), f(fu, "fu"),
                                                f(fpi, "fpi"), _stream(stream)))

    def restrict(self, fu, fpi, cu, cpi, stream=None):
        c, f = self._c, self._fn
        B.check(B.lib().sc_hierarchy_restrict(self._h, f(fu, "fu"), f(fpi, "fpi"), c(cu, "cu"),
                                              c(cpi, "cpi"), _stream(stream)))

    def step(self, cu, cpi, cc2, fu, fpi, fc2, dt: float, nsteps: int,
             mode: int = B.SC_MODE_GRAPH, stream=None):
        c, f = self._c, self._fn
        B.check(B.lib().sc_hierarchy_step(self._h, c(cu, "cu"), c(cpi, "cpi"), c(cc2, "cc2"),
                                          f(fu, "fu"), f(fpi, "fpi"), f(fc2, "fc2"), float(dt),
                                          int(nsteps), int(mode), _stream(stream)))
