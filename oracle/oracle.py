"""Oracle: plain CPU FP64 reference for the stencil / RK4 level path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import this module.  It shares no code
with the CUDA library in ``paper_1308_1343_gb300`` and never imports it.

The arithmetic lives in ``oracle.c`` (compiled here with
``-O2 -ffp-contract=off``); this file only marshals numpy arrays.  Arrays are
float64, C-contiguous, shape ``(nz, ny, nx)`` (x fastest) for whole periodic
domains, or ``(nz+4, ny+4, nx+4)`` for one padded box with ghost width 2.

What each function follows:

* ``lap_periodic`` / ``lap_padded`` -- the 4th-order centred second
  difference summed over the axes, the centred-difference idiom on padded
  arrays of the paper's Sec. 4.3 ("Iterators").
* ``rk4_periodic`` -- classic RK4 stage form for y' = A y,
  A(u, pi) = (pi, c2 * L u); ``rk4_padded`` -- the same step on one padded
  box whose ghosts hold boundary values.
* ``tlm_periodic`` / ``adj_step_periodic`` / ``grad_periodic`` -- the
  tangent-linear and adjoint of that step and the checkpointed reverse sweep.
* ``fill_ghosts`` / ``ghost_owners`` -- the ghost exchange of a level of
  boxes (paper Sec. 2: the communication schedule derived from bboxsets),
  by brute-force search for each ghost point's owner.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64 = ctypes.c_int64
_dp = ctypes.POINTER(ctypes.c_double)
_lp = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, OpenMP)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _configure(lib):
    """Declare the C signatures on a loaded oracle library."""
    lib.oracle_set_threads.argtypes = [ctypes.c_int]
    lib.oracle_set_threads.restype = ctypes.c_int
    lib.oracle_has_openmp.restype = ctypes.c_int
    lib.oracle_lap_periodic.argtypes = [_dp, _dp, _i64, _i64, _i64, ctypes.c_double]
    lib.oracle_lap_padded.argtypes = [_dp, _dp, _i64, _i64, _i64, ctypes.c_double]
    lib.oracle_rk4_periodic.argtypes = [_dp, _dp, _dp, _i64, _i64, _i64,
                                        ctypes.c_double, ctypes.c_double, _i64]
    lib.oracle_rk4_periodic.restype = ctypes.c_int
    lib.oracle_rk4_padded.argtypes = [_dp, _dp, _dp, _i64, _i64, _i64, ctypes.c_double,
                                      ctypes.c_double]
    lib.oracle_rk4_padded.restype = ctypes.c_int
    lib.oracle_energy_periodic.argtypes = [_dp, _dp, _dp, _i64, _i64, _i64,
                                           ctypes.c_double]
    lib.oracle_energy_periodic.restype = ctypes.c_double
    lib.oracle_tlm_periodic.argtypes = [_dp, _dp, _dp, _dp, _dp, _dp, _i64, _i64,
                                        _i64, ctypes.c_double, ctypes.c_double, _i64]
    lib.oracle_tlm_periodic.restype = ctypes.c_int
    lib.oracle_adj_step_periodic.argtypes = [_dp, _dp, _dp, _dp, _dp, _dp, _i64,
                                             _i64, _i64, ctypes.c_double,
                                             ctypes.c_double]
    lib.oracle_adj_step_periodic.restype = ctypes.c_int
    lib.oracle_grad_periodic.argtypes = [_dp, _dp, _dp, _i64, _i64, _i64,
                                         ctypes.c_double, ctypes.c_double, _i64, _i64,
                                         _dp, _dp, _dp, _dp, _dp]
    lib.oracle_grad_periodic.restype = ctypes.c_int
    lib.oracle_fill_ghosts.argtypes = [ctypes.c_int, _lp, _lp, ctypes.c_int,
                                       ctypes.POINTER(_dp)]
    lib.oracle_fill_ghosts.restype = ctypes.c_int
    lib.oracle_ghost_owners.argtypes = [ctypes.c_int, _lp, _lp, ctypes.c_int, _lp,
                                        _i64]
    lib.oracle_ghost_owners.restype = _i64
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
    return _lib


def compile_variant(src_text: str, path: str) -> str:
    """Compile a modified copy of oracle.c (tests that plant a mistake in
    the oracle use this to show that the pins catch it)."""
    src = path + ".c"
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", path, src,
                    "-lm"], check=True)
    return path


@contextlib.contextmanager
def using_library(path: str):
    """Route this module's calls to another build of the oracle for the
    duration of the block (planted-mistake tests only)."""
    global _lib
    _load()
    with _lock:
        saved = _lib
        _lib = _configure(ctypes.CDLL(path))
    try:
        yield
    finally:
        with _lock:
            _lib = saved


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int) -> int:
    """OpenMP threads for the oracle's loops; returns the number in effect."""
    return _load().oracle_set_threads(int(n))


def has_openmp() -> bool:
    return bool(_load().oracle_has_openmp())


def lap_periodic(u, h: float) -> np.ndarray:
    """L u on a whole periodic domain; u has shape (nz, ny, nx)."""
    u = _f64(u)
    out = np.empty_like(u)
    nz, ny, nx = u.shape
    _load().oracle_lap_periodic(_d(u), _d(out), nx, ny, nz, float(h))
    return out


def lap_padded(up, h: float) -> np.ndarray:
    """L u on one padded box (ghost width 2); returns the interior values."""
    up = _f64(up)
    nz, ny, nx = (s - 4 for s in up.shape)
    out = np.empty((nz, ny, nx))
    _load().oracle_lap_padded(_d(up), _d(out), nx, ny, nz, float(h))
    return out


def rk4_periodic(u, pi, c2, h: float, dt: float, nsteps: int):
    """nsteps classic RK4 steps on a periodic domain; returns new (u, pi)."""
    u = _f64(u).copy()
    pi = _f64(pi).copy()
    c2 = _f64(c2)
    nz, ny, nx = u.shape
    rc = _load().oracle_rk4_periodic(_d(u), _d(pi), _d(c2), nx, ny, nz, float(h),
                                     float(dt), int(nsteps))
    if rc:
        raise MemoryError("oracle_rk4_periodic: allocation failed")
    return u, pi


def rk4_padded(up, pip, c2p, h: float, dt: float):
    """One classic RK4 step on one padded box (ghost width 2) whose ghosts
    hold boundary values, held fixed over the step; returns new padded
    (u, pi) with the ghosts unchanged."""
    up = _f64(up).copy()
    pip = _f64(pip).copy()
    c2p = _f64(c2p)
    nz, ny, nx = (s - 4 for s in up.shape)
    rc = _load().oracle_rk4_padded(_d(up), _d(pip), _d(c2p), nx, ny, nz, float(h), float(dt))
    if rc:
        raise MemoryError("oracle_rk4_padded: allocation failed")
    return up, pip


def energy(u, pi, c2, h: float) -> float:
    """E = 1/2 sum(pi^2/c2 - u L u) h^3 on a periodic domain."""
    u, pi, c2 = _f64(u), _f64(pi), _f64(c2)
    nz, ny, nx = u.shape
    return _load().oracle_energy_periodic(_d(u), _d(pi), _d(c2), nx, ny, nz, float(h))


def tlm_periodic(u, pi, c2, du, dpi, dc2, h: float, dt: float, nsteps: int):
    """Returns (u_T, pi_T, du_T, dpi_T): state and its tangent along
    (du, dpi, dc2) after nsteps RK4 steps."""
    u, pi, du, dpi = (_f64(a).copy() for a in (u, pi, du, dpi))
    c2, dc2 = _f64(c2), _f64(dc2)
    nz, ny, nx = u.shape
    rc = _load().oracle_tlm_periodic(_d(u), _d(pi), _d(c2), _d(du), _d(dpi), _d(dc2),
                                     nx, ny, nz, float(h), float(dt), int(nsteps))
    if rc:
        raise MemoryError("oracle_tlm_periodic: allocation failed")
    return u, pi, du, dpi


def adj_step_periodic(u, pi, c2, bu, bpi, bc2, h: float, dt: float):
    """One reverse RK4 step at input state (u, pi): returns (bu, bpi, bc2)
    with bu, bpi the adjoint of the step input and bc2 accumulated."""
    u, pi, c2 = _f64(u), _f64(pi), _f64(c2)
    bu, bpi, bc2 = (_f64(a).copy() for a in (bu, bpi, bc2))
    nz, ny, nx = u.shape
    rc = _load().oracle_adj_step_periodic(_d(u), _d(pi), _d(c2), _d(bu), _d(bpi), _d(bc2),
                                          nx, ny, nz, float(h), float(dt))
    if rc:
        raise MemoryError("oracle_adj_step_periodic: allocation failed")
    return bu, bpi, bc2


def grad_periodic(u0, pi0, c2, h: float, dt: float, nsteps: int, ckpt_every: int,
                  gu_T, gpi_T):
    """Checkpointed reverse sweep: returns (g_u0, g_pi0, g_c2) given the
    adjoint seeds (gu_T, gpi_T) of the final state."""
    u0, pi0, c2, gu_T, gpi_T = (_f64(a) for a in (u0, pi0, c2, gu_T, gpi_T))
    g_u0, g_pi0, g_c2 = (np.empty_like(u0) for _ in range(3))
    nz, ny, nx = u0.shape
    rc = _load().oracle_grad_periodic(_d(u0), _d(pi0), _d(c2), nx, ny, nz, float(h),
                                      float(dt), int(nsteps), int(ckpt_every), _d(gu_T),
                                      _d(gpi_T), _d(g_u0), _d(g_pi0), _d(g_c2))
    if rc:
        raise MemoryError("oracle_grad_periodic: allocation failed")
    return g_u0, g_pi0, g_c2


def misfit_loss(u_T, u_obs, h: float) -> float:
    """L = 1/2 sum (u_T - u_obs)^2 h^3."""
    d = _f64(u_T) - _f64(u_obs)
    return 0.5 * float(np.sum(d * d)) * h ** 3


def misfit_seed(u_T, u_obs, h: float) -> np.ndarray:
    """dL/du_T = h^3 (u_T - u_obs)."""
    return (_f64(u_T) - _f64(u_obs)) * h ** 3


def _boxes_arr(boxes) -> np.ndarray:
    b = np.ascontiguousarray(np.asarray(boxes, dtype=np.int64).reshape(-1, 6))
    return b


def fill_ghosts(boxes, dom, periodic: int, fields) -> None:
    """Fill, in place, the star ghosts of every box of one domain.

    boxes: (nb, 6) int (lo xyz, hi xyz); dom: (6,) int; periodic: bit mask
    x=1, y=2, z=4; fields: list of dense padded float64 arrays, one per box.
    """
    b = _boxes_arr(boxes)
    d = np.ascontiguousarray(np.asarray(dom, dtype=np.int64).reshape(6))
    for f, B in zip(fields, b):
        assert f.shape == (B[5] - B[2] + 4, B[4] - B[1] + 4, B[3] - B[0] + 4)
        assert f.dtype == np.float64 and f.flags.c_contiguous
    ptrs = (_dp * len(fields))(*[_d(f) for f in fields])
    rc = _load().oracle_fill_ghosts(len(b), b.ctypes.data_as(_lp), d.ctypes.data_as(_lp),
                                    int(periodic), ptrs)
    if rc:
        raise ValueError("oracle_fill_ghosts: boxes overlap")


def ghost_owners(boxes, dom, periodic: int) -> np.ndarray:
    """(n, 8) int64 rows (dst_box, px, py, pz, src_box, qx, qy, qz)."""
    b = _boxes_arr(boxes)
    d = np.ascontiguousarray(np.asarray(dom, dtype=np.int64).reshape(6))
    lib = _load()
    n = lib.oracle_ghost_owners(len(b), b.ctypes.data_as(_lp), d.ctypes.data_as(_lp),
                                int(periodic), None, 0)
    if n < 0:
        raise ValueError("oracle_ghost_owners: boxes overlap")
    out = np.empty((max(n, 1), 8), dtype=np.int64)
    n2 = lib.oracle_ghost_owners(len(b), b.ctypes.data_as(_lp), d.ctypes.data_as(_lp),
                                 int(periodic), out.ctypes.data_as(_lp), n)
    assert n2 == n
    return out[:n]
