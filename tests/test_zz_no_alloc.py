"""The RK4 entry point that allocates no device memory.

Callers that cannot call cudaMalloc (their own allocator owns the device, or
allocation is forbidden after start-up) use sc_box_rk4_step_noalloc, whose
stage arrays live in a static device array inside the library.  This test
calls it through the C ABI and checks it against sc_level_rk4_step (FP64
form) on the same one-box periodic level and against the CPU oracle, for two
calls in a row: the second call reuses the static array the first call left
behind.  Odd and tiny boxes (extents 2 and 3, whose ghosts wrap around the
box more than once, and an odd x extent whose last point is stored alone)
are checked against the oracle.  It is collected last so that a failure here
cannot hide failures elsewhere."""
import ctypes

import numpy as np
import pytest

from paper_1308_1343_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1308_1343_gb300 import build
    build.build()


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _box_ptr(lev, t):
    """Address of the first element of the one box's padded array in t."""
    off, _, (_, py, pz) = lev.layout[0]
    return ctypes.c_void_p(t.data_ptr() + 8 * (off - 2 - 2 * py - 2 * pz))


def test_noalloc_matches_level_step_two_calls(orc):
    import torch
    from paper_1308_1343_gb300 import binding as B
    lib = B.lib()
    for n, seed in (((40, 36, 28), 2), ((24, 20, 31), 7)):
        from paper_1308_1343_gb300.level import Level
        inst = W.bumpy_instance(W.Domain(n, 1.0 / n[1]), seed)
        lev = Level.from_instances([inst])
        lev.set_arith(B.SC_ARITH_FP64)
        lev.set_fusion(1)
        u = lev.to_device([inst.u])
        pi = lev.to_device([inst.pi])
        c2 = lev.to_device([inst.c2], fill=1.0)
        u2, pi2 = u.clone(), pi.clone()
        stream = torch.cuda.current_stream().cuda_stream
        for call in range(2):
            lev.rk4_step(u, pi, c2, inst.dt, 3, B.SC_MODE_GRAPH)
            B.check(lib.sc_box_rk4_step_noalloc(_box_ptr(lev, u2), _box_ptr(lev, pi2),
                                                _box_ptr(lev, c2), n[0], n[1], n[2],
                                                inst.dom.h, inst.dt, 3, stream))
            lev.sync()
            torch.cuda.synchronize()
            a, b = lev.gather(u2)[0], lev.gather(u)[0]
            assert _rel(a, b) <= TOL, (n, call)
            assert _rel(lev.gather(pi2)[0], lev.gather(pi)[0]) <= TOL, (n, call)
            ou, op = orc.rk4_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt,
                                      3 * (call + 1))
            assert _rel(a, ou) <= TOL, (n, call)
            assert _rel(lev.gather(pi2)[0], op) <= TOL, (n, call)
        lev.close()


@pytest.mark.parametrize("n", [(3, 2, 5), (2, 3, 2), (17, 9, 6), (2, 2, 2), (33, 3, 4)])
def test_noalloc_odd_and_tiny_boxes_vs_oracle(orc, n):
    """Extents 2 and 3 (each ghost layer wraps onto the box more than once)
    and odd x extents (the last point of a row is stored alone), two calls
    in a row, against the oracle's periodic RK4."""
    import torch
    from paper_1308_1343_gb300 import binding as B
    from paper_1308_1343_gb300.level import Level
    lib = B.lib()
    inst = W.bumpy_instance(W.Domain(n, 1.0 / max(n)), 11)
    lev = Level.from_instances([inst])
    u = lev.to_device([inst.u])
    pi = lev.to_device([inst.pi])
    c2 = lev.to_device([inst.c2], fill=1.0)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        B.check(lib.sc_box_rk4_step_noalloc(_box_ptr(lev, u), _box_ptr(lev, pi),
                                            _box_ptr(lev, c2), n[0], n[1], n[2], inst.dom.h,
                                            inst.dt, 2, stream))
        torch.cuda.synchronize()
        ou, op = orc.rk4_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, 2 * (call + 1))
        assert _rel(lev.gather(u)[0], ou) <= TOL, (n, call)
        assert _rel(lev.gather(pi)[0], op) <= TOL, (n, call)
    lev.close()


def test_noalloc_zero_steps_leaves_the_state():
    import torch
    from paper_1308_1343_gb300 import binding as B
    from paper_1308_1343_gb300.level import Level
    lib = B.lib()
    n = (20, 18, 10)
    inst = W.bumpy_instance(W.Domain(n, 1.0 / 18), 5)
    lev = Level.from_instances([inst])
    u = lev.to_device([inst.u])
    pi = lev.to_device([inst.pi])
    c2 = lev.to_device([inst.c2], fill=1.0)
    u0, p0 = u.clone(), pi.clone()
    B.check(lib.sc_box_rk4_step_noalloc(_box_ptr(lev, u), _box_ptr(lev, pi), _box_ptr(lev, c2),
                                        n[0], n[1], n[2], inst.dom.h, inst.dt, 0,
                                        torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert torch.equal(u, u0) and torch.equal(pi, p0)
    lev.close()


def test_noalloc_rejects_too_large_box():
    import torch
    from paper_1308_1343_gb300 import binding as B
    lib = B.lib()
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    rc = lib.sc_box_rk4_step_noalloc(p, p, p, 96, 96, 96, 0.01, 0.0025, 1, None)
    assert rc == B.SC_EINVAL
    assert b"too large" in lib.sc_last_error()
