"""GPU cases whose traversal index arithmetic is the most involved: ragged
tiles, thin and odd boxes, self-periodic boxes with wrapped ghosts, uneven
multi-box levels, ensembles, both forms and stagings, the adjoint and the
two-level hierarchy.  `run()` evolves each one through whichever library the
binding loaded and returns a digest of its results; the checked build
(`SC_BOUNDS_CHECK`) must give the release build's digests and report no
failed check.  Holds no arithmetic of the method.

Run as a script, it prints the digests as one JSON object."""
import hashlib
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def _digest(arrays):
    h = hashlib.sha1()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def _evolve(insts, nsteps, fuse, mode=0, arith=1, staging=None):
    from paper_1308_1343_gb300.level import Level
    lev = Level.from_instances(insts)
    lev.set_arith(arith)
    lev.set_fusion(fuse)
    if staging is not None:
        lev.set_staging(staging)
    u = lev.to_device([i.u for i in insts])
    pi = lev.to_device([i.pi for i in insts])
    c2 = lev.to_device([i.c2 for i in insts], fill=1.0)
    dts = [i.dt for i in insts]
    lev.rk4_step(u, pi, c2, dts if len(set(dts)) > 1 else dts[0], nsteps, mode)
    lev.sync()
    return lev.gather(u) + lev.gather(pi)


def _gradient(inst, nsteps, every):
    import torch
    from paper_1308_1343_gb300.level import Level
    lev = Level.from_instances([inst])
    lev.set_arith(1)
    lev.set_fusion(2)
    u0, pi0 = lev.to_device([inst.u]), lev.to_device([inst.pi])
    c2 = lev.to_device([inst.c2], fill=1.0)
    uT, seed = torch.empty_like(u0), torch.empty_like(u0)
    g = [torch.empty_like(u0) for _ in range(3)]
    lev.forward_tape(u0, pi0, c2, inst.dt, nsteps, every, uT, None)
    lev.misfit(uT, u0, seed)
    lev.backward_tape(c2, seed, None, g[0], g[1], g[2])
    lev.sync()
    return [x for t in g for x in lev.gather(t)]


def _laplacian(inst):
    import torch
    from paper_1308_1343_gb300.level import Level
    lev = Level.from_instances([inst])
    lev.set_arith(1)
    u = lev.to_device([inst.u])
    out = torch.zeros_like(u)
    lev.fill_ghosts(u)
    lev.apply_laplacian(u, out)
    lev.sync()
    return lev.gather(out)


def _hierarchy():
    import torch
    from paper_1308_1343_gb300 import workloads as W
    from paper_1308_1343_gb300.level import Hierarchy, Level
    n, lo, hi = 24, (8, 6, 10), (38, 36, 36)
    coarse, (fu_h, fp_h, fc_h) = W.refined_fields(n, 7, lo, hi)
    c = Level.from_instances([coarse])
    f = Level([(lo, ((lo[0] + hi[0]) // 2, hi[1], hi[2]), 0),
               (((lo[0] + hi[0]) // 2, lo[1], lo[2]), hi, 0)],
              [dict(lo=lo, hi=hi, h=0.5 / n, periodic=0)])
    for lev in (c, f):
        lev.set_arith(1)
        lev.set_fusion(2)
    h = Hierarchy(c, f, buffer=4)
    cu, cpi = c.to_device([coarse.u]), c.to_device([coarse.pi])
    cc2 = c.to_device([coarse.c2], fill=1.0)
    fu, fpi = f.to_device([fu_h]), f.to_device([fp_h])
    fc2 = f.to_device([fc_h], fill=1.0)
    h.step(cu, cpi, cc2, fu, fpi, fc2, coarse.dt, 2)
    c.sync()
    f.sync()
    torch.cuda.synchronize()
    return c.gather(cu) + c.gather(cpi) + f.gather(fu) + f.gather(fpi)


def run():
    from paper_1308_1343_gb300 import workloads as W
    out = {}
    ragged = W.bumpy_instance(W.Domain((40, 36, 28), 1.0 / 36), 2)
    for fuse in (1, 2):
        for mode in (0, 1):
            out["ragged f%d m%d" % (fuse, mode)] = _digest(_evolve([ragged], 4, fuse, mode))
    out["ragged fp64"] = _digest(_evolve([ragged], 3, 2, arith=0))
    out["ragged shared staging"] = _digest(_evolve([ragged], 3, 1, staging=1))
    uneven = W.uneven_level(n=(128, 128, 64), h=1.0 / 64, levels=6, seed=3, box_seed=30)
    for fuse in (1, 2):
        out["uneven f%d" % fuse] = _digest(_evolve([uneven], 3, fuse))
    thin = W.bumpy_instance(W.Domain((13, 11, 9), 1.0 / 11), 7)
    thin.boxes = [((0, 0, 0), (2, 11, 9)), ((2, 0, 0), (5, 11, 9)), ((5, 0, 0), (13, 4, 9)),
                  ((5, 4, 0), (13, 11, 2)), ((5, 4, 2), (13, 11, 9))]
    for fuse in (1, 2):
        out["thin f%d" % fuse] = _digest(_evolve([thin], 3, fuse))
    for n in ((2, 3, 5), (6, 7, 2), (12, 10, 3), (5, 6, 4)):
        inst = W.bumpy_instance(W.Domain(n, 1.0 / 8), 11)
        for fuse in (1, 2):
            out["self-periodic %s f%d" % (n, fuse)] = _digest(_evolve([inst], 2, fuse))
    ens = W.ensemble(count=3)
    out["ensemble"] = _digest(_evolve(ens, 3, 2))
    out["laplacian ragged"] = _digest(_laplacian(ragged))
    small_uneven = W.uneven_level(n=(64, 64, 32), h=1.0 / 32, levels=3, seed=3, box_seed=30)
    out["gradient uneven"] = _digest(_gradient(small_uneven, 4, 2))
    out["gradient box"] = _digest(_gradient(W.gradient_problem(24, 4), 4, 2))
    out["hierarchy"] = _digest(_hierarchy())
    return out


if __name__ == "__main__":
    print(json.dumps(run()), flush=True)
