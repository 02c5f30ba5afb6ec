"""Shared helpers of the GPU parity tests (no arithmetic of the method)."""
import numpy as np


def rel_err(got, want) -> float:
    """||got - want||_inf / ||want||_inf over the given (interior) values."""
    got = np.asarray(got)
    want = np.asarray(want)
    den = np.abs(want).max()
    return float(np.abs(got - want).max() / (den if den > 0 else 1.0))


def make_level(instances):
    from paper_1308_1343_gb300.level import Level
    return Level.from_instances(instances)


def upload(lev, arrays, fill=0.0):
    return lev.to_device(list(arrays), fill=fill)


def run_gpu(instances, nsteps, arith, mode, lev=None, fuse=1):
    """Evolve every instance on the GPU; returns (lev, [u], [pi]).  A new
    level runs `fuse` RK4 stages per stencil pass; a given one keeps its
    setting."""
    import torch
    if lev is None:
        lev = make_level(instances)
        lev.set_fusion(fuse)
    lev.set_arith(arith)
    u = upload(lev, [i.u for i in instances])
    pi = upload(lev, [i.pi for i in instances])
    c2 = upload(lev, [i.c2 for i in instances], fill=1.0)
    dts = [i.dt for i in instances]
    lev.rk4_step(u, pi, c2, dts if len(set(dts)) > 1 else dts[0], nsteps, mode)
    lev.sync()
    torch.cuda.synchronize()
    return lev, lev.gather(u), lev.gather(pi)
