"""Helpers for the GPU tests: run a sweep through the C ABI on host arrays' device copies."""
import numpy as np

import paper_1510_04995_gb300 as girih


def to_dev(a, dtype):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.to(device="cuda", dtype=torch.float64 if dtype == "f64" else torch.float32).contiguous()


def gpu_sweep(stencil, dtype, u, up, co, c, T, nx, ny, nz, cfg, ldx=0):
    """Return (u, u_prev) after T steps on the GPU, as float64 numpy arrays."""
    import torch
    p = girih.plan(stencil, nx, ny, nz, dtype=dtype, T=T, ldx=ldx)
    du, dup = to_dev(u, dtype), to_dev(up, dtype)
    dco = to_dev(co, dtype) if co is not None else None
    girih.run(p, du, dup, dco, c=c, cfg=cfg)
    girih.status(p)  # no bounded device wait ran out
    torch.cuda.synchronize()
    return du.double().cpu().numpy(), dup.double().cpu().numpy()


def normwise(g, o, R):
    """max |g - o| / max |o| over the interior (the FP64 contract)."""
    sl = (slice(R, -R),) * 2
    gi, oi = g[R:-R, R:-R, R:-R], o[R:-R, R:-R, R:-R]
    gi = gi[:, :, :oi.shape[2]]
    return float(np.max(np.abs(gi - oi)) / np.max(np.abs(oi)))


def rel_l2(g, o, R):
    gi, oi = g[R:-R, R:-R, R:-R], o[R:-R, R:-R, R:-R]
    return float(np.linalg.norm((gi - oi).ravel()) / np.linalg.norm(oi.ravel()))


def feasible_cfg(stencil, dtype, nx, ny, nz, kw, ldx=0):
    """The MWD config kw, or the nearest feasible one on this device: double the cluster (narrower
    slabs, less shared memory per block), then wavefront width 1, then other block sizes."""
    p = girih.plan(stencil, nx, ny, nz, dtype=dtype, T=1, ldx=ldx)
    tries = []
    for cl in (kw["cluster"], 2 * kw["cluster"], 4 * kw["cluster"], 8 * kw["cluster"]):
        for nf in (kw["nf"], 1):
            for th in (kw["threads"], 288, 544, 256, 512, 1024):
                if cl <= 16:
                    tries.append(dict(kw, cluster=cl, nf=nf, threads=th))
    for t in tries:
        c = girih.config(girih.MWD, **t)
        if p.feasible(c):
            return c
    raise AssertionError(f"no feasible configuration near {kw}")
