"""Full-size checks in the benchmark's launch configuration.

* Blocked == naive bit for bit on every benchmark workload (full grids, full T).
* Sampled outputs against the FP64 oracle: the value of a point after T steps depends only on
  initial values within distance R*T along each axis, so the oracle run on the (2RT+1)^3 block
  around a sample (clipped by the real halo at the domain faces) reproduces that point exactly;
  the block's own artificial boundary cannot reach the centre within T steps.
"""
import json
import os

import numpy as np
import pytest

import oracle
import paper_1510_04995_gb300 as girih
from paper_1510_04995_gb300 import inputs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__
    __graft_entry__.build()


def _blocked_cfg(workload, p):
    """The blocked configuration the benchmark reports for this workload (the tuner's fastest
    blocked candidate), else the plan's default blocked configuration."""
    import bench
    best, blocked = bench._tuned(workload)
    for c in (blocked, best):
        if c and c["algo"] == girih.MWD and p.feasible(girih.Config(**c)):
            return girih.Config(**c)
    return p.config


def _run_pair(workload):
    import torch
    import bench
    stencil, dtype, nx, ny, nz, T = bench.WORKLOADS[workload]
    R = inputs.RADIUS[stencil]
    a16 = 16 // (8 if dtype == "f64" else 4)
    ldx = -(-(nx + 2 * R) // a16) * a16  # the benchmark's 16-byte aligned leading dimension
    p = girih.plan(stencil, nx, ny, nz, dtype=dtype, T=T, ldx=ldx)
    cfg = _blocked_cfg(workload, p)
    assert cfg.algo == girih.MWD
    u, up, co, c = inputs.make_problem(stencil, nx, ny, nz, backend="torch", device="cuda", ldx=ldx)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    u, up = u.to(tdt).contiguous(), up.to(tdt).contiguous()
    co = co.to(tdt).contiguous() if co is not None else None
    bu, bup = u.clone(), up.clone()
    girih.run(p, bu, bup, co, c=c, cfg=cfg)
    girih.run(p, u, up, co, c=c, cfg=girih.config(girih.NAIVE))
    torch.cuda.synchronize()
    return p, cfg, (bu, bup), (u, up), (stencil, dtype, nx, ny, nz, T)


@pytest.mark.parametrize("workload", ["7pt_const_f64_512", "7pt_const_f32_512", "7pt_var_f32_480",
                                      "25pt_const_f32_384", "25pt_var_f32_384", "25pt_const_f64_384",
                                      "25pt_cgrid_f32_384", "27pt_box_f32_512", "7pt_rbgs_f32_512"])
def test_blocked_equals_naive_full_size(workload):
    import torch
    p, cfg, (bu, bup), (nu, nup), _ = _run_pair(workload)
    assert torch.equal(bu, nu) and torch.equal(bup, nup), (workload, cfg)


@pytest.mark.parametrize("workload", ["7pt_const_f64_512", "25pt_cgrid_f64_384", "27pt_box_f64_512",
                                      "7pt_rbgs_f64_512"])
def test_sampled_points_against_oracle_cones(workload):
    import torch
    p, cfg, (bu, _), _, (stencil, dtype, nx, ny, nz, T) = _run_pair(workload)
    R = inputs.RADIUS[stencil]
    h = R * T
    u0, _, co, c = inputs.make_problem(stencil, nx, ny, nz)
    scale = float(bu.abs().max())
    samples = [(0, 0, 0), (nx - 1, ny // 2, nz - 1), (nx // 2, ny // 2, nz // 2), (nx // 3, ny - 1, 5)]
    for (i, j, k) in samples:
        lo = [max(q - h, 0) for q in (i, j, k)]
        hi = [min(q + h + 1, n) for q, n in zip((i, j, k), (nx, ny, nz))]
        if stencil == 6 and sum(lo) % 2:
            # red-black colours are fixed by the coordinate parity: start the sub-block on an
            # even corner (one more column, row or plane still holds the whole cone)
            ax = next(a for a in range(3) if lo[a] > 0)
            lo[ax] -= 1
        sub = np.ascontiguousarray(u0[lo[2]:hi[2] + 2 * R, lo[1]:hi[1] + 2 * R, lo[0]:hi[0] + 2 * R])
        sup = sub.copy()
        sco = None if co is None else np.ascontiguousarray(
            co[:, lo[2]:hi[2] + 2 * R, lo[1]:hi[1] + 2 * R, lo[0]:hi[0] + 2 * R])
        oracle.sweep(stencil, sub, sup, sco, c, T, hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2], nthreads=16)
        ref = sub[k - lo[2] + R, j - lo[1] + R, i - lo[0] + R]
        got = float(bu[k + R, j + R, i + R])
        assert abs(got - ref) <= 1e-12 * scale, ((i, j, k), got, ref)


@pytest.mark.parametrize("variant", ["NAIVE", "FED", "FED_BULK", "FED_ELEM", "RELAXED", "FED_PERSISTENT",
                                     "RELAXED_PERSISTENT", "OVERLAP_PERSISTENT"])
def test_blocked_repeatable_under_load(variant):
    """Repeated large sweeps in each data path, bit for bit against one naive sweep: a staging or
    synchronisation race shows up as a rare, localised difference, so several long runs with many
    concurrent tiles (grids larger than L2) are compared."""
    import torch
    stencil, dtype, nx, ny, nz, T = 0, "f32", 512, 512, 256, 32
    ldx = 516
    p = girih.plan(stencil, nx, ny, nz, dtype=dtype, T=T, ldx=ldx)
    cfg = (girih.config(girih.NAIVE) if variant == "NAIVE" else
           girih.config(girih.MWD, dw=8, nf=1, cluster=8, threads=352 if variant.endswith("_PERSISTENT") and
                        variant != "FED_PERSISTENT" else 512, variant=getattr(girih, variant)))
    u, up, co, c = inputs.make_problem(stencil, nx, ny, nz, backend="torch", device="cuda", ldx=ldx)
    u, up = u.float().contiguous(), up.float().contiguous()
    nu, nup = u.clone(), up.clone()
    girih.run(p, nu, nup, None, c=c, cfg=girih.config(girih.NAIVE))
    for _ in range(4):
        bu, bup = u.clone(), up.clone()
        girih.run(p, bu, bup, None, c=c, cfg=cfg)
        girih.status(p)
        torch.cuda.synchronize()
        assert torch.equal(bu, nu) and torch.equal(bup, nup), (variant, int((bu != nu).sum()))


@pytest.mark.parametrize("workload,cfgkw", [
    ("7pt_const_f32_512", dict(dw=8, nf=1, cluster=8, threads=352, variant=6)),
    ("7pt_const_f64_512", dict(dw=8, nf=1, cluster=16, threads=352, variant=6)),
    ("7pt_var_f32_480", dict(dw=8, nf=1, cluster=8, threads=320, variant=6)),
    ("7pt_rbgs_f32_512", dict(dw=12, nf=1, cluster=16, threads=416, variant=6)),
    ("7pt_const_f32_512", dict(dw=8, nf=1, cluster=8, threads=352, variant=7)),
    ("7pt_const_f64_512", dict(dw=4, nf=1, cluster=8, threads=192, variant=7)),
    ("7pt_var_f32_480", dict(dw=6, nf=1, cluster=8, threads=192, variant=7)),
    ("7pt_rbgs_f32_512", dict(dw=12, nf=1, cluster=16, threads=480, variant=7)),
    # tiles split along z into segments
    ("7pt_var_f32_480", dict(dw=6, nf=1, cluster=8, threads=224, variant=7, zseg=64)),
    ("7pt_const_f64_512", dict(dw=4, nf=1, cluster=4, threads=352, variant=7, zseg=32)),
    ("7pt_rbgs_f32_512", dict(dw=8, nf=1, cluster=4, threads=640, variant=7, zseg=128)),
    ("25pt_const_f32_384", dict(dw=16, nf=1, cluster=16, threads=352, variant=7, zseg=48)),
])
def test_persistent_tma_kernels_full_size(workload, cfgkw):
    """The warp-specialised persistent kernels (RELAXED_PERSISTENT = 6, OVERLAP_PERSISTENT = 7,
    also with its tiles split along z) on the benchmark grids (full T), in cluster and diamond
    shapes that hold one or two blocks per SM: bit for bit the naive sweep."""
    import torch
    import bench
    stencil, dtype, nx, ny, nz, T = bench.WORKLOADS[workload]
    a16 = 16 // (8 if dtype == "f64" else 4)
    ldx = -(-(nx + 2 * inputs.RADIUS[stencil]) // a16) * a16
    p = girih.plan(stencil, nx, ny, nz, dtype=dtype, T=T, ldx=ldx)
    cfg = girih.config(girih.MWD, **cfgkw)
    assert p.feasible(cfg), cfg
    u, up, co, c = inputs.make_problem(stencil, nx, ny, nz, backend="torch", device="cuda", ldx=ldx)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    u, up = u.to(tdt).contiguous(), up.to(tdt).contiguous()
    co = co.to(tdt).contiguous() if co is not None else None
    bu, bup = u.clone(), up.clone()
    girih.run(p, bu, bup, co, c=c, cfg=cfg)
    girih.status(p)
    girih.run(p, u, up, co, c=c, cfg=girih.config(girih.NAIVE))
    torch.cuda.synchronize()
    assert torch.equal(bu, u) and torch.equal(bup, up), (workload, cfg)
