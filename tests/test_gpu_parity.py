"""GPU sweeps against the FP64 oracle (element by element) and blocked against naive (bit for bit).

Sizes are ragged on purpose (not multiples of the 32-wide x slabs, of the diamond width or of
the z chunk) and span several tiles; T covers 1, H-1, H, H+1 and 2H+3 so that truncated diamond
rows are exercised.  Tolerances: FP64 max normwise relative error <= 1e-12; FP32 relative L2
error <= 1e-5 (7-point) and <= 1e-4 (25-point) against the FP64 oracle run on the FP64 inputs.
"""
import numpy as np
import pytest

import oracle
import paper_1510_04995_gb300 as girih
from paper_1510_04995_gb300 import inputs

from gpu_util import feasible_cfg, gpu_sweep, normwise, rel_l2

pytestmark = pytest.mark.gpu

SIZES = {1: (70, 45, 33), 4: (70, 50, 29)}
FP32_TOL = {0: 1e-5, 1: 1e-5, 2: 1e-4, 3: 1e-4, 4: 1e-4, 5: 1e-5, 6: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__
    __graft_entry__.build()


def _ref(stencil, nx, ny, nz, T, seed=3):
    u, up, co, c = inputs.make_problem(stencil, nx, ny, nz, seed=seed)
    ru, rup = u.copy(), up.copy()
    oracle.sweep(stencil, ru, rup, co, c, T, nx, ny, nz, nthreads=8)
    return u, up, co, c, ru, rup


MWD_CFGS = {
    1: [dict(dw=4, nf=1, cluster=1, threads=256), dict(dw=8, nf=2, cluster=2, threads=256),
        dict(dw=12, nf=1, cluster=8, threads=1024), dict(dw=6, nf=3, cluster=2, threads=512)],
    4: [dict(dw=8, nf=1, cluster=4, threads=256), dict(dw=16, nf=1, cluster=8, threads=256),
        dict(dw=8, nf=2, cluster=8, threads=128), dict(dw=16, nf=1, cluster=16, threads=256)],
}


@pytest.mark.parametrize("stencil", [0, 1, 2, 3, 4, 5, 6])
def test_naive_fp64_vs_oracle(stencil):
    R = inputs.RADIUS[stencil]
    nx, ny, nz = SIZES[R]
    T = 5
    u, up, co, c, ru, rup = _ref(stencil, nx, ny, nz, T)
    gu, gup = gpu_sweep(stencil, "f64", u, up, co, c, T, nx, ny, nz, girih.config(girih.NAIVE))
    assert normwise(gu, ru, R) <= 1e-12
    assert normwise(gup, rup, R) <= 1e-12
    # the halo is never written
    m = np.ones(u.shape, bool)
    m[R:-R, R:-R, R:-R] = False
    assert np.array_equal(gu[m], u[m]) and np.array_equal(gup[m], up[m])


@pytest.mark.parametrize("stencil", [0, 1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("ci", [0, 1, 2, 3])
def test_mwd_fp64_vs_oracle_and_naive(stencil, ci):
    R = inputs.RADIUS[stencil]
    cfgs = MWD_CFGS[R]
    if ci >= len(cfgs):
        pytest.skip("no such config for this radius")
    kw = cfgs[ci]
    H = kw["dw"] // R
    nx, ny, nz = SIZES[R]
    Ts = [1, H - 1, H, H + 1, 2 * H + 3] if ci == 0 else [H + 1]
    for T in sorted(set(t for t in Ts if t >= 1)):
        u, up, co, c, ru, rup = _ref(stencil, nx, ny, nz, T)
        cfg = feasible_cfg(stencil, "f64", nx, ny, nz, kw)
        bu, bup = gpu_sweep(stencil, "f64", u, up, co, c, T, nx, ny, nz, cfg)
        assert normwise(bu, ru, R) <= 1e-12, (T, kw)
        assert normwise(bup, rup, R) <= 1e-12, (T, kw)
        nu, nup = gpu_sweep(stencil, "f64", u, up, co, c, T, nx, ny, nz, girih.config(girih.NAIVE))
        assert np.array_equal(bu, nu), (T, kw)
        assert np.array_equal(bup, nup), (T, kw)


@pytest.mark.parametrize("stencil", [0, 1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("algo", ["naive", "mwd"])
def test_fp32_error_vs_fp64_oracle(stencil, algo):
    R = inputs.RADIUS[stencil]
    nx, ny, nz = SIZES[R]
    T = 12
    u, up, co, c, ru, rup = _ref(stencil, nx, ny, nz, T)
    cfg = girih.config(girih.NAIVE) if algo == "naive" else feasible_cfg(stencil, "f32", nx, ny, nz, MWD_CFGS[R][1])
    gu, _ = gpu_sweep(stencil, "f32", u, up, co, c, T, nx, ny, nz, cfg)
    assert rel_l2(gu, ru, R) <= FP32_TOL[stencil]


@pytest.mark.parametrize("stencil", [0, 3, 4, 5, 6])
def test_fp32_mwd_bitwise_equals_naive(stencil):
    R = inputs.RADIUS[stencil]
    nx, ny, nz = SIZES[R]
    T = 2 * (8 // R) + 3 if R == 1 else 7
    u, up, co, c = inputs.make_problem(stencil, nx, ny, nz, seed=5)
    for kw in MWD_CFGS[R]:
        bu, bup = gpu_sweep(stencil, "f32", u, up, co, c, T, nx, ny, nz, feasible_cfg(stencil, "f32", nx, ny, nz, kw))
        nu, nup = gpu_sweep(stencil, "f32", u, up, co, c, T, nx, ny, nz, girih.config(girih.NAIVE))
        assert np.array_equal(bu, nu) and np.array_equal(bup, nup), kw


@pytest.mark.parametrize("stencil", [0, 2])
def test_padded_leading_dimension(stencil):
    R = inputs.RADIUS[stencil]
    nx, ny, nz, T = 45, 21, 17, 6
    ldx = nx + 2 * R + 11
    u, up, co, c = inputs.make_problem(stencil, nx, ny, nz, seed=9, ldx=ldx)
    ru, rup = u.copy(), up.copy()
    oracle.sweep(stencil, ru, rup, co, c, T, nx, ny, nz)
    mwd = feasible_cfg(stencil, "f64", nx, ny, nz, dict(dw=2 * R, nf=1, cluster=2, threads=128), ldx=ldx)
    for cfg in (girih.config(girih.NAIVE), mwd):
        gu, _ = gpu_sweep(stencil, "f64", u, up, co, c, T, nx, ny, nz, cfg, ldx=ldx)
        assert normwise(gu[:, :, :nx + 2 * R], ru[:, :, :nx + 2 * R], R) <= 1e-12
        assert np.array_equal(gu[:, :, nx + 2 * R:], u[:, :, nx + 2 * R:])  # padding untouched


@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 2, 5), (33, 1, 9), (1, 40, 3), (5, 7, 1)])
def test_degenerate_shapes(shape):
    nx, ny, nz = shape
    for stencil in (0, 2):
        R = inputs.RADIUS[stencil]
        T = 5
        u, up, co, c, ru, rup = _ref(stencil, nx, ny, nz, T)
        mwd = feasible_cfg(stencil, "f64", nx, ny, nz, dict(dw=2 * R, nf=1, cluster=1, threads=256))
        for cfg in (girih.config(girih.NAIVE), mwd):
            gu, gup = gpu_sweep(stencil, "f64", u, up, co, c, T, nx, ny, nz, cfg)
            assert np.max(np.abs(gu - ru)) <= 1e-12 * max(1.0, np.max(np.abs(ru))), (shape, stencil, cfg)


def test_t0_is_noop():
    u, up, co, c = inputs.make_problem(0, 20, 20, 20)
    gu, gup = gpu_sweep(0, "f64", u, up, co, c, 0, 20, 20, 20,
                        feasible_cfg(0, "f64", 20, 20, 20, dict(dw=8, nf=1, cluster=1, threads=256)))
    assert np.array_equal(gu, u) and np.array_equal(gup, up)


def test_invalid_arguments_leave_buffers_untouched():
    import torch
    p = girih.plan(girih.S7V, 16, 16, 16, dtype="f64", T=3)
    u = torch.ones(p.shape, dtype=torch.float64, device="cuda")
    up = torch.ones(p.shape, dtype=torch.float64, device="cuda")
    assert girih.lib().girih_run(p.handle, u.data_ptr(), up.data_ptr(), None, None, None) == 1  # no coefficients
    assert girih.lib().girih_run(p.handle, u.data_ptr(), u.data_ptr(), None, None, None) == 1  # aliasing
    assert girih.lib().girih_run(p.handle, u.data_ptr() + 4, up.data_ptr(), u.data_ptr(), None, None) == 1
    # FED_BULK on a layout whose rows are not 16-byte multiples (18 FP32 elements) is rejected up front
    p32 = girih.plan(girih.S7C, 16, 16, 16, dtype="f32", T=3)
    assert not p32.feasible(girih.config(girih.MWD, dw=2, nf=1, cluster=1, threads=288, variant=girih.FED_BULK))
    assert p32.feasible(girih.config(girih.MWD, dw=2, nf=1, cluster=1, threads=256, variant=girih.FED))
    bad = girih.config(girih.MWD, dw=3, nf=1, cluster=1, threads=128)
    with pytest.raises(girih.GirihError):
        p.set_config(bad)
    with pytest.raises(girih.GirihError):
        girih.run(p, u, up, torch.ones((7,) + p.shape, dtype=torch.float64, device="cuda"), cfg=bad)
    torch.cuda.synchronize()
    assert bool((u == 1).all()) and bool((up == 1).all())


def test_run_host_matches_device_run():
    stencil, nx, ny, nz, T = 2, 30, 26, 22, 6
    u, up, co, c = inputs.make_problem(stencil, nx, ny, nz, seed=4)
    p = girih.plan(stencil, nx, ny, nz, dtype="f64", T=T)
    hu, hup = u.copy(), up.copy()
    girih.run_host(p, hu, hup, None, c=c)
    gu, gup = gpu_sweep(stencil, "f64", u, up, co, c, T, nx, ny, nz, p.config)
    assert np.array_equal(hu, gu) and np.array_equal(hup, gup)


def test_run_host_first_order_reads_only_u():
    """For a first-order stencil the host entry point builds u_prev on the device from u (its
    halo must equal u's anyway): whatever the host u_prev holds inside, the result equals the
    device run from a u_prev that is a copy of u.  T = 0 leaves both host arrays untouched."""
    stencil, nx, ny, nz, T = 0, 30, 26, 22, 5
    u, up, co, c = inputs.make_problem(stencil, nx, ny, nz, seed=6)
    p = girih.plan(stencil, nx, ny, nz, dtype="f64", T=T)
    hu, hup = u.copy(), up.copy()
    hup[1:-1, 1:-1, 1:-1] = 123.0
    girih.run_host(p, hu, hup, None, c=c)
    gu, gup = gpu_sweep(stencil, "f64", u, u.copy(), co, c, T, nx, ny, nz, p.config)
    assert np.array_equal(hu, gu) and np.array_equal(hup, gup)
    p0 = girih.plan(stencil, nx, ny, nz, dtype="f64", T=0)
    a, b = u.copy(), up.copy()
    b[1:-1, 1:-1, 1:-1] = 7.0
    b0 = b.copy()
    girih.run_host(p0, a, b, None, c=c)
    assert np.array_equal(a, u) and np.array_equal(b, b0)


def test_launch_count():
    p = girih.plan(0, 64, 64, 64, dtype="f64", T=9)
    assert p.launch_count(girih.config(girih.NAIVE)) == 10  # 9 steps + one exchange for odd T
    # dw=8, R=1: rows 0..(T-2)//4+1 -> 3 rows, plus the exchange
    assert p.launch_count(girih.config(girih.MWD, dw=8)) == 4


@pytest.mark.parametrize("stencil,dtype", [(0, "f32"), (1, "f32"), (2, "f32"), (3, "f64"), (0, "f64"), (4, "f32"), (4, "f64")])
def test_bulk_copy_path_equals_element_path(stencil, dtype):
    """The bulk-copy (TMA) data movement of the blocked kernel (FED_BULK, 16-byte aligned leading
    dimension) and the per-element path (FED, unaligned leading dimension) agree bit for bit, and
    with the naive sweep."""
    R = inputs.RADIUS[stencil]
    nx, ny, nz, T = 67, 41, 23, 9
    elem = 8 if dtype == "f64" else 4
    a16 = 16 // elem
    ld_al = -(-(nx + 2 * R) // a16) * a16 + a16       # aligned, with spare columns
    ld_un = ld_al + 1                                  # not a multiple of 16 bytes
    assert (ld_al * elem) % 16 == 0 and (ld_un * elem) % 16 != 0
    dw = 8 if (R == 1 or dtype == "f64") else 16
    outs = []
    # FED_BULK: bulk-copy rows; FED on the aligned layout: 16-byte vector path; FED_ELEM on the
    # aligned layout and FED on the unaligned one: per-element path
    for ldx, variant in ((ld_al, girih.FED_BULK), (ld_al, girih.FED), (ld_al, girih.FED_ELEM), (ld_un, girih.FED)):
        cfg = feasible_cfg(stencil, dtype, nx, ny, nz, dict(dw=dw, nf=1, cluster=4, threads=544, variant=variant),
                           ldx=ldx)
        assert cfg.variant == variant
        u, up, co, c = inputs.make_problem(stencil, nx, ny, nz, seed=21, ldx=ldx)
        gu, gup = gpu_sweep(stencil, dtype, u, up, co, c, T, nx, ny, nz, cfg, ldx=ldx)
        nu, nup = gpu_sweep(stencil, dtype, u, up, co, c, T, nx, ny, nz, girih.config(girih.NAIVE), ldx=ldx)
        w = nx + 2 * R
        assert np.array_equal(gu[:, :, :w], nu[:, :, :w]) and np.array_equal(gup[:, :, :w], nup[:, :, :w])
        assert np.all(gu[:, :, w:] == 0) and np.all(gup[:, :, w:] == 0)  # row padding keeps its (zero) values
        outs.append(gu[:, :, :w])
    assert all(np.array_equal(outs[0], o) for o in outs[1:])


@pytest.mark.parametrize("stencil,dtype", [(0, "f32"), (3, "f32"), (1, "f64"), (2, "f64")])
def test_vector_path_on_unaligned_buffers_falls_back(stencil, dtype):
    """A 16-byte aligned layout whose buffers start off a 16-byte boundary runs the per-element
    path, with the same result."""
    import torch
    from gpu_util import to_dev
    R = inputs.RADIUS[stencil]
    nx, ny, nz, T = 61, 37, 19, 7
    elem = 8 if dtype == "f64" else 4
    a16 = 16 // elem
    ldx = -(-(nx + 2 * R) // a16) * a16
    u, up, co, c = inputs.make_problem(stencil, nx, ny, nz, seed=8, ldx=ldx)
    p = girih.plan(stencil, nx, ny, nz, dtype=dtype, T=T, ldx=ldx)
    cfg = feasible_cfg(stencil, dtype, nx, ny, nz, dict(dw=4 * R, nf=1, cluster=2, threads=256), ldx=ldx)
    outs = []
    for shift in (0, 1):
        n = u.size
        tdt = torch.float64 if dtype == "f64" else torch.float32
        bu = torch.zeros(n + 1, dtype=tdt, device="cuda")[shift:shift + n].view(u.shape)
        bup = torch.zeros(n + 1, dtype=tdt, device="cuda")[shift:shift + n].view(u.shape)
        bu.copy_(to_dev(u, dtype))
        bup.copy_(to_dev(up, dtype))
        assert (bu.data_ptr() % 16 == 0) == (shift == 0)
        dco = to_dev(co, dtype) if co is not None else None
        girih.run(p, bu, bup, dco, c=c, cfg=cfg)
        girih.status(p)
        torch.cuda.synchronize()
        outs.append((bu.double().cpu().numpy(), bup.double().cpu().numpy()))
    nu, nup = gpu_sweep(stencil, dtype, u, up, co, c, T, nx, ny, nz, girih.config(girih.NAIVE), ldx=ldx)
    for gu, gup in outs:
        assert np.array_equal(gu, nu) and np.array_equal(gup, nup)


@pytest.mark.parametrize("stencil", [0, 1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_relaxed_variant(stencil, dtype):
    """The RELAXED synchronisation (neighbour hand-off between the blocks of a cluster instead of a
    cluster barrier) reorders no arithmetic: bit-identical to FED and to the naive sweep, and
    within the FP64 contract of the oracle, for clusters of 2 to 16 blocks."""
    R = inputs.RADIUS[stencil]
    nx, ny, nz = SIZES[R]
    dw = 8 if R == 1 else 16
    T = 2 * (dw // R) + 3
    u, up, co, c, ru, rup = _ref(stencil, nx, ny, nz, T)
    nu, nup = gpu_sweep(stencil, dtype, u, up, co, c, T, nx, ny, nz, girih.config(girih.NAIVE))
    if dtype == "f64":
        assert normwise(nu, ru, R) <= 1e-12
    for cl in (2, 4, 8, 16):
        kw = dict(dw=dw, nf=1 if cl != 4 else 2, cluster=cl, threads=256, variant=girih.RELAXED)
        cfg = feasible_cfg(stencil, dtype, nx, ny, nz, kw)
        assert cfg.variant == girih.RELAXED and cfg.cluster >= 2
        bu, bup = gpu_sweep(stencil, dtype, u, up, co, c, T, nx, ny, nz, cfg)
        assert np.array_equal(bu, nu) and np.array_equal(bup, nup), (cl, cfg)
        fed = girih.config(girih.MWD, dw=cfg.dw, nf=cfg.nf, cluster=cfg.cluster, threads=cfg.threads)
        fu, _ = gpu_sweep(stencil, dtype, u, up, co, c, T, nx, ny, nz, fed)
        assert np.array_equal(bu, fu), (cl, cfg)


def test_bounded_wait_times_out_and_reports():
    """The failure path of the device-side waits: a RELAXED neighbour wait on counters nothing
    advances gives up after its limit, girih_status reports GIRIH_ETIMEOUT once (and clears it),
    and the context stays usable for a correct sweep afterwards."""
    import ctypes
    import time
    p = girih.plan(girih.S7C, 40, 30, 20, dtype="f64", T=4)
    t0 = time.perf_counter()
    girih.check(girih.lib().girih_check_bounded_wait(p.handle, ctypes.c_int64(20_000_000), None))  # 20 ms
    rc = girih.lib().girih_status(p.handle, None)
    assert rc == 5, (rc, girih.last_error())  # GIRIH_ETIMEOUT
    assert time.perf_counter() - t0 < 10.0
    assert girih.lib().girih_status(p.handle, None) == 0  # cleared
    assert girih.lib().girih_check_bounded_wait(p.handle, ctypes.c_int64(10), None) == 1  # limit out of range
    u, up, co, c, ru, rup = _ref(0, 40, 30, 20, 4)
    gu, _ = gpu_sweep(0, "f64", u, up, co, c, 4, 40, 30, 20,
                      feasible_cfg(0, "f64", 40, 30, 20, dict(dw=4, nf=1, cluster=2, threads=256, variant=girih.RELAXED)))
    assert normwise(gu, ru, 1) <= 1e-12


def _aligned_ldx(nx, R, dtype):
    a16 = 16 // (8 if dtype == "f64" else 4)
    return -(-(nx + 2 * R) // a16) * a16


@pytest.mark.parametrize("stencil", [0, 1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_persistent_schedule(stencil, dtype):
    """FED_PERSISTENT (one launch per sweep; clusters take diamonds from a FIFO and start each once
    its two parent diamonds have completed, Sect. 4.2.3) changes the order tiles run in, not their
    arithmetic: bit-identical to the naive sweep and to the row-by-row FED launches, for truncated
    and full diamond rows, clusters of 1 to 8 blocks, and repeated sweeps on one plan."""
    R = inputs.RADIUS[stencil]
    nx, ny, nz = SIZES[R]
    ldx = _aligned_ldx(nx, R, dtype)
    dws = (4, 8) if R == 1 else (8, 16)
    for dw, cl, nf in ((dws[0], 1, 1), (dws[1], 2, 2), (dws[1], 8, 1)):
        H = dw // R
        for T in (1, H - 1, 2 * H + 3):
            u, up, co, c = inputs.make_problem(stencil, nx, ny, nz, seed=31 + T, ldx=ldx)
            nu, nup = gpu_sweep(stencil, dtype, u, up, co, c, T, nx, ny, nz, girih.config(girih.NAIVE), ldx=ldx)
            kw = dict(dw=dw, nf=nf, cluster=cl, threads=256, variant=girih.FED_PERSISTENT)
            cfg = feasible_cfg(stencil, dtype, nx, ny, nz, kw, ldx=ldx)
            assert cfg.variant == girih.FED_PERSISTENT
            pu, pup = gpu_sweep(stencil, dtype, u, up, co, c, T, nx, ny, nz, cfg, ldx=ldx)
            assert np.array_equal(pu, nu) and np.array_equal(pup, nup), (dw, cl, T, cfg)
            fed = girih.config(girih.MWD, dw=cfg.dw, nf=cfg.nf, cluster=cfg.cluster, threads=cfg.threads)
            fu, _ = gpu_sweep(stencil, dtype, u, up, co, c, T, nx, ny, nz, fed, ldx=ldx)
            assert np.array_equal(pu, fu)


def test_persistent_schedule_reuse_and_rejects_unaligned():
    """One plan runs several persistent sweeps (the completion flags of a sweep carry its epoch,
    so earlier sweeps' flags never release a diamond) and switches diamond width (the diamond list
    is rebuilt); the variant needs the vector layout and says so otherwise."""
    import torch
    from gpu_util import to_dev
    stencil, dtype, nx, ny, nz, T = 0, "f64", 70, 45, 33, 11
    ldx = _aligned_ldx(nx, 1, dtype)
    u, up, co, c = inputs.make_problem(stencil, nx, ny, nz, seed=5, ldx=ldx)
    p = girih.plan(stencil, nx, ny, nz, dtype=dtype, T=T, ldx=ldx)
    du, dup = to_dev(u, dtype), to_dev(up, dtype)
    cur_u, cur_up = u, up
    for i, dw in enumerate((8, 8, 4, 8, 4)):
        cfg = girih.config(girih.MWD, dw=dw, nf=1, cluster=2, threads=256, variant=girih.FED_PERSISTENT)
        girih.run(p, du, dup, None, c=c, cfg=cfg)
        girih.status(p)
        torch.cuda.synchronize()
        cur_u, cur_up = gpu_sweep(stencil, dtype, cur_u, cur_up, co, c, T, nx, ny, nz, girih.config(girih.NAIVE),
                                  ldx=ldx)
        assert np.array_equal(du.cpu().numpy(), cur_u) and np.array_equal(dup.cpu().numpy(), cur_up), i
    pun = girih.plan(stencil, nx, ny, nz, dtype=dtype, T=T, ldx=ldx + 1)
    bad = girih.config(girih.MWD, dw=8, nf=1, cluster=2, threads=256, variant=girih.FED_PERSISTENT)
    assert not pun.feasible(bad)
    assert p.launch_count(bad) == 2  # one persistent launch + the exchange for odd T


# (dw, cluster, threads): 1, 2 and 4 tasks per computing thread (the last two warps move data)
ASYNC_CFGS = [(4, 1, 256), (8, 2, 224), (8, 2, 160), (8, 4, 128), (12, 8, 96), (6, 16, 96), (16, 2, 512)]


@pytest.mark.parametrize("stencil", [0, 1, 6])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_relaxed_persistent(stencil, dtype):
    """RELAXED_PERSISTENT (the persistent FIFO schedule with neighbour-only synchronisation: a block
    waits per step for its own results and for the exact halo bytes its two neighbours pushed)
    reorders tiles and synchronises differently, but never changes a point's arithmetic:
    bit-identical to the naive sweep for clusters of 1 to 16 blocks, truncated and full diamond
    rows, and thread counts that give 1, 2 or 4 tasks per computing thread."""
    nx, ny, nz = SIZES[1]
    ldx = _aligned_ldx(nx, 1, dtype)
    for dw, cl, th in ASYNC_CFGS:
        H = dw
        for T in (1, H - 1, 2 * H + 3):
            u, up, co, c = inputs.make_problem(stencil, nx, ny, nz, seed=17 + T + dw, ldx=ldx)
            nu, nup = gpu_sweep(stencil, dtype, u, up, co, c, T, nx, ny, nz, girih.config(girih.NAIVE), ldx=ldx)
            kw = dict(dw=dw, nf=1, cluster=cl, threads=th, variant=girih.RELAXED_PERSISTENT)
            cfg = feasible_cfg(stencil, dtype, nx, ny, nz, kw, ldx=ldx)
            assert cfg.variant == girih.RELAXED_PERSISTENT
            pu, pup = gpu_sweep(stencil, dtype, u, up, co, c, T, nx, ny, nz, cfg, ldx=ldx)
            assert np.array_equal(pu, nu) and np.array_equal(pup, nup), (dw, cl, T, cfg)


@pytest.mark.parametrize("shape", [(1, 1, 1), (33, 1, 9), (5, 70, 3), (129, 7, 40), (2, 2, 2)])
def test_relaxed_persistent_degenerate_shapes(shape):
    nx, ny, nz = shape
    for dtype in ("f32", "f64"):
        ldx = _aligned_ldx(nx, 1, dtype)
        for stencil in (0, 1, 6):
            T = 7
            u, up, co, c = inputs.make_problem(stencil, nx, ny, nz, seed=4, ldx=ldx)
            nu, nup = gpu_sweep(stencil, dtype, u, up, co, c, T, nx, ny, nz, girih.config(girih.NAIVE), ldx=ldx)
            for dw, cl in ((4, 2), (8, 4)):
                cfg = feasible_cfg(stencil, dtype, nx, ny, nz,
                                   dict(dw=dw, nf=1, cluster=cl, threads=256, variant=girih.RELAXED_PERSISTENT),
                                   ldx=ldx)
                pu, pup = gpu_sweep(stencil, dtype, u, up, co, c, T, nx, ny, nz, cfg, ldx=ldx)
                assert np.array_equal(pu, nu) and np.array_equal(pup, nup), (shape, dtype, stencil, cfg)


def test_relaxed_persistent_rejections():
    """The variant exists for the radius-1 first-order stencils on the vector layout: other
    stencils, unaligned layouts and unaligned coefficient grids are rejected with nothing enqueued."""
    import torch
    from gpu_util import to_dev
    cfg = girih.config(girih.MWD, dw=8, nf=1, cluster=2, threads=256, variant=girih.RELAXED_PERSISTENT)
    for stencil in (2, 3, 4, 5):
        R = inputs.RADIUS[stencil]
        nx, ny, nz = SIZES[R]
        p = girih.plan(stencil, nx, ny, nz, dtype="f32", T=3, ldx=_aligned_ldx(nx, R, "f32"))
        bad = girih.config(girih.MWD, dw=2 * R * 4, nf=1, cluster=2, threads=256, variant=girih.RELAXED_PERSISTENT)
        assert not p.feasible(bad), stencil
    nx, ny, nz = SIZES[1]
    ldx = _aligned_ldx(nx, 1, "f32")
    assert not girih.plan(0, nx, ny, nz, dtype="f32", T=3, ldx=ldx + 1).feasible(cfg)
    p0 = girih.plan(0, nx, ny, nz, dtype="f32", T=3, ldx=ldx)
    assert not p0.feasible(girih.config(girih.MWD, dw=8, nf=2, cluster=2, threads=256,
                                        variant=girih.RELAXED_PERSISTENT))  # one plane per step
    assert not p0.feasible(girih.config(girih.MWD, dw=16, nf=1, cluster=2, threads=64,
                                        variant=girih.RELAXED_PERSISTENT))  # more tasks than 4 per thread
    p = girih.plan(1, nx, ny, nz, dtype="f32", T=3, ldx=ldx)
    assert p.feasible(cfg)
    u, up, co, c = inputs.make_problem(1, nx, ny, nz, seed=2, ldx=ldx)
    du, dup = to_dev(u, "f32"), to_dev(up, "f32")
    big = torch.zeros(co.size + 1, dtype=torch.float32, device="cuda")
    dco = big[1:].view(co.shape)  # 4 bytes past a 256-byte boundary
    dco.copy_(to_dev(co, "f32"))
    before = du.clone()
    with pytest.raises(girih.GirihError):
        girih.run(p, du, dup, dco, c=c, cfg=cfg)
    torch.cuda.synchronize()
    assert torch.equal(du, before)


# (dw, cluster, threads) on the 70-wide grid: 1, 2 and 4 tasks per computing thread, clusters of 1
# to 16 blocks (slabs of 72 down to 6 columns, widened by up to 16 columns per side), one-level
# diamonds (dw = 2)
OVL_CFGS = [(4, 1, 256), (8, 2, 288), (8, 2, 160), (8, 4, 96), (12, 8, 224), (6, 16, 96), (16, 8, 512), (2, 4, 64)]


@pytest.mark.parametrize("stencil", [0, 1, 6])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_overlap_persistent(stencil, dtype):
    """OVERLAP_PERSISTENT (blocks update their x slab widened by the halo each level needs and
    repeat the neighbours' edge columns instead of exchanging them; final values wait only for
    the neighbours' staging progress) never changes a point's arithmetic: bit-identical to the
    naive sweep over cluster sizes, diamond widths, block sizes, truncated and full diamond rows."""
    nx, ny, nz = SIZES[1]
    ldx = _aligned_ldx(nx, 1, dtype)
    for dw, cl, th in OVL_CFGS:
        H = dw
        for T in (1, H - 1, 2 * H + 3):
            if T < 1:
                continue
            u, up, co, c = inputs.make_problem(stencil, nx, ny, nz, seed=29 + T + dw, ldx=ldx)
            nu, nup = gpu_sweep(stencil, dtype, u, up, co, c, T, nx, ny, nz, girih.config(girih.NAIVE), ldx=ldx)
            kw = dict(dw=dw, nf=1, cluster=cl, threads=th, variant=girih.OVERLAP_PERSISTENT)
            if dw == 16 and dtype == "f64":
                kw["dw"] = 12  # the FP64 ring of a 16-wide diamond exceeds the block's shared memory
            cfg = feasible_cfg(stencil, dtype, nx, ny, nz, kw, ldx=ldx)
            assert cfg.variant == girih.OVERLAP_PERSISTENT
            pu, pup = gpu_sweep(stencil, dtype, u, up, co, c, T, nx, ny, nz, cfg, ldx=ldx)
            assert np.array_equal(pu, nu) and np.array_equal(pup, nup), (dw, cl, T, cfg)


# radius 4 on the 70-wide grid: one-level diamonds (Dw = 2R) on a whole-row slab, and three-level
# diamonds (Dw = 4R, slabs widened by 8 and 4 columns per side) at 1 and 2 tasks per thread
OVL_R4_CFGS = [(8, 1, 256), (16, 4, 288), (16, 4, 176), (16, 8, 224)]


@pytest.mark.parametrize("stencil", [2, 3, 4])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_overlap_persistent_radius4(stencil, dtype):
    """The overlapped-slab kernel on the 25-point stencils (second order in time, constant,
    variable and factor-grid coefficients): bit-identical to the naive sweep.  FP64 rings of
    Dw = 4R diamonds exceed the shared memory, so FP64 runs Dw = 2R."""
    nx, ny, nz = SIZES[4]
    ldx = _aligned_ldx(nx, 4, dtype)
    for dw, cl, th in OVL_R4_CFGS:
        if dtype == "f64":
            dw = 8
        for T in (1, 3, 2 * (dw // 4) + 3):
            u, up, co, c = inputs.make_problem(stencil, nx, ny, nz, seed=41 + T + dw, ldx=ldx)
            nu, nup = gpu_sweep(stencil, dtype, u, up, co, c, T, nx, ny, nz, girih.config(girih.NAIVE), ldx=ldx)
            kw = dict(dw=dw, nf=1, cluster=cl, threads=th, variant=girih.OVERLAP_PERSISTENT)
            cfg = feasible_cfg(stencil, dtype, nx, ny, nz, kw, ldx=ldx)
            assert cfg.variant == girih.OVERLAP_PERSISTENT
            pu, pup = gpu_sweep(stencil, dtype, u, up, co, c, T, nx, ny, nz, cfg, ldx=ldx)
            assert np.array_equal(pu, nu) and np.array_equal(pup, nup), (dw, cl, T, cfg)


@pytest.mark.parametrize("shape", [(1, 1, 1), (33, 1, 9), (5, 70, 3), (129, 7, 40), (2, 2, 2), (300, 9, 5)])
def test_overlap_persistent_degenerate_shapes(shape):
    """Slabs narrower than their widening, blocks with no columns, one-row and one-plane grids."""
    nx, ny, nz = shape
    for dtype in ("f32", "f64"):
        ldx = _aligned_ldx(nx, 1, dtype)
        for stencil in (0, 1, 6):
            T = 7
            u, up, co, c = inputs.make_problem(stencil, nx, ny, nz, seed=6, ldx=ldx)
            nu, nup = gpu_sweep(stencil, dtype, u, up, co, c, T, nx, ny, nz, girih.config(girih.NAIVE), ldx=ldx)
            for dw, cl in ((4, 2), (8, 4), (6, 16)):
                cfg = feasible_cfg(stencil, dtype, nx, ny, nz,
                                   dict(dw=dw, nf=1, cluster=cl, threads=256, variant=girih.OVERLAP_PERSISTENT),
                                   ldx=ldx)
                pu, pup = gpu_sweep(stencil, dtype, u, up, co, c, T, nx, ny, nz, cfg, ldx=ldx)
                assert np.array_equal(pu, nu) and np.array_equal(pup, nup), (shape, dtype, stencil, cfg)


# z segments of one plane, shorter than the stored band, ragged (33 = 4 x 7 + 5) and longer than
# the band
OVL_ZSEG = [1, 3, 7, 16]


@pytest.mark.parametrize("stencil", [0, 1, 6])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_overlap_persistent_zsegments(stencil, dtype):
    """OVERLAP_PERSISTENT with its tiles split along z (Sect. 8: each parallelepiped segment is
    an item of the persistent schedule, started once the tile's previous segment and the parents'
    segments it reads have completed; values cross segments through global memory): bit-identical
    to the naive sweep over segment lengths, cluster sizes, diamond widths and truncated rows."""
    nx, ny, nz = SIZES[1]
    ldx = _aligned_ldx(nx, 1, dtype)
    for dw, cl, th in [(4, 1, 256), (8, 4, 96), (6, 16, 96), (12, 8, 224)]:
        for T in (dw - 1, 2 * dw + 3):
            u, up, co, c = inputs.make_problem(stencil, nx, ny, nz, seed=53 + T + dw, ldx=ldx)
            nu, nup = gpu_sweep(stencil, dtype, u, up, co, c, T, nx, ny, nz, girih.config(girih.NAIVE), ldx=ldx)
            for zs in OVL_ZSEG:
                kw = dict(dw=dw, nf=1, cluster=cl, threads=th, variant=girih.OVERLAP_PERSISTENT, zseg=zs)
                cfg = feasible_cfg(stencil, dtype, nx, ny, nz, kw, ldx=ldx)
                assert cfg.zseg == zs
                pu, pup = gpu_sweep(stencil, dtype, u, up, co, c, T, nx, ny, nz, cfg, ldx=ldx)
                assert np.array_equal(pu, nu) and np.array_equal(pup, nup), (dw, cl, T, zs, cfg)


@pytest.mark.parametrize("stencil", [2, 3, 4])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_overlap_persistent_zsegments_radius4(stencil, dtype):
    """z segments of the 25-point sweeps (second order in time: the stored band also carries level
    t-2 for the centre of the next segment's updates): bit-identical to the naive sweep."""
    nx, ny, nz = SIZES[4]
    ldx = _aligned_ldx(nx, 4, dtype)
    for dw, cl, th in [(8, 1, 256), (16, 4, 288)]:
        if dtype == "f64":
            dw = 8
        for T in (3, 2 * (dw // 4) + 3):
            u, up, co, c = inputs.make_problem(stencil, nx, ny, nz, seed=61 + T + dw, ldx=ldx)
            nu, nup = gpu_sweep(stencil, dtype, u, up, co, c, T, nx, ny, nz, girih.config(girih.NAIVE), ldx=ldx)
            for zs in (1, 5, 12):
                kw = dict(dw=dw, nf=1, cluster=cl, threads=th, variant=girih.OVERLAP_PERSISTENT, zseg=zs)
                cfg = feasible_cfg(stencil, dtype, nx, ny, nz, kw, ldx=ldx)
                assert cfg.zseg == zs
                pu, pup = gpu_sweep(stencil, dtype, u, up, co, c, T, nx, ny, nz, cfg, ldx=ldx)
                assert np.array_equal(pu, nu) and np.array_equal(pup, nup), (dw, cl, T, zs, cfg)


def test_zsegments_of_nz_planes_or_more_are_whole_tiles():
    """zseg >= nz leaves one segment per tile: the sweep runs whole tiles, bit for bit naive."""
    nx, ny, nz = SIZES[1]
    ldx = _aligned_ldx(nx, 1, "f32")
    u, up, co, c = inputs.make_problem(1, nx, ny, nz, seed=71, ldx=ldx)
    T = 9
    nu, nup = gpu_sweep(1, "f32", u, up, co, c, T, nx, ny, nz, girih.config(girih.NAIVE), ldx=ldx)
    for zs in (nz, 10 * nz):
        cfg = feasible_cfg(1, "f32", nx, ny, nz,
                           dict(dw=8, nf=1, cluster=4, threads=160, variant=girih.OVERLAP_PERSISTENT, zseg=zs), ldx=ldx)
        assert cfg.zseg == zs
        pu, pup = gpu_sweep(1, "f32", u, up, co, c, T, nx, ny, nz, cfg, ldx=ldx)
        assert np.array_equal(pu, nu) and np.array_equal(pup, nup), zs


def test_zsegments_rejections_and_tuner_candidates():
    """zseg is OVERLAP_PERSISTENT's alone and not negative; the tuner adds segmented candidates
    (32, 64, 128 planes) exactly where a diamond row has fewer diamonds than the device has
    clusters."""
    import torch
    nx, ny, nz = SIZES[1]
    ldx = _aligned_ldx(nx, 1, "f32")
    p = girih.plan(0, nx, ny, nz, dtype="f32", T=3, ldx=ldx)
    assert p.feasible(girih.config(girih.MWD, dw=8, nf=1, cluster=2, threads=256,
                                   variant=girih.OVERLAP_PERSISTENT, zseg=4))
    assert not p.feasible(girih.config(girih.MWD, dw=8, nf=1, cluster=2, threads=256,
                                       variant=girih.OVERLAP_PERSISTENT, zseg=-1))
    for v in (girih.FED, girih.FED_PERSISTENT, girih.RELAXED_PERSISTENT):
        assert not p.feasible(girih.config(girih.MWD, dw=8, nf=1, cluster=2, threads=320, variant=v, zseg=4)), v
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for ny in (64, 2048):
        q = girih.plan(1, 256, ny, 256, dtype="f32", T=8, ldx=_aligned_ldx(256, 1, "f32"))
        cands = q.candidates()
        ovl = [c for c in cands if c.variant == girih.OVERLAP_PERSISTENT]
        for dw, cl, th in {(c.dw, c.cluster, c.threads) for c in ovl}:
            segs = {c.zseg for c in ovl if (c.dw, c.cluster, c.threads) == (dw, cl, th)}
            few = (ny + dw - 1) // dw + 1 < max(sms // cl, 1)
            assert segs == ({0, 32, 64, 128} if few else {0}), (ny, dw, cl, th, segs)
        assert all(c.zseg == 0 for c in cands if c.variant != girih.OVERLAP_PERSISTENT)


def test_overlap_persistent_rejections():
    """The box stencil, unaligned layouts, nf > 1 and blocks too small for the widened tile are
    rejected."""
    nx, ny, nz = SIZES[1]
    for stencil in (5,):
        R = inputs.RADIUS[stencil]
        p = girih.plan(stencil, *SIZES[R], dtype="f32", T=3, ldx=_aligned_ldx(SIZES[R][0], R, "f32"))
        assert not p.feasible(girih.config(girih.MWD, dw=8 * R, nf=1, cluster=2, threads=256,
                                           variant=girih.OVERLAP_PERSISTENT)), stencil
    ldx = _aligned_ldx(nx, 1, "f32")
    cfg = girih.config(girih.MWD, dw=8, nf=1, cluster=2, threads=256, variant=girih.OVERLAP_PERSISTENT)
    assert not girih.plan(0, nx, ny, nz, dtype="f32", T=3, ldx=ldx + 1).feasible(cfg)
    p0 = girih.plan(0, nx, ny, nz, dtype="f32", T=3, ldx=ldx)
    assert p0.feasible(cfg)
    assert not p0.feasible(girih.config(girih.MWD, dw=8, nf=2, cluster=2, threads=256,
                                        variant=girih.OVERLAP_PERSISTENT))
    assert not p0.feasible(girih.config(girih.MWD, dw=16, nf=1, cluster=2, threads=64,
                                        variant=girih.OVERLAP_PERSISTENT))  # 848 tasks > 4 x 32


def test_persistent_schedule_on_fresh_plan_and_nonblocking_stream():
    """The plan's completion flags are cleared on the sweep's own stream: a persistent sweep
    launched on a non-blocking stream right after the plan is created (and after earlier plans
    whose freed flag buffers the allocator may hand out again, still holding their epochs) is
    ordered after that clear and equals the naive sweep bit for bit."""
    import torch
    from gpu_util import to_dev
    stencil, dtype, nx, ny, nz, T = 0, "f32", 70, 45, 33, 9
    ldx = _aligned_ldx(nx, 1, dtype)
    u, up, co, c = inputs.make_problem(stencil, nx, ny, nz, seed=8, ldx=ldx)
    nu, nup = gpu_sweep(stencil, dtype, u, up, co, c, T, nx, ny, nz, girih.config(girih.NAIVE), ldx=ldx)
    cfg = girih.config(girih.MWD, dw=4, nf=1, cluster=2, threads=256, variant=girih.FED_PERSISTENT)
    side = torch.cuda.Stream()  # torch's side streams do not synchronise with the legacy stream
    for rep in range(4):
        p = girih.plan(stencil, nx, ny, nz, dtype=dtype, T=T, ldx=ldx)
        du, dup = to_dev(u, dtype), to_dev(up, dtype)
        torch.cuda.synchronize()
        with torch.cuda.stream(side):
            girih.run(p, du, dup, None, c=c, cfg=cfg, stream=side)
            girih.status(p, stream=side)
        side.synchronize()
        assert np.array_equal(du.cpu().numpy(), nu) and np.array_equal(dup.cpu().numpy(), nup), rep
        del p


@pytest.mark.parametrize("stencil", [5, 6])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_vector_only_stencils_paths_and_layouts(stencil, dtype):
    """The 27-point box stencil and red-black Gauss-Seidel (Sect. 8.4): the box stencil's diagonal
    dependencies (edges and corners of the tile) and red-black's colour-masked half-sweeps are
    met by the same diamonds and wavefront.  The vector path (FED), the bulk-copy path
    (FED_BULK) and the persistent schedule agree with the naive sweep bit for bit, including
    truncated diamond rows and clusters that split x; layouts the vector path cannot take are
    rejected for the blocked sweep, while the naive sweep takes them."""
    nx, ny, nz = 61, 47, 29
    ldx = _aligned_ldx(nx, 1, dtype) + (16 // (8 if dtype == "f64" else 4))   # spare columns
    for T in (1, 3, 4, 5, 11):
        u, up, co, c = inputs.make_problem(stencil, nx, ny, nz, seed=40 + T, ldx=ldx)
        nu, nup = gpu_sweep(stencil, dtype, u, up, co, c, T, nx, ny, nz, girih.config(girih.NAIVE), ldx=ldx)
        if dtype == "f64":
            ru, rup = u.copy(), up.copy()
            oracle.sweep(stencil, ru, rup, None, c, T, nx, ny, nz, nthreads=8)
            assert normwise(nu[:, :, :nx + 2], ru[:, :, :nx + 2], 1) <= 1e-12
        for kw in (dict(dw=4, nf=1, cluster=2, threads=256, variant=girih.FED),
                   dict(dw=8, nf=2, cluster=4, threads=256, variant=girih.FED_BULK),
                   dict(dw=6, nf=1, cluster=8, threads=256, variant=girih.FED_PERSISTENT),
                   dict(dw=2, nf=1, cluster=1, threads=256, variant=girih.FED_PERSISTENT)):
            cfg = feasible_cfg(stencil, dtype, nx, ny, nz, kw, ldx=ldx)
            assert cfg.variant == kw["variant"]
            bu, bup = gpu_sweep(stencil, dtype, u, up, co, c, T, nx, ny, nz, cfg, ldx=ldx)
            assert np.array_equal(bu, nu) and np.array_equal(bup, nup), (T, kw)
    p_un = girih.plan(stencil, nx, ny, nz, dtype=dtype, T=3, ldx=ldx + 1)
    assert not p_un.feasible(girih.config(girih.MWD, dw=4, nf=1, cluster=2, threads=256))
    assert not girih.plan(stencil, nx, ny, nz, dtype=dtype, T=3, ldx=ldx).feasible(
        girih.config(girih.MWD, dw=4, nf=1, cluster=2, threads=256, variant=girih.FED_ELEM))
    u, up, co, c = inputs.make_problem(stencil, nx, ny, nz, seed=3, ldx=ldx + 1)
    ru, rup = u.copy(), up.copy()
    oracle.sweep(stencil, ru, rup, None, c, 3, nx, ny, nz)
    gu, _ = gpu_sweep(stencil, "f64", u, up, co, c, 3, nx, ny, nz, girih.config(girih.NAIVE), ldx=ldx + 1)
    assert normwise(gu[:, :, :nx + 2], ru[:, :, :nx + 2], 1) <= 1e-12


@pytest.mark.parametrize("stencil", [5, 6])
@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 2, 5), (33, 1, 9), (1, 40, 3), (5, 7, 1)])
def test_vector_only_stencils_degenerate_shapes(stencil, shape):
    nx, ny, nz = shape
    ldx = _aligned_ldx(nx, 1, "f64")
    u, up, co, c = inputs.make_problem(stencil, nx, ny, nz, ldx=ldx)
    ru, rup = u.copy(), up.copy()
    oracle.sweep(stencil, ru, rup, None, c, 5, nx, ny, nz)
    mwd = feasible_cfg(stencil, "f64", nx, ny, nz, dict(dw=2, nf=1, cluster=1, threads=256), ldx=ldx)
    for cfg in (girih.config(girih.NAIVE), mwd):
        gu, _ = gpu_sweep(stencil, "f64", u, up, co, c, 5, nx, ny, nz, cfg, ldx=ldx)
        assert np.max(np.abs(gu - ru)) <= 1e-12 * max(1.0, np.max(np.abs(ru))), (shape, cfg)
