"""Benchmark of the temporally blocked stencil sweep on GB300.

One "step" is one complete sweep: girih_run advancing the whole grid by T time steps with the
configuration the tuner chose for the workload (naive or wavefront-diamond blocked).  Default
workload: 7-point constant-coefficient stencil, FP64, 512^3 interior, T = 64 (the blocked-vs-naive
configuration).  Prints ONE JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]

value     GLUP/s of the configuration the exhaustive tuner recorded as fastest for the workload
          (tuned_configs.json: the naive sweep or a blocked one), inputs resident in HBM; each grid
          (1 GiB per buffer at FP64 512^3) is larger than L2.
naive     the naive GPU sweep (one pass per time step) on the same workload, same timing.
blocked   the fastest wavefront-diamond configuration the tuner recorded, timed the same way, with
          its own roofline (FP64: the DP pipe; FP32: HBM at the Eq. 5 code balance) and DRAM traffic.
e2e       same metric through girih_run_host: pinned host buffers copied in and out every step.
roofline  the roofline of the kernel that `value` times (FP64: the DP pipe, peak = the FMA rate
          measured on this GPU; FP32: HBM, peak = the measured copy bandwidth).
cpu_baseline  the FP64 oracle (plain C loops, OpenMP over z) on this host's cores, on a bounded
          sample of the same grid (fewer time steps).
--impl reference  times only that oracle, per step on a bounded sample, as the reference arm.
Multi-GPU (torchrun): every rank runs an independent replica of the workload (the sweep is not
sharded across GPUs); value = all ranks' updates / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (stencil, dtype, nx, ny, nz, T)
    "7pt_const_f64_512": (0, "f64", 512, 512, 512, 64),
    "7pt_const_f32_512": (0, "f32", 512, 512, 512, 64),
    "7pt_var_f64_480": (1, "f64", 480, 480, 480, 32),
    "7pt_var_f32_480": (1, "f32", 480, 480, 480, 32),
    "25pt_const_f64_384": (2, "f64", 384, 384, 384, 32),
    "25pt_const_f32_384": (2, "f32", 384, 384, 384, 32),
    "25pt_var_f64_384": (3, "f64", 384, 384, 384, 32),
    "25pt_var_f32_384": (3, "f32", 384, 384, 384, 32),
    "25pt_cgrid_f64_384": (4, "f64", 384, 384, 384, 32),
    "25pt_cgrid_f32_384": (4, "f32", 384, 384, 384, 32),
    "27pt_box_f64_512": (5, "f64", 512, 512, 512, 64),
    "27pt_box_f32_512": (5, "f32", 512, 512, 512, 64),
    "7pt_rbgs_f64_512": (6, "f64", 512, 512, 512, 64),
    "7pt_rbgs_f32_512": (6, "f32", 512, 512, 512, 64),
}
DEFAULT = "7pt_const_f64_512"
STENCIL_NAME = {0: "7-point constant", 1: "7-point variable", 2: "25-point constant", 3: "25-point variable",
                4: "25-point constant with factor grid", 5: "27-point box",
                6: "7-point red-black Gauss-Seidel (T half-sweeps)"}
# FP instructions per LUP of the point update (explicitly rounded ops, see csrc/stencil.cuh)
INSTR_PER_LUP = {0: 7, 1: 7, 2: 28, 3: 28, 4: 28, 5: 27, 6: 7}
# DRAM bytes per LUP measured by ncu (dram__bytes_read.sum + dram__bytes_write.sum of one launch
# / LUPs of that launch) for a kernel on a smaller grid of the same workload, with the summary it
# comes from; the roofline's "traffic" scales it to one launch of the benchmark grid.  Keys:
# (kernel, stencil, dtype) with kernel ("naive",) or ("mwd", variant, dw, cluster, threads)
MEASURED_BYTES_PER_LUP = {
    (("naive",), 0, "f64"): (15.67, "profiles/naive_7pt_const_f64_512x384x256.md"),
    (("naive",), 0, "f32"): (7.33, "profiles/naive_7pt_const_f32_512x384x256.md"),
    (("naive",), 1, "f64"): (72.81, "profiles/naive_7pt_var_f64_480x384x192.md"),
    (("naive",), 1, "f32"): (36.45, "profiles/naive_7pt_var_f32_480x384x256.md"),
    (("naive",), 2, "f64"): (24.05, "profiles/naive_25pt_const_f64_384x384x192.md"),
    (("naive",), 2, "f32"): (11.66, "profiles/naive_25pt_const_f32_384x384x256.md"),
    (("naive",), 3, "f64"): (132.06, "profiles/naive_25pt_var_f64_384x384x128.md"),
    (("naive",), 3, "f32"): (65.91, "profiles/naive_25pt_var_f32_384x384x192.md"),
    (("naive",), 4, "f64"): (32.35, "profiles/naive_25pt_cgrid_f64_384x384x192.md"),
    (("naive",), 4, "f32"): (16.11, "profiles/naive_25pt_cgrid_f32_384x384x256.md"),
    (("naive",), 5, "f64"): (15.33, "profiles/naive_27pt_box_f64_512x384x256.md"),
    (("naive",), 5, "f32"): (7.38, "profiles/naive_27pt_box_f32_512x384x256.md"),
    (("naive",), 6, "f64"): (15.7, "profiles/naive_7pt_rbgs_f64_512x384x256.md"),
    (("naive",), 6, "f32"): (7.33, "profiles/naive_7pt_rbgs_f32_512x384x256.md"),
    (("mwd", 7, 6, 8, 224), 1, "f32"): (15.5, "profiles/mwd_ovl_7pt_var_f32_480x384x192.md"),
    (("mwd", 7, 8, 4, 640), 0, "f32"): (4.01, "profiles/mwd_ovl_7pt_const_f32_512x384x256.md"),
    (("mwd", 7, 4, 4, 352), 0, "f64"): (14.57, "profiles/mwd_ovl_7pt_const_f64_512x384x256.md"),
}
# domain-sized streams N_D of the code-balance model and the spatial minimum bytes per LUP (in elements)
ND = {0: 2, 1: 9, 2: 2, 3: 15, 4: 3, 5: 2, 6: 2}
SPATIAL_ELEMS = {0: 2, 1: 9, 2: 3, 3: 16, 4: 4, 5: 2, 6: 2}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def _tuned(workload):
    """(best config, fastest blocked config) recorded by the exhaustive tuner for a workload."""
    path = os.path.join(ROOT, "paper_1510_04995_gb300", "tuned_configs.json")
    try:
        with open(path) as f:
            e = json.load(f).get(workload)
    except Exception:
        return None, None
    if not e:
        return None, None
    if "best" not in e:  # a bare configuration
        return e, None
    return e["best"], e.get("blocked")


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, ws, device):
    """The largest value of x over the ranks (the slowest rank's time); x itself with one rank.
    Used with NCCL on the GPUs, and with gloo on the host in the multi-rank tests."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_glups(lups_per_rank, steps, ws, ms):
    """Whole-job throughput: the updates all ranks made (each rank runs its own replica of the
    workload) divided by the slowest rank's time."""
    return lups_per_rank * steps * ws / (ms * 1e-3) * 1e-9


def cpu_baseline(stencil, nx, ny, nz, budget_s=10.0, max_T=64, min_T=1):
    """Time the FP64 oracle on this host's cores on the workload's grid for a bounded number of steps."""
    import numpy as np

    import oracle
    from paper_1510_04995_gb300 import inputs
    oracle.build()
    cores = len(os.sched_getaffinity(0))
    u, up, co, c = inputs.make_problem(stencil, nx, ny, nz)
    t0 = time.perf_counter()
    oracle.sweep(stencil, u, up, co, c, 1, nx, ny, nz, nthreads=cores)
    t1 = time.perf_counter() - t0
    T = int(max(min_T, min(max_T, budget_s / max(t1, 1e-6))))
    # repeat sweeps of T steps (the workload's T at most) until about budget_s of CPU time
    t0 = time.perf_counter()
    oracle.sweep(stencil, u, up, co, c, T, nx, ny, nz, nthreads=cores)
    reps = int(max(1, min(50, budget_s / max(time.perf_counter() - t0, 1e-6))))
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.sweep(stencil, u, up, co, c, T, nx, ny, nz, nthreads=cores)
    dt = time.perf_counter() - t0
    glups = nx * ny * nz * T * reps / dt * 1e-9
    del u, up, co
    return {"value": glups, "unit": "GLUP/s", "cores": cores, "kind": "oracle",
            "sample": f"{nx}x{ny}x{nz} grid, {reps} sweep(s) of {T} time steps (FP64 oracle, OpenMP over z), "
                      f"{dt:.1f} s"}


def accuracy(stencil, dtype, nx, ny, nz, T, ldx, configs, p, device):
    """Error of the GPU sweep after the full T steps against the FP64 oracle run on the FP64
    inputs: FP64 max normwise relative error (bound 1e-12), FP32 relative L2 error (bound 1e-5
    for the 7-point stencils, 1e-4 for the 25-point ones)."""
    import numpy as np
    import torch

    import oracle
    import paper_1510_04995_gb300 as girih
    from paper_1510_04995_gb300 import inputs
    oracle.build()
    R = inputs.RADIUS[stencil]
    u, up, co, c = inputs.make_problem(stencil, nx, ny, nz)
    ru, rup = u.copy(), up.copy()
    oracle.sweep(stencil, ru, rup, co, c, T, nx, ny, nz, nthreads=len(os.sched_getaffinity(0)))
    ref = ru[R:-R, R:-R, R:-R]
    del ru, rup, u, up, co
    tdt = torch.float64 if dtype == "f64" else torch.float32
    res = {}
    for name, cfg in configs:
        gu, gup, gco, _ = inputs.make_problem(stencil, nx, ny, nz, backend="torch", device=device, ldx=ldx)
        gu, gup = gu.to(tdt).contiguous(), gup.to(tdt).contiguous()
        gco = gco.to(tdt).contiguous() if gco is not None else None
        girih.run(p, gu, gup, gco, c=c, cfg=cfg)
        girih.status(p)
        g = gu[R:-R, R:-R, R:R + nx].double().cpu().numpy()
        del gu, gup, gco
        if dtype == "f64":
            res[name] = float(np.max(np.abs(g - ref)) / np.max(np.abs(ref)))
        else:
            res[name] = float(np.linalg.norm((g - ref).ravel()) / np.linalg.norm(ref.ravel()))
    bound = 1e-12 if dtype == "f64" else (1e-5 if inputs.RADIUS[stencil] == 1 else 1e-4)
    return {"metric": "max normwise relative error" if dtype == "f64" else "relative L2 error",
            "vs": "FP64 oracle, full T", "bound": bound, **res, "ok": all(v <= bound for v in res.values())}


def run_reference(args, wl):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    stencil, dtype, nx, ny, nz, T = WORKLOADS[wl]
    import oracle
    from paper_1510_04995_gb300 import inputs
    oracle.build()
    cores = len(os.sched_getaffinity(0))
    u, up, co, c = inputs.make_problem(stencil, nx, ny, nz)
    t0 = time.perf_counter()
    oracle.sweep(stencil, u, up, co, c, 1, nx, ny, nz, nthreads=cores)
    one = time.perf_counter() - t0
    # each step is a bounded sample: as many time steps of the grid as fit in ~10 s (>= 1)
    steps_per = int(max(1, min(T, 10.0 / max(one, 1e-6) / max(1, args.steps + args.warmup) * 3)))
    for _ in range(args.warmup):
        oracle.sweep(stencil, u, up, co, c, steps_per, nx, ny, nz, nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.sweep(stencil, u, up, co, c, steps_per, nx, ny, nz, nthreads=cores)
    dt = time.perf_counter() - t0
    glups = nx * ny * nz * steps_per * args.steps / dt * 1e-9
    sample = f"{nx}x{ny}x{nz} grid, {steps_per} time steps per bench step (of the workload's {T})"
    line = {"impl": "reference", "metric": "GLUP/s", "value": glups, "unit": "GLUP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl, "stencil": STENCIL_NAME[stencil], "nx": nx, "ny": ny,
                                            "nz": nz, "T": T, "bench_dtype": dtype},
            "cpu_baseline": {"value": glups, "unit": "GLUP/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": glups, "unit": "GLUP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="girih")
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--algo", default="tuned", choices=["tuned", "naive", "mwd"])
    ap.add_argument("--dw", type=int, default=0)
    ap.add_argument("--nf", type=int, default=1)
    ap.add_argument("--cluster", type=int, default=0)
    ap.add_argument("--threads", type=int, default=256)
    ap.add_argument("--variant", type=int, default=0, help="0 FED, 1 RELAXED, 2 FED_BULK, 3 FED_ELEM, 4 RELAXED_ELEM, "
                    "5 FED_PERSISTENT, 6 RELAXED_PERSISTENT, 7 OVERLAP_PERSISTENT")
    ap.add_argument("--zseg", type=int, default=0, help="OVERLAP_PERSISTENT: z planes per tile segment (0: whole tiles)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-naive", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the error check against the FP64 oracle")
    ap.add_argument("--grid", default="", help="override nx,ny,nz (profiling a smaller case of the same kernel)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args, args.workload)

    import torch
    import torch.distributed as dist

    import paper_1510_04995_gb300 as girih
    from paper_1510_04995_gb300 import build as gbuild
    from paper_1510_04995_gb300 import inputs

    ws, rank, local = _dist()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    gbuild.build()
    stencil, dtype, nx, ny, nz, T = WORKLOADS[args.workload]
    if args.grid:
        nx, ny, nz = (int(v) for v in args.grid.split(","))
    # leading dimension padded to a 16-byte multiple (Sect. 4.2.3 pads the leading dimension): rows
    # start on 16-byte boundaries, which lets the blocked kernel move whole rows with bulk copies
    R = inputs.RADIUS[stencil]
    a16 = 16 // (8 if dtype == "f64" else 4)
    ldx = -(-(nx + 2 * R) // a16) * a16
    p = girih.plan(stencil, nx, ny, nz, dtype=dtype, T=T, ldx=ldx)
    if args.algo == "naive":
        cfg = girih.config(girih.NAIVE)
    elif args.algo == "mwd" and args.dw:
        cfg = girih.config(girih.MWD, dw=args.dw, nf=args.nf, cluster=args.cluster or 1, threads=args.threads,
                           variant=args.variant, zseg=args.zseg)
    else:
        tuned, _ = _tuned(args.workload)
        cfg = girih.Config(**tuned) if tuned else p.config
    p.set_config(cfg)
    _, blocked_d = _tuned(args.workload)
    blocked_cfg = girih.Config(**blocked_d) if (blocked_d and args.algo == "tuned") else None
    if cfg.algo == girih.MWD:
        blocked_cfg = cfg

    u, up, co, c = inputs.make_problem(stencil, nx, ny, nz, backend="torch", device=dev, ldx=ldx)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    u, up = u.to(tdt).contiguous(), up.to(tdt).contiguous()
    co = co.to(tdt).contiguous() if co is not None else None
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def timed(config, steps, warmup):
        for _ in range(warmup):
            girih.run(p, u, up, co, c=c, cfg=config, stream=stream)
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            girih.run(p, u, up, co, c=c, cfg=config, stream=stream)
        ev1.record(stream)
        barrier()
        return max_over_ranks(ev0.elapsed_time(ev1), ws, dev)

    lups = nx * ny * nz * T
    with ClockSampler(local) as clk:
        ms = timed(cfg, args.steps, args.warmup)
    clocks = clk.summary()
    value = whole_job_glups(lups, args.steps, ws, ms)
    naive = None
    if not args.no_naive:
        if cfg.algo == girih.NAIVE:
            naive = value
        else:
            nms = timed(girih.config(girih.NAIVE), max(1, args.steps // 2), 1)
            naive = whole_job_glups(lups, max(1, args.steps // 2), ws, nms)
    elem = 8 if dtype == "f64" else 4
    peaks, src = _peaks()
    # spatial-blocking roofline: HBM bandwidth / minimal bytes per LUP (u in, u out; coefficients in)
    spatial = float(peaks["hbm_gbs"]) / (SPATIAL_ELEMS[stencil] * elem)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fma = None
    if dtype == "f64":
        # the DP pipe's rate on this GPU, measured now (8 independent FMA chains per thread over
        # every SM), next to the nominal SMs x 2 DFMA/clk x maximum SM clock
        rate, secs = girih.measure_fma_rate("f64", stream)
        fma = {"measured": rate, "seconds": secs, "sms": sms,
               "nominal": sms * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6}

    def roofline(config, glups_per_gpu):
        """Roofline of one configuration's kernel: FP64 against the DP pipe (explicitly rounded
        ops per LUP x LUP/s vs the measured FMA rate), FP32 against HBM (algorithmic bytes = Eq. 5
        code balance for a blocked sweep, the spatial minimum for the naive one, x LUP/s)."""
        mwd = config.algo == girih.MWD
        key = (("mwd", config.variant, config.dw, config.cluster, config.threads) if mwd else ("naive",),
               stencil, dtype)
        meas = MEASURED_BYTES_PER_LUP.get(key)
        n_launch = p.launch_count(config)
        # one launch of the naive sweep is one time step over the grid; of a blocked sweep, one
        # diamond row (the persistent variants: the whole sweep)
        lpl = nx * ny * nz if not mwd else lups / max(n_launch, 1)
        per_s = glups_per_gpu * 1e9
        if dtype == "f64":
            achieved = per_s * INSTR_PER_LUP[stencil]
            r = {"bound": "alu", "achieved": achieved * 1e-12, "peak": fma["measured"] * 1e-12, "unit": "Tinst/s",
                 "frac": achieved / fma["measured"],
                 "note": f"FP64 instructions/s ({INSTR_PER_LUP[stencil]} explicitly rounded ops per LUP) vs the "
                         f"FMA rate measured on this GPU ({sms} SMs; nominal {sms} x 2 DFMA/clk x max clock = "
                         f"{fma['nominal'] * 1e-12:.3f} T/s); HBM is not the bound"}
        else:
            bc = (girih.model_code_balance(config.dw, inputs.RADIUS[stencil], ND[stencil], elem) if mwd
                  else SPATIAL_ELEMS[stencil] * elem)
            achieved = per_s * bc
            r = {"bound": "hbm", "achieved": achieved * 1e-9, "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                 "frac": achieved * 1e-9 / float(peaks["hbm_gbs"]),
                 "note": f"algorithmic bytes = {'Eq. 5 code balance' if mwd else 'spatial minimum'} {bc:.2f} B/LUP"
                         f" x LUPs ({src} HBM peak)"}
        r["traffic"] = meas[0] * lpl if meas else None
        r["lups_per_launch"] = lpl
        if meas:
            r["traffic_source"] = f"{meas[1]}: {meas[0]} DRAM bytes/LUP x {lpl:.4g} LUPs per launch"
        return r

    blocked = None
    if blocked_cfg is not None:
        if blocked_cfg.as_dict() == cfg.as_dict():
            bg = value
        else:
            bms = timed(blocked_cfg, max(1, args.steps // 2), 1)
            bg = whole_job_glups(lups, max(1, args.steps // 2), ws, bms)
        blocked = {"glups": bg, "config": blocked_cfg.as_dict(), "vs_naive": (bg / naive) if naive else None,
                   "frac_spatial_roofline": bg / ws / spatial, "roofline": roofline(blocked_cfg, bg / ws)}

    # roofline of the dominant kernel: every launch of the timed region is the chosen
    # configuration's kernel (plus the exchange kernel for odd T, which no workload here has)
    launches = p.launch_count(cfg)
    roof = roofline(cfg, value / ws)

    e2e = None
    if not args.no_e2e:
        hu = torch.empty(u.shape, dtype=tdt, pin_memory=True)
        hup = torch.empty(u.shape, dtype=tdt, pin_memory=True)
        hco = torch.empty(co.shape, dtype=tdt, pin_memory=True) if co is not None else None
        hu.copy_(u)
        hup.copy_(up)
        if hco is not None:
            hco.copy_(co)
        girih.run_host(p, hu, hup, hco, c=c, stream=stream)  # warm-up (allocates the staging buffers)
        barrier()
        t0 = time.perf_counter()
        n_e2e = max(1, min(args.steps, 3))
        for _ in range(n_e2e):
            girih.run_host(p, hu, hup, hco, c=c, stream=stream)
        barrier()
        et = max_over_ranks(time.perf_counter() - t0, ws, dev)
        nbytes = u.numel() * elem
        e2e = {"value": lups * n_e2e * ws / et * 1e-9, "unit": "GLUP/s",
               "h2d_bytes_per_step": (2 if inputs.SECOND_ORDER[stencil] else 1) * nbytes
                                     + (co.numel() * elem if co is not None else 0),
               "d2h_bytes_per_step": 2 * nbytes}
        del hu, hup, hco

    cpu = None
    acc = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        del u, up, co
        torch.cuda.empty_cache()
        cpu = cpu_baseline(stencil, nx, ny, nz, max_T=T)
        if not args.no_accuracy:
            cfgs = [("tuned" if args.algo == "tuned" else "measured", cfg)]
            if blocked_cfg is not None and blocked_cfg.as_dict() != cfg.as_dict():
                cfgs.append(("blocked", blocked_cfg))
            acc = accuracy(stencil, dtype, nx, ny, nz, T, ldx, cfgs, p, dev)

    if rank == 0:
        line = {
            "metric": "GLUP/s", "value": value, "unit": "GLUP/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": args.workload, "stencil": STENCIL_NAME[stencil], "nx": nx, "ny": ny, "nz": nz,
                       "T": T, "ldx": ldx, "algo": "mwd" if cfg.algo == girih.MWD else "naive",
                       "kernel_config": cfg.as_dict(),
                       "l2": "inputs larger than L2 (each grid > 126 MB)", "parallelism": f"replicas x{ws}"},
            "naive_glups": naive, "speedup_vs_naive": (value / naive) if naive else None,
            "blocked": blocked, "spatial_roofline_glups": spatial,
            "frac_spatial_roofline": value / ws / spatial,
            "gpu_launches": launches * args.steps,
            "roofline": roof, "clocks": clocks, "e2e": e2e, "cpu_baseline": cpu, "accuracy": acc,
        }
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
