"""Tune the benchmark workloads with the library's exhaustive tuner and record the winners.

    python -m paper_1510_04995_gb300.tune_workloads [--workloads a,b] [--out tuned_configs.json]

For every workload (stencil, dtype, grid, T) this runs girih_tune_exhaustive (Sect. 4.2.2: all
feasible candidates, test length grown until two repetitions agree) on tuner-owned arrays of the
full grid, with the 16-byte aligned leading dimension the benchmark uses, and writes
{workload: {"best": config, "best_glups": rate, "blocked": config, "blocked_glups": rate}} to
tuned_configs.json next to this file ("blocked" is the fastest wavefront-diamond candidate, which
the benchmark reports beside the overall winner), plus the timing database.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import time

from . import F32, F64, MWD, TuneRow, build, check, lib, plan

HERE = os.path.dirname(os.path.abspath(__file__))

WORKLOADS = {
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
RADIUS = {0: 1, 1: 1, 2: 4, 3: 4, 4: 4, 5: 1, 6: 1}


def aligned_ldx(stencil: int, dtype: str, nx: int) -> int:
    a16 = 16 // (8 if dtype == "f64" else 4)
    return -(-(nx + 2 * RADIUS[stencil]) // a16) * a16


def _best_blocked(db_path, stencil, dtype, nx, ny, nz):
    """(config dict, GLUP/s) of the fastest blocked candidate of one problem in the database."""
    from .learned import load_db, problem_key, row_config
    key = (stencil, F64 if dtype == "f64" else F32, nx, ny, nz)
    rows = [r for r in load_db(db_path) if problem_key(r) == key and int(r["algo"]) == MWD]
    if not rows:
        return None
    r = max(rows, key=lambda r: r["glups"])
    return row_config(r).as_dict(), r["glups"]


def tune(names, out_path, db_path, tol=0.05, max_steps=64, log=print):
    build.build()
    res = {}
    if os.path.exists(out_path):
        with open(out_path) as f:
            res = json.load(f)
    for name in names:
        s, d, nx, ny, nz, T = WORKLOADS[name]
        p = plan(s, nx, ny, nz, dtype=d, T=T, ldx=aligned_ldx(s, d, nx))
        best = TuneRow()
        nm = ctypes.c_int32()
        t0 = time.perf_counter()
        check(lib().girih_tune_exhaustive(p.handle, None, 0, tol, max_steps, db_path.encode(), ctypes.byref(best),
                                          ctypes.byref(nm)))
        blk = _best_blocked(db_path, s, d, nx, ny, nz)
        res[name] = {"best": best.cfg.as_dict(), "best_glups": best.glups,
                     "blocked": blk[0] if blk else None, "blocked_glups": blk[1] if blk else None}
        if log:
            log(f"{name}: {nm.value} candidates, {time.perf_counter() - t0:.1f} s, best {best.glups:.1f} GLUP/s "
                f"{best.cfg}")
        p.close()
        with open(out_path, "w") as f:
            json.dump(res, f, indent=1, sort_keys=True)
    return res


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--workloads", default=",".join(WORKLOADS))
    ap.add_argument("--out", default=os.path.join(HERE, "tuned_configs.json"))
    ap.add_argument("--db", default=os.path.join(HERE, "tuned_db.csv"))
    ap.add_argument("--tol", type=float, default=0.05)
    ap.add_argument("--max-steps", type=int, default=64)
    a = ap.parse_args()
    tune(a.workloads.split(","), a.out, a.db, a.tol, a.max_steps)
