"""Learned tuner: the network of ``csrc/mlp.cu`` trained on the exhaustive tuner's own timings.

The paper's auto-tuner (Sect. 4.2.2) measures every thread-group shape and hill-climbs the
diamond and wavefront widths.  Here the exhaustive tuner (``girih_tune_exhaustive``) records one
row per feasible candidate into a CSV timing database.  This module:

* ``collect``  runs the exhaustive tuner over a list of problems and appends to the database,
  recording the wall time each problem's exhaustive tuning took;
* ``train``    fits the 3-layer network (16 -> 64 -> 64 -> 1, ReLU) with the library's CUDA
  forward/backward/Adam kernels to the per-problem centred log throughput of each candidate
  (only the ranking within a problem matters, so the problem's mean is removed);
* ``evaluate`` scores held-out problems: the network ranks all candidates, the best measured of
  its top k is compared with the exhaustive best (regret) and the k measurements' cost with the
  exhaustive tuning cost;
* ``tune``     the live learned tuner on one plan (``girih_tune_learned``: score, measure top k).

Everything numeric runs in the library (features, network, measurement); numpy only reshapes.
"""
from __future__ import annotations

import ctypes
import csv
import math
import os
import time

import numpy as np

from . import (F32, F64, FED, FED_BULK, MLP_FEATURES, MWD, NAIVE, OVERLAP_PERSISTENT, RADIUS, RELAXED,
               RELAXED_PERSISTENT, Config, TuneRow, check, config, config_array, lib, model_code_balance, plan)

# The 12 non-cubic grids of the learned-tuner sweep (nx, ny, nz), and the held-out ones (#3, #7, #10).
GRIDS = [(128, 256, 512), (256, 128, 512), (192, 384, 512), (256, 512, 512), (384, 256, 512),
         (320, 640, 512), (512, 384, 512), (448, 768, 512), (640, 512, 512), (576, 704, 512),
         (768, 512, 512), (768, 768, 512)]
HELD_OUT = (2, 6, 9)
FIELDS = ["stencil", "dtype", "nx", "ny", "nz", "algo", "dw", "nf", "cluster", "threads", "variant", "glups",
          "seconds", "steps", "smem", "tune_seconds", "zseg"]  # zseg: absent in rows written before it existed


def _dt(d):
    return {"f64": F64, "f32": F32, F64: F64, F32: F32}[d]


def aligned_ldx(stencil, nx, dtype) -> int:
    """The leading dimension the experiment uses: nx + 2R rounded up to 16 bytes (the layout the
    vector, bulk-copy and neighbour-synchronised paths of the blocked sweep take)."""
    a16 = 16 // (8 if _dt(dtype) == F64 else 4)
    return -(-(nx + 2 * RADIUS[stencil]) // a16) * a16


def problem_plan(stencil, dtype, nx, ny, nz, T):
    return plan(stencil, nx, ny, nz, dtype=dtype, T=T, ldx=aligned_ldx(stencil, nx, dtype))


def space(p) -> list:
    """The experiment's search space for a plan: the naive sweep and the feasible blocked sweeps
    with diamond widths 2R, 4R, 8R, 16R, wavefront widths 1 and 2, clusters 1, 4, 8, 16, 256 or
    512 threads, and the FED / FED_BULK data paths (RELAXED where the cluster has more than one
    block, with 512 threads); plus the neighbour-synchronised and overlapped-slab persistent
    sweeps (RELAXED_PERSISTENT, OVERLAP_PERSISTENT) for the same diamond widths and clusters 4, 8,
    16, in the block sizes the tuner enumerates for them (the tile's tasks at 1, 2 or 4 per
    computing thread)."""
    R = p.R
    out = [config(NAIVE, 0, 1, 1, 256, FED)]
    for dw in (2 * R, 4 * R, 8 * R, 16 * R):
        for nf in (1, 2):
            for cl in (1, 4, 8, 16):
                for th in (256, 512):
                    vs = [FED, FED_BULK] + ([RELAXED] if cl > 1 and th == 512 else [])
                    for v in vs:
                        c = config(MWD, dw, nf, cl, th, v)
                        if p.feasible(c):
                            out.append(c)
    n = ctypes.c_int32()
    check(lib().girih_tune_candidates(p.handle, None, 0, ctypes.byref(n)))
    if n.value:
        arr = (Config * n.value)()
        check(lib().girih_tune_candidates(p.handle, arr, n.value, ctypes.byref(n)))
        out += [c for c in arr if c.variant in (RELAXED_PERSISTENT, OVERLAP_PERSISTENT)
                and c.dw in (2 * R, 4 * R, 8 * R, 16 * R) and c.cluster in (4, 8, 16) and c.zseg == 0]
    return out


def collect(db_path: str, problems, T: int = 16, tol: float = 0.05, max_steps: int = 32, times_path: str | None = None,
            log=print):
    """Exhaustively tune every (stencil, dtype, nx, ny, nz) problem over space(); rows go to db_path."""
    for (stencil, dtype, nx, ny, nz) in problems:
        p = problem_plan(stencil, dtype, nx, ny, nz, T)
        best = TuneRow()
        nm = ctypes.c_int32()
        arr, n = config_array(space(p))
        t0 = time.perf_counter()
        check(lib().girih_tune_exhaustive(p.handle, arr, n, tol, max_steps, db_path.encode(), ctypes.byref(best),
                                          ctypes.byref(nm)))
        dt = time.perf_counter() - t0
        if times_path:
            with open(times_path, "a") as f:
                f.write(f"{stencil},{_dt(dtype)},{nx},{ny},{nz},{nm.value},{dt:.4f},{best.glups:.4f}\n")
        if log:
            log(f"tuned s={stencil} {dtype} {nx}x{ny}x{nz}: {nm.value} candidates in {dt:.1f} s, best "
                f"{best.glups:.1f} GLUP/s {best.cfg}")
        p.close()


def load_db(path: str):
    rows = []
    with open(path) as f:
        for r in csv.reader(f):
            if not r or r[0].startswith("#"):
                continue
            vals = [float(v) for v in r]
            rows.append(dict(zip(FIELDS, vals)))
    return rows


def problem_key(r):
    return (int(r["stencil"]), int(r["dtype"]), int(r["nx"]), int(r["ny"]), int(r["nz"]))


def row_config(r) -> Config:
    return Config(int(r["algo"]), int(r["dw"]), int(r["nf"]), int(r["cluster"]), int(r["threads"]),
                  int(r["variant"]), int(r.get("zseg", 0)))


def features(rows) -> np.ndarray:
    X = np.zeros((len(rows), MLP_FEATURES), dtype=np.float32)
    for i, r in enumerate(rows):
        cfg = row_config(r)
        check(lib().girih_mlp_features(int(r["stencil"]), int(r["dtype"]), int(r["nx"]), int(r["ny"]), int(r["nz"]),
                                       ctypes.byref(cfg), X[i].ctypes.data_as(ctypes.c_void_p)))
    return X


def targets(rows) -> np.ndarray:
    """Per-problem centred log throughput."""
    y = np.array([math.log(max(r["glups"], 1e-6)) for r in rows])
    keys = [problem_key(r) for r in rows]
    for k in set(keys):
        idx = [i for i, kk in enumerate(keys) if kk == k]
        y[idx] -= y[idx].mean()
    return y.astype(np.float32)


def init_params(seed: int = 0) -> np.ndarray:
    """He-uniform initial weights, zero biases (host-side random draw, passed to the kernels)."""
    rng = np.random.default_rng(seed)
    d, h = MLP_FEATURES, 64
    W1 = rng.uniform(-1, 1, (h, d)) * math.sqrt(6.0 / d)
    W2 = rng.uniform(-1, 1, (h, h)) * math.sqrt(6.0 / h)
    W3 = rng.uniform(-1, 1, (1, h)) * math.sqrt(6.0 / h)
    return np.concatenate([W1.ravel(), np.zeros(h), W2.ravel(), np.zeros(h), W3.ravel(), np.zeros(1)]).astype(
        np.float32)


def train(X: np.ndarray, y: np.ndarray, epochs: int = 2000, lr: float = 3e-3, seed: int = 0, log=None):
    """Full-batch Adam on the GPU with the library's kernels; returns (params, loss history)."""
    import torch
    L = lib()
    n, d = X.shape
    npar = L.girih_mlp_num_params(d)
    dev = "cuda"
    P = torch.from_numpy(init_params(seed)).to(dev)
    dX = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(dev)
    dy = torch.from_numpy(np.ascontiguousarray(y, dtype=np.float32)).to(dev)
    g = torch.zeros(npar, device=dev)
    m = torch.zeros(npar, device=dev)
    v = torch.zeros(npar, device=dev)
    loss = torch.zeros(1, device=dev)
    ws = torch.zeros(L.girih_mlp_workspace_floats(n), device=dev)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    hist = []
    for step in range(1, epochs + 1):
        check(L.girih_mlp_backward(ptr(P), ptr(dX), ptr(dy), n, d, ptr(g), ptr(loss), ptr(ws), None))
        check(L.girih_mlp_adam(ptr(P), ptr(g), ptr(m), ptr(v), npar, step, ctypes.c_float(lr), ctypes.c_float(0.9),
                               ctypes.c_float(0.999), ctypes.c_float(1e-8), None))
        if step % 100 == 0 or step == epochs:
            hist.append((step, float(loss.item())))
            if log:
                log(f"epoch {step}: loss {hist[-1][1]:.5f}")
    torch.cuda.synchronize()
    return P.cpu().numpy(), hist


def predict(params: np.ndarray, X: np.ndarray) -> np.ndarray:
    import torch
    L = lib()
    n, d = X.shape
    P = torch.from_numpy(np.ascontiguousarray(params, dtype=np.float32)).cuda()
    dX = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    y = torch.zeros(n, device="cuda")
    ws = torch.zeros(L.girih_mlp_workspace_floats(n), device="cuda")
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    check(L.girih_mlp_forward(ptr(P), ptr(dX), n, d, ptr(y), ptr(ws), None))
    torch.cuda.synchronize()
    return y.cpu().numpy()


def evaluate(rows, scores: np.ndarray, k: int):
    """Per problem: exhaustive best, best of the network's top k, and the measurement-cost ratio."""
    out = []
    keys = [problem_key(r) for r in rows]
    for key in sorted(set(keys)):
        idx = [i for i, kk in enumerate(keys) if kk == key]
        g = np.array([rows[i]["glups"] for i in idx])
        cost = np.array([rows[i]["tune_seconds"] for i in idx])
        top = np.argsort(-scores[idx], kind="stable")[:k]
        out.append({"problem": key, "candidates": len(idx), "exhaustive_best": float(g.max()),
                    "learned_best": float(g[top].max()), "ratio": float(g[top].max() / g.max()),
                    "cost_fraction": float(cost[top].sum() / cost.sum())})
    return out


# domain-sized streams N_D of the code-balance model (Eq. 5) and spatial minimum elements per LUP
_ND = {0: 2, 1: 9, 2: 2, 3: 15, 4: 3, 5: 2, 6: 2}
_SPATIAL = {0: 2, 1: 9, 2: 3, 3: 16, 4: 4, 5: 2, 6: 2}


def model_bytes(r) -> float:
    """Bytes per LUP a candidate moves by the paper's models: the spatial minimum for the naive
    sweep, Eq. 5's code balance B_C for a blocked one."""
    s = int(r["stencil"])
    elem = 8 if int(r["dtype"]) == F64 else 4
    if int(r["algo"]) == NAIVE:
        return float(_SPATIAL[s] * elem)
    return model_code_balance(int(r["dw"]), RADIUS[s], _ND[s], elem)


def baselines(rows, scores: np.ndarray, k: int, draws: int = 2000, seed: int = 7):
    """The network's top k against the methods without it, per problem: the naive sweep alone
    ("always naive"), the k candidates the code-balance model ranks cheapest (ties kept in the
    tuner's order), and k candidates drawn at random (mean over `draws` seeded draws of the best
    of k).  Each method: fraction of the exhaustive best and fraction of the exhaustive tuning
    time spent measuring its candidates."""
    rng = np.random.default_rng(seed)
    out = []
    keys = [problem_key(r) for r in rows]
    for key in sorted(set(keys)):
        idx = [i for i, kk in enumerate(keys) if kk == key]
        g = np.array([rows[i]["glups"] for i in idx])
        cost = np.array([rows[i]["tune_seconds"] for i in idx])
        best, total = g.max(), cost.sum()
        net = np.argsort(-scores[idx], kind="stable")[:k]
        mb = np.array([model_bytes(rows[i]) for i in idx])
        mod = np.argsort(mb, kind="stable")[:k]
        naive = [j for j, i in enumerate(idx) if int(rows[i]["algo"]) == NAIVE]
        kk = min(k, len(idx))
        rnd = [rng.choice(len(idx), kk, replace=False) for _ in range(draws)]
        def method(ratio, cost_s):
            return {"ratio": float(ratio), "cost_fraction": float(cost_s / total), "cost_seconds": float(cost_s)}
        out.append({"problem": key, "candidates": len(idx), "exhaustive_seconds": float(total),
                    "network": method(g[net].max() / best, cost[net].sum()),
                    "model_top_k": method(g[mod].max() / best, cost[mod].sum()),
                    "always_naive": method(g[naive].max() / best, cost[naive].sum()) if naive else None,
                    "random_k": method(np.mean([g[c].max() for c in rnd]) / best,
                                       np.mean([cost[c].sum() for c in rnd]))})
    return out


def summarize(res):
    """Per method of baselines(): worst and mean fraction of the exhaustive best, problems at 95 %
    of it, the mean over problems of the fraction of exhaustive tuning time spent measuring, and
    that fraction over all problems together (the time the method spends tuning the whole set;
    problems with a handful of candidates make the per-problem mean large for any k)."""
    out = {}
    for m in ("network", "model_top_k", "always_naive", "random_k"):
        rows = [r for r in res if r.get(m)]
        if not rows:
            continue
        vals = [r[m] for r in rows]
        out[m] = {"worst_ratio": min(v["ratio"] for v in vals), "mean_ratio": float(np.mean([v["ratio"] for v in vals])),
                  "problems_at_95pct": sum(v["ratio"] >= 0.95 for v in vals), "problems": len(vals),
                  "mean_cost_fraction": float(np.mean([v["cost_fraction"] for v in vals])),
                  "total_cost_fraction": float(sum(v["cost_seconds"] for v in vals) /
                                               sum(r["exhaustive_seconds"] for r in rows))}
    return out


def reevaluate(out_dir: str, k: int = 5):
    """Recompute the offline parts of an experiment's report (the network's top k, the methods
    without it, over all candidates and over the blocked ones) from its database and trained
    parameters, keeping the live measurements; no GPU needed."""
    import json
    rp = os.path.join(out_dir, "report.json")
    rep = json.load(open(rp))
    rows = load_db(os.path.join(out_dir, "tune_db.csv"))
    params = np.load(os.path.join(out_dir, "mlp_params.npy"))
    held = {tuple(GRIDS[i]) for i in HELD_OUT}
    test_rows = [r for r in rows if (int(r["nx"]), int(r["ny"]), int(r["nz"])) in held]
    scores = predict(params, features(test_rows))
    bl = [i for i, r in enumerate(test_rows) if int(r["algo"]) == MWD]
    cmp_all = baselines(test_rows, scores, k)
    cmp_blocked = baselines([test_rows[i] for i in bl], scores[bl], k)
    rep.update({"offline": evaluate(test_rows, scores, k), "baselines": cmp_all,
                "baselines_summary": summarize(cmp_all), "blocked_only": cmp_blocked,
                "blocked_only_summary": summarize(cmp_blocked)})
    with open(rp, "w") as f:
        json.dump(rep, f, indent=1)
    return rep


def tune(p, params: np.ndarray, k: int = 5, tol: float = 0.05, max_steps: int = 32):
    """Live learned tuning of a plan: returns (TuneRow, measured count, seconds)."""
    import torch
    P = torch.from_numpy(np.ascontiguousarray(params, dtype=np.float32)).cuda()
    best = TuneRow()
    nm = ctypes.c_int32()
    arr, n = config_array(space(p))
    t0 = time.perf_counter()
    check(lib().girih_tune_learned(p.handle, ctypes.c_void_p(P.data_ptr()), arr, n, k, tol, max_steps,
                                   ctypes.byref(best), ctypes.byref(nm)))
    return best, nm.value, time.perf_counter() - t0


def experiment(out_dir: str, stencils=(0, 1, 2, 3), dtypes=("f64", "f32"), grids=None, T: int = 16,
               tol: float = 0.05, max_steps: int = 32, k: int = 5, epochs: int = 3000, live: bool = True,
               log=print):
    """The learned-tuner experiment: exhaustive timings on all grids, network trained on the
    non-held-out grids, regret and tuning-time fraction on the held-out grids (offline from the
    database, and live with girih_tune_learned)."""
    import json
    grids = grids or GRIDS
    os.makedirs(out_dir, exist_ok=True)
    db = os.path.join(out_dir, "tune_db.csv")
    times = os.path.join(out_dir, "tune_times.csv")
    problems = [(s, d, *g) for s in stencils for d in dtypes for g in grids]
    done = set()
    if os.path.exists(db):
        done = {problem_key(r) for r in load_db(db)}
    todo = [p for p in problems if (p[0], _dt(p[1]), p[2], p[3], p[4]) not in done]
    collect(db, todo, T=T, tol=tol, max_steps=max_steps, times_path=times, log=log)
    rows = load_db(db)
    held = {tuple(grids[i]) for i in HELD_OUT if i < len(grids)}
    train_rows = [r for r in rows if (int(r["nx"]), int(r["ny"]), int(r["nz"])) not in held]
    test_rows = [r for r in rows if (int(r["nx"]), int(r["ny"]), int(r["nz"])) in held]
    Xtr, ytr = features(train_rows), targets(train_rows)
    t0 = time.perf_counter()
    params, hist = train(Xtr, ytr, epochs=epochs, log=None)
    train_s = time.perf_counter() - t0
    np.save(os.path.join(out_dir, "mlp_params.npy"), params)
    res = evaluate(test_rows, predict(params, features(test_rows)), k) if test_rows else []
    # the method without the network: the plan's model-based default configuration
    base = []
    for key in sorted({problem_key(r) for r in test_rows}):
        s, d, nx, ny, nz = key
        p = problem_plan(s, d, nx, ny, nz, T)
        dflt = p.config.as_dict()
        rs = [r for r in test_rows if problem_key(r) == key]
        best = max(r["glups"] for r in rs)
        match = [r["glups"] for r in rs if row_config(r).as_dict() == dflt]
        base.append({"problem": key, "default_ratio": (match[0] / best) if match else None})
        p.close()
    live_res = []
    if live:
        for key in sorted({problem_key(r) for r in test_rows}):
            s, d, nx, ny, nz = key
            rs = [r for r in test_rows if problem_key(r) == key]
            p = problem_plan(s, d, nx, ny, nz, T)
            row, nm, secs = tune(p, params, k=k, tol=tol, max_steps=max_steps)
            exh_secs = sum(r["tune_seconds"] for r in rs)
            live_res.append({"problem": key, "learned_glups": row.glups, "measured": nm, "seconds": secs,
                             "exhaustive_best": max(r["glups"] for r in rs), "exhaustive_seconds": exh_secs})
            p.close()
    test_scores = predict(params, features(test_rows)) if test_rows else np.zeros(0)
    cmp_all = baselines(test_rows, test_scores, k) if test_rows else []
    # the blocked sub-space alone (the winner varies with the problem there): the network ranks
    # only the blocked candidates
    bl = [i for i, r in enumerate(test_rows) if int(r["algo"]) == MWD]
    blocked_rows = [test_rows[i] for i in bl]
    cmp_blocked = baselines(blocked_rows, test_scores[bl], k) if bl else []
    report = {"train_problems": len({problem_key(r) for r in train_rows}), "train_rows": len(train_rows),
              "train_seconds": train_s, "loss_history": hist, "k": k, "offline": res, "default": base,
              "live": live_res, "baselines": cmp_all, "baselines_summary": summarize(cmp_all),
              "blocked_only": cmp_blocked, "blocked_only_summary": summarize(cmp_blocked)}
    with open(os.path.join(out_dir, "report.json"), "w") as f:
        json.dump(report, f, indent=1)
    return report


def unseen(out_dir: str, params_path: str, stencils=(4, 5, 6), dtypes=("f64", "f32"), grids=None, T: int = 16,
           tol: float = 0.05, max_steps: int = 32, k: int = 5, log=print):
    """The trained network on stencils it never saw (the 25-point stencil with the factor grid,
    the 27-point box stencil, red-black Gauss-Seidel): exhaustive timings as the judge, the
    network's top k offline and live, regret and measurement-time fraction."""
    import json
    grids = grids or [GRIDS[i] for i in HELD_OUT]
    os.makedirs(out_dir, exist_ok=True)
    db = os.path.join(out_dir, "unseen_db.csv")
    times = os.path.join(out_dir, "unseen_times.csv")
    problems = [(s, d, *g) for s in stencils for d in dtypes for g in grids]
    done = {problem_key(r) for r in load_db(db)} if os.path.exists(db) else set()
    todo = [q for q in problems if (q[0], _dt(q[1]), q[2], q[3], q[4]) not in done]
    collect(db, todo, T=T, tol=tol, max_steps=max_steps, times_path=times, log=log)
    rows = load_db(db)
    params = np.load(params_path)
    res = evaluate(rows, predict(params, features(rows)), k)
    live_res = []
    for key in sorted({problem_key(r) for r in rows}):
        s, d, nx, ny, nz = key
        rs = [r for r in rows if problem_key(r) == key]
        p = problem_plan(s, d, nx, ny, nz, T)
        row, nm, secs = tune(p, params, k=k, tol=tol, max_steps=max_steps)
        live_res.append({"problem": key, "learned_glups": row.glups, "learned_config": row.cfg.as_dict(),
                         "measured": nm, "seconds": secs, "exhaustive_best": max(r["glups"] for r in rs),
                         "exhaustive_seconds": sum(r["tune_seconds"] for r in rs)})
        p.close()
    report = {"params": os.path.basename(params_path), "k": k, "offline": res, "live": live_res}
    with open(os.path.join(out_dir, "report_unseen.json"), "w") as f:
        json.dump(report, f, indent=1)
    return report


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="learned-tuner experiment (exhaustive DB, train, evaluate)")
    ap.add_argument("out_dir")
    ap.add_argument("--stencils", default="0,1,2,3")
    ap.add_argument("--dtypes", default="f64,f32")
    ap.add_argument("--grids", default="", help="indices into GRIDS, e.g. 0,1,2 (default all 12)")
    ap.add_argument("--T", type=int, default=16)
    ap.add_argument("--tol", type=float, default=0.05)
    ap.add_argument("--max-steps", type=int, default=32)
    ap.add_argument("--k", type=int, default=5)
    ap.add_argument("--epochs", type=int, default=3000)
    ap.add_argument("--no-live", action="store_true")
    ap.add_argument("--unseen-from", default="", help="trained parameters (.npy): evaluate them on --stencils "
                    "instead of training (stencils the network never saw)")
    ap.add_argument("--reevaluate", action="store_true", help="recompute the offline evaluation of OUT_DIR's "
                    "report from its database and parameters (no GPU)")
    a = ap.parse_args()
    if a.reevaluate:
        rep = reevaluate(a.out_dir, a.k)
        print(json.dumps({k: rep[k] for k in ("baselines_summary", "blocked_only_summary")}, indent=1))
        raise SystemExit(0)
    from . import build as _b
    _b.build()
    gl = [GRIDS[int(i)] for i in a.grids.split(",")] if a.grids else None
    if a.unseen_from:
        rep = unseen(a.out_dir, a.unseen_from, tuple(int(s) for s in a.stencils.split(",")), tuple(a.dtypes.split(",")),
                     gl, a.T, a.tol, a.max_steps, a.k)
        print(json.dumps(rep, indent=1))
        raise SystemExit(0)
    rep = experiment(a.out_dir, tuple(int(s) for s in a.stencils.split(",")), tuple(a.dtypes.split(",")), gl, a.T,
                     a.tol, a.max_steps, a.k, a.epochs, not a.no_live)
    print(json.dumps({k: rep[k] for k in ("train_problems", "train_rows", "train_seconds", "offline", "default",
                                          "live", "baselines_summary", "blocked_only_summary")}, indent=1))
