"""Consistency of the committed workload records (no GPU): every benchmark workload has a tuned
entry whose configurations are well formed for its stencil, the tuning script and the benchmark
agree on the workloads, and the measured bytes per update the benchmark cites come from
profile summaries that exist."""
import json
import os

import bench
from paper_1510_04995_gb300 import inputs, tune_workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_tuner_and_bench_share_the_workloads():
    assert tune_workloads.WORKLOADS == bench.WORKLOADS
    for name, (s, dt, nx, ny, nz, T) in bench.WORKLOADS.items():
        assert name.startswith(inputs.STENCIL_NAMES[s] + "_" + dt), name
        assert T % 2 == 0  # no exchange kernel inside the timed region
        assert tune_workloads.aligned_ldx(s, dt, nx) * (8 if dt == "f64" else 4) % 16 == 0


def test_tuned_entries_are_well_formed():
    tuned = json.load(open(os.path.join(ROOT, "paper_1510_04995_gb300", "tuned_configs.json")))
    assert set(tuned) == set(bench.WORKLOADS)
    for name, e in tuned.items():
        s = bench.WORKLOADS[name][0]
        R = inputs.RADIUS[s]
        best, blocked = bench._tuned(name)
        assert best == e["best"] and blocked == e["blocked"]
        assert best["algo"] in (0, 1) and e["best_glups"] > 0
        assert blocked["algo"] == 1 and e["blocked_glups"] > 0
        assert blocked["dw"] % (2 * R) == 0 and 1 <= blocked["nf"] <= 4
        assert blocked["cluster"] in (1, 2, 4, 8, 16) and blocked["threads"] % 32 == 0
        assert e["best_glups"] >= e["blocked_glups"] * (1 - 1e-6)  # the database rounds to 6 decimals


def test_measured_bytes_cite_existing_profiles():
    """Every cited DRAM byte count is printed in its profile summary.  The naive sweep moves the
    spatial minimum (u in and out, the coefficient grids in); a blocked sweep lies within 15 % of
    the Eq. 5 code balance of its diamond width."""
    import paper_1510_04995_gb300 as girih
    for (kernel, s, dt), (bpl, path) in bench.MEASURED_BYTES_PER_LUP.items():
        assert os.path.exists(os.path.join(ROOT, path)), path
        text = open(os.path.join(ROOT, path)).read()
        assert f"{bpl:.2f}" in text or f"{bpl}" in text, (path, bpl)
        elem = 8 if dt == "f64" else 4
        if kernel[0] == "naive":
            minimum = bench.SPATIAL_ELEMS[s] * elem
            assert 0.9 * minimum <= bpl <= 1.1 * minimum
        else:
            _, variant, dw, cluster, threads = kernel
            assert dw % (2 * inputs.RADIUS[s]) == 0 and cluster in (1, 2, 4, 8, 16) and threads % 32 == 0
            bc = girih.model_code_balance(dw, inputs.RADIUS[s], bench.ND[s], elem)
            assert 0.85 * bc <= bpl <= 1.15 * bc, (kernel, bpl, bc)
