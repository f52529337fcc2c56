"""Arithmetic peaks of the current GPU, measured: the FMA rate in FP64 and FP32.

    python -m paper_1510_04995_gb300.peaks [--repeats N]

Prints one JSON line: the device's SM count and maximum SM clock (as the runtime reports them),
the FMA instructions per second of girih_measure_fma_rate for each dtype (best of N launches),
the per-SM, per-clock rates they imply at the maximum clock, and the SM clocks nvidia-smi sampled
while the launches ran.  The FP64 rate is the roofline of the FP64 sweeps (7 or 28 explicitly
rounded FP64 instructions per update, at most one per FMA slot).
"""
from __future__ import annotations

import argparse
import json
import subprocess

from . import build, measure_fma_rate


def sample_clocks(fn):
    """Run fn() while nvidia-smi samples the SM clock every 50 ms; (fn's result, samples in MHz)."""
    p = None
    try:
        p = subprocess.Popen(["nvidia-smi", "-i", "0", "--query-gpu=clocks.sm", "--format=csv,noheader,nounits",
                              "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except Exception:
        p = None
    try:
        res = fn()
    finally:
        out = ""
        if p:
            p.terminate()
            try:
                out, _ = p.communicate(timeout=5)
            except Exception:
                p.kill()
    mhz = []
    for line in out.splitlines():
        try:
            mhz.append(float(line.strip()))
        except ValueError:
            pass
    return res, mhz


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--repeats", type=int, default=5)
    a = ap.parse_args()
    import torch
    build.build()
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    max_mhz = None
    try:
        max_mhz = float(subprocess.run(["nvidia-smi", "-i", "0", "--query-gpu=clocks.max.sm",
                                        "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                       timeout=10).stdout.strip())
    except Exception:
        pass
    line = {"device": props.name, "sms": sms, "sm_max_mhz": max_mhz}
    for dt in ("f64", "f32"):
        measure_fma_rate(dt)  # warm-up

        def run():
            return max(measure_fma_rate(dt) for _ in range(a.repeats))

        (rate, secs), mhz = sample_clocks(run)
        line[dt] = {"fma_per_s": rate, "seconds_per_launch": secs,
                    "per_sm_per_clock": (rate / sms / (max_mhz * 1e6)) if max_mhz else None,
                    "sm_mhz_samples": mhz}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
