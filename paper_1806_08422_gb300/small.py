"""Time per run at 100 spins: the plain FP64 configuration (SK N = 100, 100 replicas,
t_f = 1000) and the per-run cost of every path at the size the paper times (Sec. III
quotes 12.3 us per NMFA run of a 100-spin dense MAX-CUT instance on a GTX 1080 Ti,
against 1.6 ms and 5 ms per run for the two coherent Ising machines).

For each instance (SK +-1, and MAX-CUT on G(100, 0.5) with J = +1 per edge) and each
path (FP64 and FP32 CUDA-core kernels, BF16 tensor kernel) the driver runs R replicas
of t_f steps in one launch on device buffers and reports the kernel time per launch,
the time per replica-run (kernel time / R), spin-updates/s, and the arithmetic rate
against the path's measured peak (FP64 or FP32 FMA from nmfa_measure_alu_peaks, BF16
from MEASURED_PEAKS.json; the tensor path computes the 128-padded product).  The
paper's figure is context from other hardware, not a target.

    python -m paper_1806_08422_gb300.small [--t-f 1000] [--reps 5]

Prints one JSON line.  This module only drives the C ABI.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics

import numpy as np

from . import instances as inst
from . import nmfa

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N = 100


def _bf16_burst():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--t-f", type=int, default=1000)
    ap.add_argument("--reps", type=int, default=5)
    args = ap.parse_args()

    import torch

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream()
    T = torch.as_tensor(inst.schedule(args.t_f), device=dev)
    alu = nmfa.nmfa_measure_alu_peaks(stream)
    bf16, bf16_src = _bf16_burst()
    n_pad = 128
    # (precision, replicas per launch): the plain FP64 configuration, then the other
    # paths at replica counts that fill the GPU
    plans = [("fp64", 100), ("fp64", 4096), ("fp32", 4096), ("bf16", 16384)]
    out = {"workload": "N=%d, t_f=%d, sigma=alpha=0.15, default schedule; SK +-1 and G(%d,0.5) max-cut" % (N, args.t_f, N),
           "paper_context": {"us_per_run": 12.3, "hardware": "GTX 1080 Ti", "workload": "N=100 dense MAX-CUT",
                             "cim_us_per_run": {"Stanford": 1600.0, "NTT": 5000.0}},
           "peaks": {"fp64_fma_tflops": alu["fp64_fma_tflops"], "fp32_fma_tflops": alu["fp32_fma_tflops"],
                     "bf16_tflops_burst": bf16, "bf16_source": bf16_src},
           "runs": []}
    for kind, J in (("sk", inst.sk(N, 0)), ("gnp_maxcut", inst.gnp_maxcut(N, 0.5, 0))):
        for prec, R in plans:
            p = nmfa.Problem(J, precision=prec)
            signs = torch.empty((R, N), dtype=torch.int8, device=dev)
            e64 = torch.empty(R, dtype=torch.int64, device=dev)
            nmfa.nmfa_profile_enable(p.handle, True)
            ms = []
            for i in range(args.reps + 1):
                p.run_device(T, 0.15, 0.15, R, seed=0, stream_id=i, signs=signs, energy_i64=e64, stream=stream)
                p.sync()
                if i > 0:
                    ms.append(nmfa.nmfa_last_kernel_ms(p.handle))
            k = statistics.median(ms)
            n_eff = n_pad if prec == "bf16" else N
            tflops = 2.0 * n_eff * n_eff * R * args.t_f / (k / 1e3) / 1e12
            peak = {"fp64": alu["fp64_fma_tflops"], "fp32": alu["fp32_fma_tflops"], "bf16": bf16}[prec]
            e = e64.cpu().numpy()
            out["runs"].append({
                "instance": kind, "precision": prec, "replicas": R, "kernel_ms": k,
                "us_per_replica_run": 1e3 * k / R,
                "spin_updates_per_s": N * R * args.t_f / (k / 1e3),
                "tflops": tflops, "frac_of_peak": tflops / peak,
                "min_energy": int(e.min()), "mean_energy": float(e.mean()),
            })
            p.close()
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
