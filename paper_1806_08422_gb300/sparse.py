"""Sparse MAX-CUT throughput on the CSR path (CUDA cores, FP32 or FP64).

Workload (the sparse instances of the paper's Sec. III / Fig. 3-4 classes): Moebius
ladders with N in {100, 400, 1000, 2000} (ring plus antipodal chords, J = +1 per
edge) and a random 3-regular graph with N = 2000, stored as CSR with int8 values,
512 replicas each, t_f = 1000 steps of the default schedule, sigma = alpha = 0.15,
energies of the sign vectors included.

    python -m paper_1806_08422_gb300.sparse [--replicas 512] [--reps 3] [--precision fp32]

Prints one JSON line per instance: spin-updates/s (device buffers, CUDA events around
the C call) and the kernel time.  This module only drives the C ABI; all annealing
runs in the library's kernels.
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import instances as inst
from . import nmfa


def instances():
    out = [("moebius", n, inst.moebius(n)) for n in (100, 400, 1000, 2000)]
    out.append(("regular3", 2000, inst.regular3(2000, seed=5)))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--replicas", type=int, default=512)
    ap.add_argument("--t-f", type=int, default=1000)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--rc", type=int, default=0, help="replicas per CTA (0: the library's pick)")
    args = ap.parse_args()

    import torch

    dev = torch.device("cuda", 0)
    T = torch.as_tensor(inst.schedule(args.t_f), device=dev)
    R = args.replicas
    for kind, n, J in instances():
        row_ptr, col, val = inst.to_csr(J)
        p = nmfa.Problem(csr=(row_ptr, col, val), n=n, precision=args.precision)
        if args.rc:
            nmfa.nmfa_tune_replicas_per_cta(p.handle, args.rc)
        signs = torch.empty((R, n), dtype=torch.int8, device=dev)
        e = torch.empty(R, dtype=torch.int64, device=dev)
        stream = torch.cuda.current_stream()
        nmfa.nmfa_profile_enable(p.handle, True)
        p.run_device(T, 0.15, 0.15, R, signs=signs, energy_i64=e, stream=stream)
        p.sync()
        ms, kms = [], []
        for _ in range(args.reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            p.run_device(T, 0.15, 0.15, R, signs=signs, energy_i64=e, stream=stream)
            b.record(stream)
            p.sync()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
            kms.append(nmfa.nmfa_last_kernel_ms(p.handle))
        per = float(np.median(ms)) / 1e3
        units = n * R * args.t_f
        print(json.dumps({"instance": kind, "n": n, "nnz": int(len(col)), "replicas": R, "t_f": args.t_f,
                          "precision": args.precision, "rc": args.rc, "ms_per_run": float(np.median(ms)),
                          "kernel_ms": float(np.median(kms)), "spin_updates_per_s": units / per,
                          "min_energy": int(e.min().item())}), flush=True)
        p.close()


if __name__ == "__main__":
    main()
