"""Time the annealing kernels on single SK +-1 instances across sizes and storage of J.

For each (N, R) and each storage of the couplings (BF16, or FP8-E4M3 widened to BF16
in the kernel, on the tensor path; or FP32 on the CUDA-core path) the driver runs R
replicas of Algorithm 1 for t_f steps in one persistent launch on device buffers and
reports the launch time per step, the tile plan, the algorithmic rate 2 N^2 R per
product against the burst BF16 peak of MEASURED_PEAKS.json (tensor path) or the
measured FP32 FMA rate (FP32 path), and the best energy.  Both tensor storages of the
same instance give bit-identical runs, so their energies must agree.

    python -m paper_1806_08422_gb300.sizes [--sizes 8192:512,2000:1024] [--t-f 200]
                                           [--storage bf16,bf16_fp8j,fp32] [--reps 3] [--options 0]

Prints one JSON line.  This module only drives the C ABI.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics

from . import instances as inst
from . import nmfa

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def burst_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except Exception:
        return 1900.0


def time_one(J, R, t_f, storage, reps, options=0):
    import torch
    dev = torch.device("cuda", 0)
    n = J.shape[0]
    p = nmfa.Problem(J, precision=storage)
    T = torch.as_tensor(inst.schedule(t_f), device=dev)
    s = torch.empty((R, n), dtype=torch.int8, device=dev)
    e = torch.empty(R, dtype=torch.int64, device=dev)
    st = torch.cuda.Stream()
    # FP8 storage: the kernel's own widening (batches would widen n <= 4096 once)
    if storage == "bf16_fp8j":
        options |= nmfa.NMFA_BATCH_FP8_IN_KERNEL
    b = nmfa.nmfa_batch_create([p.handle], [nmfa.make_job(T, 0.15, 0.15, R, signs=s, energy_i64=e)], options)
    try:
        nmfa.nmfa_batch_launch(b, st)  # warm-up
        nmfa.nmfa_batch_sync(b)
        ms = []
        for _ in range(reps):
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            nmfa.nmfa_batch_launch(b, st)
            z.record(st)
            nmfa.nmfa_batch_sync(b)
            st.synchronize()
            ms.append(a.elapsed_time(z))
        plan = nmfa.nmfa_batch_plan(b)
    finally:
        nmfa.nmfa_batch_destroy(b)
        info = p.info()
        p.close()
    med = statistics.median(ms)
    return {"ms_per_launch": med, "us_per_step": 1e3 * med / t_f, "plan": plan,
            "tflops": 2.0 * n * n * R * (t_f + 1) / (med * 1e-3) / 1e12,
            "min_energy": int(e.min().item()), "device_bytes": info["device_bytes"]}


def time_fp32(J, R, t_f, reps):
    """The FP32 CUDA-core path (one cooperative launch per run); the launch time is
    taken by the library's profile events around the annealing kernel."""
    import torch
    dev = torch.device("cuda", 0)
    n = J.shape[0]
    p = nmfa.Problem(J, precision="fp32")
    T = torch.as_tensor(inst.schedule(t_f), device=dev)
    s = torch.empty((R, n), dtype=torch.int8, device=dev)
    e = torch.empty(R, dtype=torch.int64, device=dev)
    st = torch.cuda.Stream()
    nmfa.nmfa_profile_enable(p.handle, True)
    try:
        p.run_device(T, 0.15, 0.15, R, signs=s, energy_i64=e, stream=st)  # warm-up
        p.sync()
        ms = []
        for _ in range(reps):
            p.run_device(T, 0.15, 0.15, R, signs=s, energy_i64=e, stream=st)
            p.sync()
            ms.append(nmfa.nmfa_last_kernel_ms(p.handle))
        info = p.info()
    finally:
        p.close()
    med = statistics.median(ms)
    return {"ms_per_launch": med, "us_per_step": 1e3 * med / t_f, "plan": "FP32 CUDA-core tiles",
            "tflops": 2.0 * n * n * R * t_f / (med * 1e-3) / 1e12,
            "min_energy": int(e.min().item()), "device_bytes": info["device_bytes"]}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--sizes", default="8192:512,2000:1024")
    ap.add_argument("--t-f", type=int, default=200)
    ap.add_argument("--storage", default="bf16,bf16_fp8j")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--options", type=int, default=0,
                    help="nmfa_batch_create options, e.g. 16 / 64 to force 128 / 256 replicas per tile")
    args = ap.parse_args()
    peak = burst_peak()
    storages = args.storage.split(",")
    fp32_peak = None
    if "fp32" in storages:
        fp32_peak = nmfa.nmfa_measure_alu_peaks()["fp32_fma_tflops"]
    out = []
    for item in args.sizes.split(","):
        n, R = (int(x) for x in item.split(":"))
        J = inst.sk(n, args.seed)
        row = {"n": n, "replicas": R}
        for storage in storages:
            if storage == "fp32":
                r = time_fp32(J, R, args.t_f, args.reps)
                r["frac_of_fp32_fma"] = r["tflops"] / fp32_peak
            else:
                r = time_one(J, R, args.t_f, storage, args.reps, args.options)
                r["frac_of_burst_bf16"] = r["tflops"] / peak
            row[storage] = r
        out.append(row)
    print(json.dumps({"t_f": args.t_f, "options": args.options, "burst_bf16_tflops": peak,
                      "fp32_fma_tflops": fp32_peak, "runs": out}))


if __name__ == "__main__":
    main()
