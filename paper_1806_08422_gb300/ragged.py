"""Ragged-batch throughput: many instances of different sizes annealed in one
persistent tensor-core launch, captured once as a CUDA graph and replayed.

Workload (the shape of the paper's instance sweeps, Sec. III): `count` instances with
N uniform in [n_lo, n_hi], the first half SK +-1 and the second half MAX-CUT on
G(N, 0.5) with J = +1 per edge, `replicas` replicas each, t_f steps of the default
schedule, sigma = alpha = 0.15, BF16 J and S with FP32 accumulation, energies of the
sign vectors formed in the kernel.  Tile widths per instance come from the
autotuner (`--tiles auto`), the default pick, or are 64 throughout.

    python -m paper_1806_08422_gb300.ragged [--count 512] [--replicas 64] [--reps 5]

Prints one JSON line: spin-updates/s, the tensor work rate (2 n^2 R per step and
instance at the 128-padded size the kernel computes, and at the unpadded size) and
its fraction of the measured BF16 peaks (burst: the launch is timed on its own;
sustained beside it), and the memory view: the BF16 couplings the kernel reads
(padded), the HBM bytes the batch needs at least (J once plus the outputs) and the
rate at which the product consumes J (t_f passes over it, which would bound the
batch at the measured HBM bandwidth if J were re-read from HBM every step; the
kernel keeps each running tile's J block in L2 instead).  This module only drives
the C ABI; all annealing runs in the library's kernels.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import instances as inst
from . import nmfa

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def measured_peaks():
    """(burst BF16 TFLOP/s, sustained BF16 TFLOP/s, HBM GB/s, source)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return (float(d.get("bf16_tflops", d.get("bf16_tflops_sustained"))),
                float(d.get("bf16_tflops_sustained", d.get("bf16_tflops"))), float(d["hbm_gbs"]), "measured")
    except Exception:
        return 1900.0, 1700.0, 6800.0, "fallback"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=512)
    ap.add_argument("--n-lo", type=int, default=16)
    ap.add_argument("--n-hi", type=int, default=1000)
    ap.add_argument("--replicas", type=int, default=64)
    ap.add_argument("--t-f", type=int, default=1000)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--tiles", default="auto", choices=["auto", "pick", "64"],
                    help="tile widths: autotuned, the default pick (64 for <= 64 replicas), or 64 throughout")
    args = ap.parse_args()

    import torch

    dev = torch.device("cuda", 0)
    mix = inst.ragged_batch(args.count, args.n_lo, args.n_hi, seed=args.seed)
    t0 = time.perf_counter()
    probs = [nmfa.Problem(J, precision="bf16") for _, _, J in mix]
    t_create = time.perf_counter() - t0
    T = torch.as_tensor(inst.schedule(args.t_f), device=dev)
    R = args.replicas
    energies = [torch.empty(R, dtype=torch.int64, device=dev) for _ in mix]
    jobs = [nmfa.make_job(T, 0.15, 0.15, R, seed=args.seed, stream_id=k, energy_i64=e)
            for k, e in enumerate(energies)]
    t0 = time.perf_counter()
    opts = nmfa.NMFA_BATCH_GRAPH | {"auto": nmfa.NMFA_BATCH_AUTOTUNE, "pick": 0, "64": nmfa.NMFA_BATCH_BN64}[args.tiles]
    b = nmfa.nmfa_batch_create([p.handle for p in probs], jobs, opts)
    t_batch = time.perf_counter() - t0
    info = nmfa.nmfa_batch_info(b)
    stream = torch.cuda.Stream()
    nmfa.nmfa_batch_launch(b, stream)
    nmfa.nmfa_batch_sync(b)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for _ in range(args.reps):
        ev0.record(stream)
        nmfa.nmfa_batch_launch(b, stream)
        ev1.record(stream)
        nmfa.nmfa_batch_sync(b)
        stream.synchronize()
        ms.append(ev0.elapsed_time(ev1))
    nmfa.nmfa_batch_destroy(b)
    ns = np.array([n for _, n, _ in mix], dtype=np.float64)
    npad = np.ceil(ns / 128.0) * 128.0
    per = float(np.median(ms)) / 1e3
    units = float(ns.sum()) * R * args.t_f
    flops_pad = 2.0 * float((npad ** 2).sum()) * R * (args.t_f + 1)
    flops = 2.0 * float((ns ** 2).sum()) * R * args.t_f
    burst, sustained, hbm, kind = measured_peaks()
    j_bytes = 2.0 * float((npad ** 2).sum())                  # BF16 J at the padded sizes
    out_bytes = float(ns.sum()) * R + 8.0 * R * len(ns)     # int8 signs + int64 energies
    e0 = energies[0].cpu().numpy()
    out = {
        "workload": "%d instances, N uniform in [%d, %d] (half SK +-1, half G(N,0.5) max-cut), %d replicas each, "
                    "t_f=%d, BF16 J/S, FP32 accumulation, one persistent launch replayed from a CUDA graph"
                    % (args.count, args.n_lo, args.n_hi, R, args.t_f),
        "ms_per_batch": float(np.median(ms)), "ms_all": ms,
        "spin_updates_per_s": units / per,
        "tensor_tflops_padded": flops_pad / per / 1e12,
        "tensor_tflops_unpadded": flops / per / 1e12,
        "frac_of_burst_bf16_padded": flops_pad / per / 1e12 / burst,
        "frac_of_sustained_bf16_padded": flops_pad / per / 1e12 / sustained,
        "peak_tflops_burst": burst, "peak_tflops_sustained": sustained, "peak_source": kind,
        "j_bytes_bf16_padded": j_bytes,
        "hbm_bytes_algorithmic": j_bytes + out_bytes,
        "hbm_frac_algorithmic": (j_bytes + out_bytes) / per / 1e9 / hbm,
        "j_consumption_gbs": j_bytes * (args.t_f + 1) / per / 1e9,
        "j_consumption_over_hbm_peak": j_bytes * (args.t_f + 1) / per / 1e9 / hbm,
        "hbm_gbs_peak": hbm,
        "tiles": args.tiles, "grid": info["grid"], "groups": info["groups"], "workspace_bytes": info["workspace_bytes"],
        "host_create_s": t_create, "batch_create_s": t_batch,
        "check_first_instance_min_energy": int(e0.min()),
    }
    for p in probs:
        p.close()
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
