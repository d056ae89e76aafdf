"""Serving benchmark driver: a Poisson stream of NMFA requests through the library's
server (continuous batching on the tensor path) and, for comparison, through the
plain FP32 per-instance path in arrival order (FIFO, one request at a time).

    python -m paper_1806_08422_gb300.serve [--rate 200] [--duration 1.0] [--n-hi 8192]

Requests follow the serving workload shape: exponential inter-arrival gaps, N
log-uniform in [n_lo, n_hi] (rounded to one of 16 log-spaced sizes so that a pool of
pre-generated instances can serve the stream), SK +-1 or G(N, 0.5) MAX-CUT with
equal probability, replicas uniform over {64, 128, 256, 512, 1024}, t_f = 1000, the
default schedule, sigma = alpha = 0.15.  A request succeeds when a replica's energy
reaches its target; the target is an energy density the default schedule reaches
with high probability: H <= -0.70 N^1.5 (SK) and H <= -0.34 N^1.5 (G(N, 0.5)).
Time-to-target = completion of the first successful run - arrival.  This module only
drives the C ABI; all annealing runs in the library's kernels.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import instances as inst
from . import nmfa

TARGET_DENSITY = {"sk": -0.70, "gnp": -0.34}


def target_energy(kind: str, n: int) -> float:
    return TARGET_DENSITY[kind] * n ** 1.5


def size_buckets(n_lo: int, n_hi: int, count: int = 16):
    return sorted({int(round(x)) for x in np.geomspace(n_lo, n_hi, count)})


def make_stream(rate_hz, duration_s, n_lo=64, n_hi=8192, seed=0):
    count = max(1, int(round(rate_hz * duration_s)))
    reqs = inst.poisson_requests(count, rate_hz, n_lo, n_hi, seed=seed)
    buckets = np.array(size_buckets(n_lo, n_hi))
    for r in reqs:
        r["n"] = int(buckets[np.argmin(np.abs(np.log(buckets) - math.log(r["n"])))])
    return reqs


class InstancePool:
    """One seeded instance per (kind, size); J in float64 as the C ABI takes it."""

    def __init__(self):
        self.cache = {}

    def get(self, kind, n):
        key = (kind, n)
        if key not in self.cache:
            self.cache[key] = inst.make_instance(kind, n, seed=1000 + n)
        return self.cache[key]


def percentile(xs, q):
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q)) if len(xs) else None


def run_server(reqs, pool, t_f=1000, precision="bf16_fp8j", max_inflight=2, max_attempts=4, timeout_s=600.0):
    T = inst.schedule(t_f)
    srv = nmfa.nmfa_server_create(0, max_inflight, max_attempts)
    tickets = []
    t0 = time.perf_counter()
    for r in reqs:
        delay = r["arrival"] - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        J = pool.get(r["kind"], r["n"])
        tickets.append(nmfa.nmfa_server_submit(srv, J, T, r["replicas"], target_energy(r["kind"], r["n"]),
                                               precision=precision, seed=r["seed"]))
    nmfa.nmfa_server_drain(srv, timeout_s)
    wall = time.perf_counter() - t0
    res = [nmfa.nmfa_server_poll(srv, t) for t in tickets]
    stats = nmfa.nmfa_server_stats(srv)
    nmfa.nmfa_server_destroy(srv)
    ttt = [x["time_to_target"] for x in res if x["success"]]
    spin = sum(x["spin_updates"] for x in res)
    return {"requests": len(res), "succeeded": len(ttt), "p50_ttt_s": percentile(ttt, 50),
            "p99_ttt_s": percentile(ttt, 99), "spin_updates_per_s": spin / wall, "wall_s": wall,
            "launches": stats["launches"], "batches_reused": stats["batches_reused"], "mean_attempts": float(np.mean([x["attempts"] for x in res])),
            "errors": sum(1 for x in res if x["state"] < 0)}


def run_fp32_fifo(reqs, pool, t_f=1000, max_attempts=4, time_cap_s=60.0):
    """The plain FP32 per-instance path: requests served one at a time in arrival
    order; stops taking new requests after time_cap_s (the rest count as unserved)."""
    import torch

    dev = torch.device("cuda", 0)
    Td = torch.as_tensor(inst.schedule(t_f), device=dev)
    t0 = time.perf_counter()
    ttt, served, spin = [], 0, 0
    for r in reqs:
        now = time.perf_counter() - t0
        if now > time_cap_s:
            break
        if r["arrival"] > now:
            time.sleep(r["arrival"] - now)
        J = pool.get(r["kind"], r["n"])
        p = nmfa.Problem(J, precision="fp32")
        R = r["replicas"]
        e = torch.empty(R, dtype=torch.float64, device=dev)
        target = target_energy(r["kind"], r["n"])
        for attempt in range(max_attempts):
            p.run_device(Td, 0.15, 0.15, R, seed=r["seed"], stream_id=attempt, energy=e)
            p.sync()
            spin += R * r["n"] * t_f
            if float(e.min().item()) <= target:
                ttt.append(time.perf_counter() - t0 - r["arrival"])
                break
        p.close()
        served += 1
    wall = time.perf_counter() - t0
    return {"requests": len(reqs), "served": served, "succeeded": len(ttt), "p50_ttt_s": percentile(ttt, 50),
            "p99_ttt_s": percentile(ttt, 99), "spin_updates_per_s": spin / wall, "wall_s": wall}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--duration", type=float, default=1.0)
    ap.add_argument("--n-lo", type=int, default=64)
    ap.add_argument("--n-hi", type=int, default=8192)
    ap.add_argument("--t-f", type=int, default=1000)
    ap.add_argument("--max-inflight", type=int, default=2)
    ap.add_argument("--precision", default="bf16_fp8j", choices=["bf16", "bf16_fp8j"],
                    help="storage of J: bf16, or bf16_fp8j (E4M3, half the bytes; batches widen n <= 4096 once, "
                         "larger n in the kernel)")
    ap.add_argument("--fp32-cap", type=float, default=30.0, help="seconds of FP32 FIFO serving (0: skip)")
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args()
    reqs = make_stream(args.rate, args.duration, args.n_lo, args.n_hi, args.seed)
    pool = InstancePool()
    for r in reqs:  # generate every instance before the clock starts
        pool.get(r["kind"], r["n"])
    out = {"workload": "Poisson %.0f req/s for %.2f s, N log-uniform in [%d, %d] (16 sizes), SK or G(N,0.5), "
                       "R in {64..1024}, t_f=%d, %s J" % (args.rate, args.duration, args.n_lo, args.n_hi, args.t_f,
                                                          args.precision),
           "tensor_server": run_server(reqs, pool, args.t_f, args.precision, args.max_inflight)}
    if args.fp32_cap > 0:
        out["fp32_fifo"] = run_fp32_fifo(reqs, pool, args.t_f, time_cap_s=args.fp32_cap)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
