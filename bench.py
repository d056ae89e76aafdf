"""Benchmark of the NMFA hot path on one GB300 (or N GPUs, one process each).

Workload (one "step" = one full run of Algorithm 1 plus readout and energies):
Sherrington-Kirkpatrick instance, N = 2000 spins, J_ij = +-1 symmetric, h = 0,
1024 replicas, t_f = 1000 steps, sigma = alpha = 0.15, the default three-segment
schedule; J and S in BF16 with FP32 accumulation on the tcgen05 tensor cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl nmfa|reference]

Prints one JSON line.  `value` is whole-job spin-updates/s with inputs resident in
HBM; `e2e` is the same metric through the host-buffer C call (nmfa_run) with the
temperature upload and the sign/energy download inside the timed region.
`--impl reference` times the FP64 CPU oracle on a bounded sample of the workload.
Multi-GPU: each rank runs its own replicas (weak scaling, no data-path collective).

On rank 0 the line also carries the metric's second half and the other workloads,
each measured after the timed region (`--no-extra` skips them):
  time_to_target -- a bounded served leg: Poisson arrivals (200 req/s for 0.5 s, N
                    log-uniform in [64, 2048], SK or G(N, 0.5), 64-1024 replicas,
                    FP8-stored J) through the library's server, and the same request
                    stream through the plain FP32 per-instance path in arrival order:
                    p50/p99 time-to-target and success fractions of both;
  c1_fp64        -- SK N = 100, 100 replicas, t_f = 1000 on the FP64 path;
  c3_csr         -- Moebius ladder N = 2000, int8 CSR, 512 replicas, FP32;
  c4_ragged      -- 512 instances, N uniform in [16, 1000], 64 replicas each, one
                    persistent launch replayed from a CUDA graph;
each with its own roofline fraction.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NMFA spin-updates/s and p50/p99 time-to-target vs plain FP32 path, one GB300"
N_SPINS, REPLICAS, T_F = 2000, 1024, 1000
SIGMA = ALPHA = 0.15


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons, powers = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                powers.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(powers) if powers else None}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def sources_digest(paths):
    """SHA-256 of the kernel sources' code: `//` comments, trailing blanks and empty
    lines are left out, so that editing a comment does not invalidate a capture."""
    import hashlib
    import re

    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), encoding="utf-8") as f:
            for line in f:
                code = re.sub(r"//.*", "", line).rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()


def kernel_traffic():
    """DRAM bytes per launch of the tensor kernel from the committed ncu capture of the
    bench workload, or None when the kernel sources' code has changed since the capture."""
    try:
        with open(os.path.join(ROOT, "profiles", "nmfa_tc_kernel_sk2000_r1024_traffic.json")) as f:
            rec = json.load(f)
        ok = sources_digest(rec["sources"]) == rec["sources_code_sha256"]
        return rec["dram_bytes_per_launch"] if ok else None
    except Exception:
        return None


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or None."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def cpu_baseline(sample_replicas=48, sample_steps=T_F, nthreads=0, extra=True):
    """The FP64 oracle (as it stands) on a bounded sample of the workload: the same
    instance and schedule, `sample_replicas` of the 1024 replicas over the first
    `sample_steps` steps (about 10 s of CPU work at the defaults), OpenMP over
    replicas on every host core.  With `extra`, also the same code on one thread (2
    replicas x 500 steps) and the plain FP64 workload (SK N = 100, 100 replicas,
    t_f = 1000) in full on every core."""
    import numpy as np

    import oracle
    from paper_1806_08422_gb300 import instances as inst

    J = inst.sk(N_SPINS, 0)
    T = inst.schedule(T_F)[:sample_steps]
    cores = os.cpu_count() if nthreads <= 0 else nthreads
    t0 = time.perf_counter()
    oracle.run(J, T, SIGMA, ALPHA, sample_replicas, seed=0, nthreads=cores)
    dt = time.perf_counter() - t0
    units = sample_replicas * N_SPINS * sample_steps
    out = {"value": units / dt, "unit": "spin-updates/s", "cores": cores, "kind": "oracle",
           "sample": "SK N=%d, %d replicas x first %d of %d steps (FP64 C oracle, OpenMP over replicas), %.2f s"
                     % (N_SPINS, sample_replicas, sample_steps, T_F, dt),
           "cpu_model": cpu_model(), "nproc": os.cpu_count()}
    if extra:
        t0 = time.perf_counter()
        oracle.run(J, inst.schedule(T_F)[:500], SIGMA, ALPHA, 2, seed=0, nthreads=1)
        d1 = time.perf_counter() - t0
        out["single_thread"] = {"value": 2 * N_SPINS * 500 / d1, "unit": "spin-updates/s", "cores": 1,
                                "sample": "SK N=%d, 2 replicas x first 500 steps, one thread, %.2f s"
                                          % (N_SPINS, d1)}
        J1 = inst.sk(100, 0)
        t0 = time.perf_counter()
        oracle.run(J1, inst.schedule(T_F), SIGMA, ALPHA, 100, seed=0, nthreads=cores)
        dc = time.perf_counter() - t0
        out["c1_full"] = {"value": 100 * 100 * T_F / dc, "unit": "spin-updates/s", "cores": cores,
                          "sample": "plain FP64 workload in full: SK N=100, 100 replicas, t_f=%d, %.2f s"
                                    % (T_F, dc)}
    return out


# ------------------------------------------------------------------ other workloads
# CSR kernel's warp instructions per spin-update on the Moebius ladder N = 2000 with
# 512 replicas (ncu: smsp__inst_executed.sum / spin-updates,
# profiles/csr_kernel_moebius2000_r512_tf100_full.md); the issue roofline is four warp
# instructions per clock on each SM.
CSR_WARP_INSTR_PER_UPDATE = 3.07


def _kernel_ms_runs(prob, reps, run):
    """Median annealing-kernel time (CUDA events the library records on the run's
    stream) over `reps` runs after one warm-up run."""
    from paper_1806_08422_gb300 import nmfa

    nmfa.nmfa_profile_enable(prob.handle, True)
    run()
    prob.sync()
    ms = []
    for _ in range(reps):
        run()
        prob.sync()
        ms.append(nmfa.nmfa_last_kernel_ms(prob.handle))
    nmfa.nmfa_profile_enable(prob.handle, False)
    return statistics.median(ms)


def leg_c1_fp64(dev, stream, alu, reps=5):
    """The plain FP64 configuration: SK N = 100, 100 replicas, t_f = 1000."""
    import torch

    from paper_1806_08422_gb300 import instances as inst
    from paper_1806_08422_gb300 import nmfa

    n, R = 100, 100
    p = nmfa.Problem(inst.sk(n, 0), precision="fp64")
    T = torch.as_tensor(inst.schedule(T_F), device=dev)
    signs = torch.empty((R, n), dtype=torch.int8, device=dev)
    e = torch.empty(R, dtype=torch.int64, device=dev)
    ms = _kernel_ms_runs(p, reps, lambda: p.run_device(T, SIGMA, ALPHA, R, signs=signs, energy_i64=e, stream=stream))
    p.close()
    tflops = 2.0 * n * n * R * T_F / (ms / 1e3) / 1e12
    pk = alu["fp64_fma_tflops"] if alu else None
    return {"workload": "SK N=100 J=+-1, 100 replicas, t_f=1000, FP64 CUDA-core path", "kernel_ms": ms,
            "spin_updates_per_s": n * R * T_F / (ms / 1e3), "us_per_replica_run": 1e3 * ms / R,
            "min_energy": int(e.min().item()),
            "roofline": {"bound": "alu", "achieved": tflops, "unit": "TFLOP/s", "peak": pk,
                         "frac": tflops / pk if pk else None,
                         "peak_source": "measured FP64 FMA rate (nmfa_measure_alu_peaks)",
                         "note": "2 n^2 flops per replica-step; 100 CTAs (one replica each) on 152 SMs"}}


def leg_c3_csr(dev, stream, sm_mhz, reps=5):
    """Sparse MAX-CUT: Moebius ladder N = 2000, int8 CSR, 512 replicas, FP32."""
    import torch

    from paper_1806_08422_gb300 import instances as inst
    from paper_1806_08422_gb300 import nmfa

    n, R = 2000, 512
    p = nmfa.Problem(csr=inst.moebius_csr(n), n=n, precision="fp32")
    T = torch.as_tensor(inst.schedule(T_F), device=dev)
    signs = torch.empty((R, n), dtype=torch.int8, device=dev)
    e = torch.empty(R, dtype=torch.int64, device=dev)
    ms = _kernel_ms_runs(p, reps, lambda: p.run_device(T, SIGMA, ALPHA, R, signs=signs, energy_i64=e, stream=stream))
    p.close()
    rate = n * R * T_F / (ms / 1e3)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * 4 * sm_mhz * 1e6 / CSR_WARP_INSTR_PER_UPDATE
    return {"workload": "Moebius ladder N=2000 (J=+1 per edge), int8 CSR, 512 replicas, t_f=1000, FP32", "kernel_ms": ms,
            "spin_updates_per_s": rate, "min_energy": int(e.min().item()), "ground_energy": 4 - 3 * n // 2,
            "roofline": {"bound": "alu", "achieved": rate, "unit": "spin-updates/s", "peak": peak, "frac": rate / peak,
                         "peak_source": "instruction issue: %d SMs x 4 warp instructions/clock x %.0f MHz / %.2f warp "
                                        "instructions per spin-update (ncu count)"
                                        % (sms, sm_mhz, CSR_WARP_INSTR_PER_UPDATE)}}


def leg_c4_ragged(dev, stream, peaks, reps=3, count=512, R=64):
    """Ragged batch: `count` instances, N uniform in [16, 1000], half SK, half
    G(N, 0.5) max-cut, R replicas each, one persistent launch replayed from a CUDA
    graph, tiles from the autotuner."""
    import numpy as np
    import torch

    from paper_1806_08422_gb300 import instances as inst
    from paper_1806_08422_gb300 import nmfa

    mix = inst.ragged_batch(count, 16, 1000, seed=0)
    probs = [nmfa.Problem(J, precision="bf16") for _, _, J in mix]
    T = torch.as_tensor(inst.schedule(T_F), device=dev)
    energies = [torch.empty(R, dtype=torch.int64, device=dev) for _ in mix]
    jobs = [nmfa.make_job(T, SIGMA, ALPHA, R, seed=0, stream_id=k, energy_i64=e) for k, e in enumerate(energies)]
    b = nmfa.nmfa_batch_create([p.handle for p in probs], jobs, nmfa.NMFA_BATCH_GRAPH | nmfa.NMFA_BATCH_AUTOTUNE)
    try:
        nmfa.nmfa_batch_launch(b, stream)
        nmfa.nmfa_batch_sync(b)
        ms = []
        for _ in range(reps):
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            nmfa.nmfa_batch_launch(b, stream)
            z.record(stream)
            nmfa.nmfa_batch_sync(b)
            stream.synchronize()
            ms.append(a.elapsed_time(z))
        info = nmfa.nmfa_batch_info(b)
    finally:
        nmfa.nmfa_batch_destroy(b)
        for p in probs:
            p.close()
    ns = np.array([n for _, n, _ in mix], dtype=np.float64)
    npad = np.ceil(ns / 128.0) * 128.0
    per = statistics.median(ms) / 1e3
    flops = 2.0 * float((ns ** 2).sum()) * R * (T_F + 1)       # t_f products + the energy product
    flops_pad = 2.0 * float((npad ** 2).sum()) * R * (T_F + 1)
    burst = peaks.get("bf16_tflops", peaks.get("bf16_tflops_sustained"))
    achieved = flops / per / 1e12
    return {"workload": "%d instances, N uniform in [16, 1000] (half SK +-1, half G(N,0.5) max-cut), %d replicas each, "
                        "t_f=1000, BF16 J/S, FP32 accumulation, one persistent launch from a CUDA graph, autotuned "
                        "tiles" % (count, R),
            "ms_per_batch": statistics.median(ms), "spin_updates_per_s": float(ns.sum()) * R * T_F / per,
            "grid": info["grid"], "groups": info["groups"],
            "roofline": {"bound": "tensor", "achieved": achieved, "unit": "TFLOP/s", "peak": burst,
                         "frac": achieved / burst, "peak_source": "bf16_tflops (burst)",
                         "achieved_at_padded_sizes": flops_pad / per / 1e12,
                         "note": "algorithmic flops 2 N^2 R (t_f + 1) at each instance's own N; the kernel computes "
                                 "128-padded tiles"}}


def leg_served(rate=200.0, duration=0.5, n_lo=64, n_hi=2048, fp32_cap=30.0):
    """The metric's second half: p50/p99 time-to-target of a Poisson request stream
    through the library's server (continuous batching on the tensor path, FP8-E4M3-
    stored J as the serving workload specifies) and through the plain FP32
    per-instance path in arrival order, same requests,
    same seeds and noise streams (attempt k draws stream k on both)."""
    from paper_1806_08422_gb300 import serve

    reqs = serve.make_stream(rate, duration, n_lo, n_hi, seed=0)
    pool = serve.InstancePool()
    for r in reqs:
        pool.get(r["kind"], r["n"])
    srv = serve.run_server(reqs, pool)
    srv16 = serve.run_server(reqs, pool, precision="bf16")
    f32 = serve.run_fp32_fifo(reqs, pool, time_cap_s=fp32_cap)

    def summary(d, served):
        return {"p50_s": d["p50_ttt_s"], "p99_s": d["p99_ttt_s"], "requests": d["requests"], "served": served,
                "succeeded": d["succeeded"], "p_success": d["succeeded"] / max(1, served),
                "spin_updates_per_s": d["spin_updates_per_s"], "wall_s": d["wall_s"]}

    return {"workload": "Poisson %.0f req/s for %.2f s (%d requests), N log-uniform in [%d, %d] (16 sizes), SK +-1 or "
                        "G(N,0.5) max-cut, R in {64,...,1024}, t_f=1000; target H <= -0.70 N^1.5 (SK) / -0.34 N^1.5 "
                        "(G(N,0.5)); up to 4 attempts (attempt k on noise stream k)"
                        % (rate, duration, len(reqs), n_lo, n_hi),
            "tensor_server": dict(summary(srv, srv["requests"]), launches=srv["launches"],
                                  batches_reused=srv["batches_reused"],
                                  mean_attempts=srv["mean_attempts"], precision="FP8-E4M3-stored J (widened to BF16 once per batch for N <= 4096), BF16 S"),
            "tensor_server_bf16_stored_j": dict(summary(srv16, srv16["requests"]), launches=srv16["launches"],
                                                batches_reused=srv16["batches_reused"]),
            "fp32_per_instance": dict(summary(f32, f32["served"]), time_cap_s=fp32_cap,
                                      note="served one request at a time in arrival order; requests not started "
                                           "within the cap are not counted")}


def bench_config(precision, tf, ws):
    """The workload both arms name: the bench's run of Algorithm 1."""
    return {"workload": "SK N=2000 J=+-1 h=0, 1024 replicas, t_f=1000, sigma=alpha=0.15, "
                        "default 3-segment schedule; %s" % (
                            "BF16 J/S, FP32 accumulation on tcgen05" if precision == "bf16"
                            else precision + " CUDA-core path"),
            "n": N_SPINS, "replicas_per_gpu": REPLICAS, "t_f": tf,
            "l2": "flushed between timed steps (256 MB write, outside the step events)",
            "parallelism": "replicas" if ws == 1 else "replicas x%d ranks" % ws}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        cpu_baseline(sample_replicas=16, sample_steps=20, extra=False)
    vals = []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(sample_replicas=16, sample_steps=200, extra=False))
    wall = time.perf_counter() - t_all
    units = sum(16 * N_SPINS * 200 for _ in vals)
    value = units / wall
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "spin-updates/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": bench_config(args.precision, args.tf, ws),
            "cpu_baseline": {"value": value, "unit": "spin-updates/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": "FP64 C oracle, OpenMP over replicas; each bench step a bounded sample of "
                                       "the workload: 16 of its 1024 replicas over the first 200 of its 1000 "
                                       "steps"},
            "e2e": {"value": value, "unit": "spin-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="nmfa", choices=["nmfa", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32-compare", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the served leg and the C1/C3/C4 workloads")
    ap.add_argument("--tf", type=int, default=T_F, help="steps per run (profiling of a shorter run)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    import __graft_entry__
    from paper_1806_08422_gb300 import instances as inst
    from paper_1806_08422_gb300 import nmfa

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        from paper_1806_08422_gb300 import multi as _multi
        _multi.init_ranks("nccl", timeout_s=300, device_id=torch.device("cuda", local))
    if rank == 0 or not os.path.exists(nmfa.LIB_PATH):
        __graft_entry__.build()
    if ws > 1:
        dist.barrier()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    J = inst.sk(N_SPINS, 0)
    T = inst.schedule(T_F)[:args.tf]
    prob = nmfa.Problem(J, precision=args.precision)
    Td = torch.as_tensor(T, device=dev)
    signs = torch.empty((REPLICAS, N_SPINS), dtype=torch.int8, device=dev)
    energy = torch.empty(REPLICAS, dtype=torch.float64, device=dev)
    energy_i64 = torch.empty(REPLICAS, dtype=torch.int64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    from paper_1806_08422_gb300 import multi
    stream_id = multi.rank_stream(rank)  # each rank anneals its own independent replicas

    def one_step():
        prob.run_device(Td, SIGMA, ALPHA, REPLICAS, seed=0, stream_id=stream_id, signs=signs, energy=energy,
                        energy_i64=energy_i64, stream=stream)

    nmfa.nmfa_profile_enable(prob.handle, True)
    for _ in range(args.warmup):
        one_step()
    prob.sync()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kernel_ms = []
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    launches0 = nmfa.nmfa_launch_count()
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()  # L2 flush between timed steps (outside the step events)
        ev[k][0].record(stream)
        one_step()
        ev[k][1].record(stream)
        kernel_ms.append(None)
        torch.cuda.synchronize()
        kernel_ms[-1] = nmfa.nmfa_last_kernel_ms(prob.handle)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    launches = nmfa.nmfa_launch_count() - launches0
    clocks = sampler.stop()
    prob.sync()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    if ws > 1:
        total_ms = multi.max_over_ranks(total_ms, device=dev)
    units_per_step = REPLICAS * N_SPINS * args.tf
    value = units_per_step * ws * args.steps / (total_ms / 1e3)

    # end to end through the host-buffer C call (T upload, signs + energies download)
    nmfa.nmfa_profile_enable(prob.handle, False)
    e2e_steps = max(3, min(args.steps, 5))
    nmfa.nmfa_run(prob.handle, N_SPINS, T, SIGMA, ALPHA, REPLICAS, 0, stream_id, True)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        nmfa.nmfa_run(prob.handle, N_SPINS, T, SIGMA, ALPHA, REPLICAS, 0, stream_id, True)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if ws > 1:
        e2e_s = multi.max_over_ranks(e2e_s, device=dev)
    e2e = {"value": units_per_step * ws / e2e_s, "unit": "spin-updates/s", "h2d_bytes_per_step": args.tf * 8,
           "d2h_bytes_per_step": REPLICAS * N_SPINS + REPLICAS * 8 * 2}

    peaks, peak_kind = _peaks()
    kern_ms = statistics.mean(kernel_ms)
    # t_f products J S (2 N^2 R each) plus, on the tensor path, the energy product J s~
    # the kernel forms after the last step
    flops = 2.0 * N_SPINS * N_SPINS * REPLICAS * (args.tf + (1 if args.precision == "bf16" else 0))
    if args.precision == "bf16":
        # each launch is timed on its own (about 10 ms, clocks at maximum below the
        # power cap), so the denominator is the burst GEMM figure; the fraction of the
        # seconds-long sustained figure is reported beside it
        peak = peaks.get("bf16_tflops", peaks.get("bf16_tflops_sustained"))
        sustained = peaks.get("bf16_tflops_sustained")
        achieved = flops / (kern_ms / 1e3) / 1e12
        roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": kernel_traffic() if args.tf == T_F else None,
                    "kernel": "nmfa_tc_kernel<128>", "kernel_ms": kern_ms,
                    "peak_source": "%s bf16_tflops (burst)" % peak_kind,
                    "frac_of_sustained": achieved / sustained if sustained else None}
    else:
        # CUDA-core path: FMA-bound; the denominator is this device's measured FMA rate
        # (measured after the timed region, outside the launch count)
        achieved = flops / (kern_ms / 1e3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": None, "unit": "TFLOP/s", "frac": None,
                    "traffic": None, "kernel_ms": kern_ms}

    extra = {}
    alu = nmfa.nmfa_measure_alu_peaks(stream) if rank == 0 else None
    if alu is not None:
        extra["alu_peaks"] = dict(alu, source="measured by nmfa_measure_alu_peaks (FMA chains on every SM)")
        if args.precision != "bf16":
            pk = alu["fp64_fma_tflops" if args.precision == "fp64" else "fp32_fma_tflops"]
            roofline.update({"peak": pk, "frac": achieved / pk,
                             "peak_source": "measured %s FMA rate" % args.precision})
    if rank == 0 and not args.no_fp32_compare and args.precision != "fp32":
        # the plain FP32 per-instance CUDA-core path on the same workload
        p32 = nmfa.Problem(J, precision="fp32")
        nmfa.nmfa_profile_enable(p32.handle, True)
        p32.run_device(Td, SIGMA, ALPHA, REPLICAS, signs=signs, energy=energy, stream=stream)
        p32.sync()
        ms32 = []
        for _ in range(2):
            p32.run_device(Td, SIGMA, ALPHA, REPLICAS, signs=signs, energy=energy, stream=stream)
            p32.sync()
            ms32.append(nmfa.nmfa_last_kernel_ms(p32.handle))
        tf32 = 2.0 * N_SPINS * N_SPINS * REPLICAS * args.tf / (statistics.mean(ms32) / 1e3) / 1e12
        extra["fp32_path"] = {"value": units_per_step / (statistics.mean(ms32) / 1e3), "unit": "spin-updates/s",
                              "kernel_ms": statistics.mean(ms32),
                              "roofline": {"bound": "alu", "achieved": tf32, "unit": "TFLOP/s",
                                           "peak": alu["fp32_fma_tflops"] if alu else None,
                                           "frac": tf32 / alu["fp32_fma_tflops"] if alu else None}}
        p32.close()

    if rank == 0 and not args.no_extra and args.precision == "bf16":
        sm_mhz = clocks.get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0
        extra["time_to_target"] = leg_served()
        extra["c1_fp64"] = leg_c1_fp64(dev, stream, alu)
        extra["c3_csr"] = leg_c3_csr(dev, stream, sm_mhz)
        extra["c4_ragged"] = leg_c4_ragged(dev, stream, peaks)

    if rank == 0:
        cpu = None if args.no_cpu_baseline else cpu_baseline()
        line = {"metric": METRIC, "value": value, "unit": "spin-updates/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
                "config": bench_config(args.precision, args.tf, ws),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks, "wall_s_timed": t_wall, "step_ms": step_ms}
        line.update(extra)
        print(json.dumps(line), flush=True)
    prob.close()
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
