"""Success probability and time-to-solution on synthetic stand-ins of the paper's
Fig. 4 instance classes (Sec. III):

  SK     -- J_ij = +-1, 10 instances per size     (Fig. 4a)
  dense  -- G(N, 0.5) MAX-CUT, 10 per size         (Fig. 4b)
  cubic  -- random 3-regular MAX-CUT, 20 per size  (Fig. 4c)

Every instance of one (class, size) runs its samples (independent replicas of
Algorithm 1, default schedule, t_f steps, sigma = alpha = 0.15) in ONE batched
tensor-core launch.  Sample time tau = launch wall time / total samples (the paper
measures NMFA time per sample as wall clock over 10,000 samples).  A sample
succeeds when it reaches the instance's target energy; the target is the lowest
energy any sample of the instance found (at these sizes, with 10,000 samples, that
is the ground state with overwhelming probability; the paper's own targets and the
CIM data are not available).  TTS99 = tau ln(0.01) / ln(1 - p) for p < 0.99, else tau.
Reported per class and size: medians and interquartile ranges over instances.

    python -m paper_1806_08422_gb300.tts [--sizes 20,40,60,80,100] [--samples 10000]

This module only drives the C ABI; all annealing runs in the library's kernels.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import instances as inst
from . import nmfa

CLASSES = {"sk": 10, "dense": 10, "cubic": 20}


def make(kind, n, k):
    if kind == "sk":
        return inst.sk(n, seed=7000 + 97 * n + k)
    if kind == "dense":
        return inst.gnp_maxcut(n, 0.5, seed=8000 + 97 * n + k)
    return inst.regular3(n, seed=9000 + 97 * n + k)


def tts99(tau, p):
    if p <= 0.0:
        return math.inf
    if p >= 0.99:
        return tau
    return tau * math.log(0.01) / math.log(1.0 - p)


def quartiles(xs):
    xs = np.asarray(xs, dtype=np.float64)
    q = np.percentile(xs, [25, 50, 75])
    return {"median": float(q[1]), "q25": float(q[0]), "q75": float(q[2])}


def sample_energies(kind, n, samples=10000, t_f=1000, seed=1, graph=True):
    """Anneals `samples` replicas of every instance of one (class, size) in one
    batched launch (instance k on noise stream k).  Returns the instances, their
    energies (one int64 array per instance, replica order) and the wall time of
    the timed launch (a warm-up launch runs first)."""
    import torch

    dev = torch.device("cuda", 0)
    Js = [make(kind, n, k) for k in range(CLASSES[kind])]
    probs = [nmfa.Problem(J, precision="bf16") for J in Js]
    T = torch.as_tensor(inst.schedule(t_f), device=dev)
    energies = [torch.empty(samples, dtype=torch.int64, device=dev) for _ in Js]
    jobs = [nmfa.make_job(T, 0.15, 0.15, samples, seed=seed, stream_id=k, energy_i64=e)
            for k, e in enumerate(energies)]
    b = nmfa.nmfa_batch_create([p.handle for p in probs], jobs, nmfa.NMFA_BATCH_GRAPH if graph else 0)
    try:
        nmfa.nmfa_batch_launch(b)  # warm-up
        nmfa.nmfa_batch_sync(b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nmfa.nmfa_batch_launch(b)
        nmfa.nmfa_batch_sync(b)
        wall = time.perf_counter() - t0
    finally:
        nmfa.nmfa_batch_destroy(b)
        for p in probs:
            p.close()
    return Js, [e.cpu().numpy() for e in energies], wall


def run_class(kind, n, samples=10000, t_f=1000, seed=1, targets=None):
    """Success probability and TTS99 per instance of one (class, size), summarised as
    medians and quartiles.  `targets` (one energy per instance) defaults to the
    lowest energy any sample of the instance found."""
    Js, energies, wall = sample_energies(kind, n, samples, t_f, seed)
    tau = wall / (samples * len(Js))
    ps, tts = [], []
    for k, ev in enumerate(energies):
        target = ev.min() if targets is None else targets[k]
        p = float(np.mean(ev <= target))
        ps.append(p)
        tts.append(tts99(tau, p))
    return {"class": kind, "n": n, "instances": len(Js), "samples": samples, "tau_us": tau * 1e6,
            "p": quartiles(ps), "tts99_us": quartiles([x * 1e6 for x in tts]),
            "per_instance": [{"p": p, "tts99_us": x * 1e6} for p, x in zip(ps, tts)]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sizes", default="20,40,60,80,100")
    ap.add_argument("--samples", type=int, default=10000)
    ap.add_argument("--t-f", type=int, default=1000)
    ap.add_argument("--classes", default="sk,dense,cubic")
    args = ap.parse_args()
    out = []
    for kind in args.classes.split(","):
        for n in [int(x) for x in args.sizes.split(",")]:
            if kind == "cubic" and n % 2:
                n += 1
            out.append(run_class(kind, n, args.samples, args.t_f))
            print(json.dumps(out[-1]), flush=True)


if __name__ == "__main__":
    main()
