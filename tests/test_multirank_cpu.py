"""The multi-GPU (replicas-only) path's host logic on two gloo ranks on the CPU:
each rank anneals its own batch on its own noise stream (here with the oracle, as
no GPU is needed to check the bookkeeping), rank 0 gathers every rank's energies,
and the whole-job time is the maximum over ranks.  Failure detection: a rank that
never joins, or dies after joining, ends rank 0's rendezvous or collective with an
error within the process group's timeout instead of a hang."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from paper_1806_08422_gb300 import instances as inst
from paper_1806_08422_gb300 import multi


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_path):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    J = inst.moebius(16)
    res = oracle.run(J, inst.schedule(60), 0.15, 0.15, 8, seed=5, stream=multi.rank_stream(rank, 10))
    e = torch.tensor(res["energy_i64"], dtype=torch.int64)
    gathered = multi.gather_to_rank0(e)
    t_max = multi.max_over_ranks(1.0 + rank)
    if rank == 0:
        np.save(out_path, gathered.numpy())
        with open(out_path + ".t", "w") as f:
            f.write(repr(t_max))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gather_and_timing(tmp_path):
    out = str(tmp_path / "gathered.npy")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
    got = np.load(out)
    J = inst.moebius(16)
    for rank in range(2):
        ref = oracle.run(J, inst.schedule(60), 0.15, 0.15, 8, seed=5, stream=10 + rank)["energy_i64"]
        np.testing.assert_array_equal(got[rank], ref)
    assert float(open(out + ".t").read()) == 2.0


def _failing_worker(rank, world, port, mode, out_path):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    if rank == 1 and mode == "never_joins":
        os._exit(3)
    stage = "init"
    try:
        multi.init_ranks("gloo", timeout_s=5, rank=rank, world_size=world)
        if rank == 1:
            os._exit(4)  # dies between steps, with nothing of its own in flight
        stage = "gather"
        multi.gather_to_rank0(torch.zeros(4, dtype=torch.int64))
        stage = "completed"
    except Exception as e:  # the failure reaches rank 0 as an error
        stage = stage + " failed: " + type(e).__name__
    with open(out_path, "w") as f:
        f.write(stage)


@pytest.mark.parametrize("mode", ["never_joins", "dies_after_join"])
def test_failed_rank_is_detected_without_a_hang(tmp_path, mode):
    import multiprocessing
    import time

    out = str(tmp_path / "rank0.txt")
    ctx = multiprocessing.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_failing_worker, args=(r, 2, port, mode, out)) for r in range(2)]
    t0 = time.time()
    for p in procs:
        p.start()
    procs[0].join(timeout=120)
    alive = procs[0].is_alive()
    for p in procs:
        if p.is_alive():
            p.kill()
        p.join()
    assert not alive, "rank 0 hung"
    assert procs[0].exitcode == 0
    got = open(out).read()
    assert ("init failed" if mode == "never_joins" else "gather failed") in got, got
    assert time.time() - t0 < 120


# ---------------------------------------------------------------- row partition
# One instance split by rows over two gloo ranks (the layout for instances whose
# replica blocks exceed one GPU).  Each rank holds only its rows of J and, every
# step, computes its own spins' new state from the full previous state (here with the
# oracle: its rows of J placed at their global rows of an otherwise empty matrix, so
# Phi of every other row reads as 0 and is discarded; the step index continues the
# noise stream); the all-gather of the blocks is the synchronising exchange.  The
# gathered trajectory must equal the oracle's unpartitioned run bit for bit.
def _rowpart_worker(rank, world, port, out_path, n, R, t_f):
    import torch.distributed as dist

    from paper_1806_08422_gb300 import rowpart

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    J = inst.sk(n, 41)
    T = inst.schedule(t_f)
    lo, hi = rowpart.row_ranges(n, world)[rank]
    mine = np.zeros((n, n))
    mine[lo:hi, :] = rowpart.local_rows(J, rank, world)  # the only rows this rank holds
    s = torch.zeros((R, n), dtype=torch.float64)
    for t in range(t_f):
        step = oracle.run(mine, T[t:t + 1], 0.15, 0.15, R, seed=3, stream=1, s0=s.numpy(), want_state=True,
                          t_first=t)["state"]
        s = rowpart.allgather_state(torch.from_numpy(np.ascontiguousarray(step[:, lo:hi])), n, world)
    if rank == 0:
        np.save(out_path, s.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("n", [300, 256])
def test_row_partition_two_ranks_matches_unpartitioned_run(tmp_path, n):
    from paper_1806_08422_gb300 import rowpart
    R, t_f = 6, 25
    rowpart.check_partition(n, 2)
    out = str(tmp_path / "state.npy")
    mp.start_processes(_rowpart_worker, args=(2, _free_port(), out, n, R, t_f), nprocs=2, start_method="spawn",
                       join=True)
    ref = oracle.run(inst.sk(n, 41), inst.schedule(t_f), 0.15, 0.15, R, seed=3, stream=1, want_state=True)["state"]
    np.testing.assert_array_equal(np.load(out), ref)


def test_row_ranges_and_memory_budget():
    from paper_1806_08422_gb300 import rowpart
    for n, w in [(1, 1), (127, 2), (128, 2), (300, 2), (100000, 8), (19457, 3), (1000, 16)]:
        rowpart.check_partition(n, w)
    # 10^5 spins on 8 ranks: 782 blocks of 128 -> 98 per rank (the last 96 + tail)
    r = rowpart.row_ranges(100000, 8)
    assert r[0] == (0, 98 * 128) and r[-1][1] == 100000
    m = rowpart.memory_per_rank(100000, 1024, 8)
    assert m["J"] == 98 * 128 * 100000            # FP8 rows of J: 1.25 GB
    assert m["state"] == 2 * 1024 * 100000 * 2     # both BF16 state buffers: 410 MB
    assert m["total"] < 2 * 10 ** 9
