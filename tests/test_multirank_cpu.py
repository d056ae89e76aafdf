"""The multi-GPU (replicas-only) path's host logic on two gloo ranks on the CPU:
each rank anneals its own batch on its own noise stream (here with the oracle, as
no GPU is needed to check the bookkeeping), rank 0 gathers every rank's energies,
and the whole-job time is the maximum over ranks."""
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
