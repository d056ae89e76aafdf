"""Row-partitioned layout of ONE instance over several GPUs (bookkeeping only).

The single-GPU tensor path needs every row-block tile of a replica block resident
at once (the tiles exchange their state every step), which caps it at
n_pad / 128 <= number of SMs (n <= 19,456 on a 152-SM GB300).  Past that, one
instance is split by rows of J across ranks:

  * rank k owns the contiguous spins [lo_k, hi_k) (multiples of 128, the tile
    height; the last rank takes the ragged tail) and holds only those rows of J
    (Algorithm 1's field of spin i reads row i of J and the whole previous state);
  * each step every rank computes Phi and the new state of its own spins for all
    replicas, from the full previous state;
  * then every rank gathers every other rank's new block (one all-gather of the
    R x n state per step).  The gather is also what keeps the update synchronous:
    no rank starts step t + 1 before every block of step t has arrived;
  * the noise draw of (replica r, step t, spin i) uses the global spin index i, so a
    partitioned run draws exactly the noise of an unpartitioned one.

This module holds the partition (ranges, local row blocks, the padded all-gather)
and no arithmetic of the method; the GPU kernels would run per rank on the local
block.
"""
from __future__ import annotations

import numpy as np

ROW_BLOCK = 128


def row_ranges(n: int, world: int, align: int = ROW_BLOCK):
    """Spins [lo, hi) of each rank: whole blocks of `align` spins dealt out as evenly
    as possible (the first ranks take one block more), the ragged tail on the last
    rank that has any.  Ranks beyond the number of blocks get empty ranges."""
    if n < 1 or world < 1:
        raise ValueError("n and world must be >= 1")
    blocks = -(-n // align)
    base, extra = divmod(blocks, world)
    out, b0 = [], 0
    for k in range(world):
        nb = base + (1 if k < extra else 0)
        lo, hi = min(n, b0 * align), min(n, (b0 + nb) * align)
        out.append((lo, hi))
        b0 += nb
    return out


def local_rows(J, rank: int, world: int):
    """Rank `rank`'s rows of the dense couplings, J[lo:hi, :] (a view)."""
    lo, hi = row_ranges(J.shape[0], world)[rank]
    return J[lo:hi, :]


def allgather_state(local, n: int, world: int):
    """All-gather of the ranks' state blocks: each rank passes its (R, hi - lo) block
    (a torch tensor, any device the process group serves); every rank receives the
    full (R, n) state in spin order.  Blocks are padded to the largest block height
    so that one equal-sized all_gather serves ragged partitions."""
    import torch
    import torch.distributed as dist

    ranges = row_ranges(n, world)
    width = max(hi - lo for lo, hi in ranges)
    R = local.shape[0]
    pad = torch.zeros((R, width), dtype=local.dtype, device=local.device)
    pad[:, :local.shape[1]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad)
    return torch.cat([p[:, :hi - lo] for p, (lo, hi) in zip(parts, ranges)], dim=1)


def memory_per_rank(n: int, replicas: int, world: int, j_bytes: int = 1, state_bytes: int = 2,
                    master_bytes: int = 4) -> dict:
    """Device bytes of the largest rank: its rows of J (j_bytes per coupling, 1 for
    FP8 E4M3), two full copies of the state for the double-buffered exchange
    (state_bytes per value, 2 for BF16) and the FP32 master state of its own spins."""
    lo, hi = max(row_ranges(n, world), key=lambda r: r[1] - r[0])
    rows = hi - lo
    j = rows * n * j_bytes
    s = 2 * replicas * n * state_bytes
    m = replicas * rows * master_bytes
    return {"rows": rows, "J": j, "state": s, "master": m, "total": j + s + m,
            "exchange_in_per_step": replicas * (n - rows) * state_bytes}


def check_partition(n: int, world: int) -> None:
    """The ranges cover [0, n) once, in order, with 128-aligned starts."""
    r = row_ranges(n, world)
    assert r[0][0] == 0 and r[-1][1] == n
    for (a, b), (c, d) in zip(r, r[1:]):
        assert b == c and a <= b
    assert all(lo % ROW_BLOCK == 0 for lo, hi in r if hi > lo)
    assert np.sum([hi - lo for lo, hi in r]) == n
