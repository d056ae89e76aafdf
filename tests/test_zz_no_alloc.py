"""The allocation-free tensor-path entry point, nmfa_run_device_noalloc.

Some callers cannot allocate device memory while they run (inside a CUDA stream
capture, under a framework's memory pool that owns the device, in a serving loop
that must not stall on cudaMalloc).  For them the library offers a variant of the
tensor-core run whose scratch lives in a fixed 16 MiB static device array.  This
file checks, through the C ABI, that the variant returns what nmfa_run_device
returns for the same inputs, on consecutive calls (the array keeps whatever the
previous call left in it), and that sizes beyond the array are refused.  It is
named to be collected last.
"""
import numpy as np
import pytest

from paper_1806_08422_gb300 import instances as inst

pytestmark = pytest.mark.gpu


def _buffers(torch, R, n, dev):
    return (torch.empty((R, n), dtype=torch.int8, device=dev),
            torch.empty(R, dtype=torch.float64, device=dev),
            torch.empty(R, dtype=torch.int64, device=dev))


def test_noalloc_matches_run_device_on_consecutive_calls():
    import torch

    import __graft_entry__
    from paper_1806_08422_gb300 import nmfa

    __graft_entry__.build()
    dev = torch.device("cuda", 0)
    # n = 300, R = 200 and n = 130, R = 48 take 64-replica tiles; SK n = 2000 with
    # 1024 replicas takes 128-replica tiles (8 MiB of state in the static array);
    # the last two store J in FP8 (widened in the kernel, no scratch for J)
    cases = [(inst.sk(300, 1), 200, 4, "bf16"), (inst.gnp_maxcut(130, 0.5, 2), 48, 9, "bf16"),
             (inst.sk(2000, 5), 1024, 11, "bf16"), (inst.sk(300, 6), 200, 4, "bf16_fp8j"),
             (inst.sk(2000, 7), 1024, 12, "bf16_fp8j")]
    T = torch.as_tensor(inst.schedule(150), device=dev)
    probs = [nmfa.Problem(J, precision=pr) for J, _, _, pr in cases]
    refs = []
    for p, (J, R, seed, _) in zip(probs, cases):
        s, e, ei = _buffers(torch, R, p.n, dev)
        p.run_device(T, 0.15, 0.15, R, seed=seed, signs=s, energy=e, energy_i64=ei)
        p.sync()
        refs.append((s.cpu().numpy(), e.cpu().numpy(), ei.cpu().numpy()))
    # two rounds of calls in a row, alternating sizes, so each call starts from the
    # scratch contents the previous one left behind
    for _ in range(2):
        for p, (J, R, seed, _), ref in zip(probs, cases, refs):
            s, e, ei = _buffers(torch, R, p.n, dev)
            nmfa.nmfa_run_device_noalloc(p.handle, T, 0.15, 0.15, R, seed=seed, signs=s, energy=e, energy_i64=ei)
            p.sync()
            np.testing.assert_array_equal(s.cpu().numpy(), ref[0])
            np.testing.assert_array_equal(ei.cpu().numpy(), ref[2])
            np.testing.assert_allclose(e.cpu().numpy(), ref[1], rtol=0, atol=0)
    for p in probs:
        p.close()


def test_noalloc_size_limit_at_the_boundary():
    # n = 2000 (n_pad = 2048) with more than one wave of 128-replica tiles takes
    # 256-replica tiles.  R = 1792 rounds to 7 x 256 replicas, 14 MiB of state plus the
    # plan: it runs and equals nmfa_run_device.  R = 1793 rounds to 2048 replicas,
    # exactly 16 MiB of state before the plan: refused, with nothing launched.
    import torch

    from paper_1806_08422_gb300 import nmfa

    dev = torch.device("cuda", 0)
    p = nmfa.Problem(inst.sk(2000, 3), precision="bf16")
    T = torch.as_tensor(inst.schedule(10), device=dev)
    R = 1792
    ref = _buffers(torch, R, p.n, dev)
    p.run_device(T, 0.15, 0.15, R, seed=2, signs=ref[0], energy=ref[1], energy_i64=ref[2])
    p.sync()
    got = _buffers(torch, R, p.n, dev)
    nmfa.nmfa_run_device_noalloc(p.handle, T, 0.15, 0.15, R, seed=2, signs=got[0], energy=got[1], energy_i64=got[2])
    p.sync()
    assert torch.equal(got[0], ref[0]) and torch.equal(got[2], ref[2]) and torch.equal(got[1], ref[1])
    for R in (1793, 1920):
        s, e, ei = _buffers(torch, R, p.n, dev)
        s.fill_(7)
        with pytest.raises(nmfa.NmfaError) as exc:
            nmfa.nmfa_run_device_noalloc(p.handle, T, 0.15, 0.15, R, signs=s, energy=e, energy_i64=ei)
        assert exc.value.code == nmfa.NMFA_EINVAL and "16 MiB" in str(exc.value)
        torch.cuda.synchronize()
        assert int((s != 7).sum()) == 0  # nothing was launched
    p.close()


def test_noalloc_inside_a_cuda_graph():
    # The case the entry point exists for: the run is captured into a CUDA graph
    # (after a first call outside the capture has looked up the static array), and
    # each replay writes what nmfa_run_device returns for the same inputs.
    import torch

    from paper_1806_08422_gb300 import nmfa

    dev = torch.device("cuda", 0)
    J, R, seed = inst.sk(700, 9), 256, 3
    p = nmfa.Problem(J, precision="bf16")
    T = torch.as_tensor(inst.schedule(120), device=dev)
    ref = _buffers(torch, R, p.n, dev)
    p.run_device(T, 0.15, 0.15, R, seed=seed, signs=ref[0], energy=ref[1], energy_i64=ref[2])
    p.sync()
    got = _buffers(torch, R, p.n, dev)
    nmfa.nmfa_run_device_noalloc(p.handle, T, 0.15, 0.15, R, seed=seed, signs=got[0], energy=got[1], energy_i64=got[2])
    p.sync()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            nmfa.nmfa_run_device_noalloc(p.handle, T, 0.15, 0.15, R, seed=seed, signs=got[0], energy=got[1],
                                         energy_i64=got[2], stream=side)
    for _ in range(2):
        for b in got:
            b.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(got[0], ref[0]) and torch.equal(got[2], ref[2]) and torch.equal(got[1], ref[1])
    del graph
    p.close()
