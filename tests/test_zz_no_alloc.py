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
    cases = [(inst.sk(300, 1), 200, 4), (inst.gnp_maxcut(130, 0.5, 2), 48, 9)]
    T = torch.as_tensor(inst.schedule(150), device=dev)
    probs = [nmfa.Problem(J, precision="bf16") for J, _, _ in cases]
    refs = []
    for p, (J, R, seed) in zip(probs, cases):
        s, e, ei = _buffers(torch, R, p.n, dev)
        p.run_device(T, 0.15, 0.15, R, seed=seed, signs=s, energy=e, energy_i64=ei)
        p.sync()
        refs.append((s.cpu().numpy(), e.cpu().numpy(), ei.cpu().numpy()))
    # two rounds of calls in a row, alternating sizes, so each call starts from the
    # scratch contents the previous one left behind
    for _ in range(2):
        for p, (J, R, seed), ref in zip(probs, cases, refs):
            s, e, ei = _buffers(torch, R, p.n, dev)
            nmfa.nmfa_run_device_noalloc(p.handle, T, 0.15, 0.15, R, seed=seed, signs=s, energy=e, energy_i64=ei)
            p.sync()
            np.testing.assert_array_equal(s.cpu().numpy(), ref[0])
            np.testing.assert_array_equal(ei.cpu().numpy(), ref[2])
            np.testing.assert_allclose(e.cpu().numpy(), ref[1], rtol=0, atol=0)
    for p in probs:
        p.close()


def test_noalloc_refuses_sizes_beyond_the_static_buffer():
    import torch

    from paper_1806_08422_gb300 import nmfa

    dev = torch.device("cuda", 0)
    p = nmfa.Problem(inst.sk(2000, 3), precision="bf16")
    R = 2048  # 4 * 2048 * 2048 bytes of state plus flags exceed 16 MiB
    s, e, ei = _buffers(torch, R, p.n, dev)
    s.fill_(7)
    T = torch.as_tensor(inst.schedule(10), device=dev)
    with pytest.raises(nmfa.NmfaError) as exc:
        nmfa.nmfa_run_device_noalloc(p.handle, T, 0.15, 0.15, R, signs=s, energy=e, energy_i64=ei)
    assert exc.value.code == nmfa.NMFA_EINVAL and "16 MiB" in str(exc.value)
    torch.cuda.synchronize()
    assert int((s != 7).sum()) == 0  # nothing was launched
    p.close()
