"""Ragged batches on the tensor path: many instances (different sizes, replica
counts, schedules and noise streams) in one persistent launch, optionally replayed
from a CUDA graph.  Every instance's result must be bit-identical to running it
alone (batching invariance), and its Eq. (1) energies exact against the oracle."""
import numpy as np
import pytest

import oracle
from paper_1806_08422_gb300 import instances as inst

pytestmark = pytest.mark.gpu


def _dev():
    import torch
    return torch, torch.device("cuda", 0)


def _alone(p, T_dev, R, seed, stream_id):
    torch, dev = _dev()
    s = torch.empty((R, p.n), dtype=torch.int8, device=dev)
    e = torch.empty(R, dtype=torch.int64, device=dev)
    p.run_device(T_dev, 0.15, 0.15, R, seed=seed, stream_id=stream_id, signs=s, energy_i64=e)
    p.sync()
    return s.cpu().numpy(), e.cpu().numpy()


def _batch(problems, specs, options):
    torch, dev = _dev()
    from paper_1806_08422_gb300 import nmfa
    outs, jobs = [], []
    for p, (T_dev, R, seed, sid) in zip(problems, specs):
        s = torch.empty((R, p.n), dtype=torch.int8, device=dev)
        e = torch.empty(R, dtype=torch.int64, device=dev)
        outs.append((s, e))
        jobs.append(nmfa.make_job(T_dev, 0.15, 0.15, R, seed=seed, stream_id=sid, signs=s, energy_i64=e))
    b = nmfa.nmfa_batch_create([p.handle for p in problems], jobs, options)
    return b, outs


@pytest.mark.parametrize("options", [0, 1, 2, 4])
def test_batch_matches_alone(options):
    torch, dev = _dev()
    from paper_1806_08422_gb300 import nmfa
    defs = [(inst.sk(100, 1), 64, 30), (inst.sk(250, 2), 100, 60), (inst.gnp_maxcut(130, 0.5, 3), 33, 45),
            (inst.moebius(400), 200, 80), (inst.gnp_maxcut(1000, 0.5, 4), 64, 25), (inst.sk(700, 5), 130, 40)]
    problems, specs = [], []
    for k, (J, R, tf) in enumerate(defs):
        problems.append(nmfa.Problem(J, precision="bf16"))
        T = torch.as_tensor(inst.schedule(tf) * (1.0 + 0.1 * k), device=dev)
        specs.append((T, R, 100 + k, k % 3))
    alone = [_alone(p, *sp) for p, sp in zip(problems, specs)]
    b, outs = _batch(problems, specs, options)
    for rep in range(2):  # a second launch (graph replay) gives the same results
        nmfa.nmfa_batch_launch(b)
        nmfa.nmfa_batch_sync(b)
        for (s, e), (sa, ea), (J, R, tf) in zip(outs, alone, defs):
            np.testing.assert_array_equal(s.cpu().numpy(), sa)
            np.testing.assert_array_equal(e.cpu().numpy(), ea)
    info = nmfa.nmfa_batch_info(b)
    assert info["grid"] <= 152 and info["groups"] >= len(defs)
    nmfa.nmfa_batch_destroy(b)
    for (s, e), (J, R, tf) in zip(outs, defs):
        sg = s.cpu().numpy()
        for r in (0, R - 1):
            assert e.cpu().numpy()[r] == oracle.energy_i64(J, sg[r])
    for p in problems:
        p.close()


def test_tile_width_does_not_change_results():
    torch, dev = _dev()
    from paper_1806_08422_gb300 import nmfa
    J = inst.sk(300, 9)
    p = nmfa.Problem(J, precision="bf16")
    T = torch.as_tensor(inst.schedule(80), device=dev)
    res = []
    for options in (0, nmfa.NMFA_BATCH_BN64):
        b, outs = _batch([p], [(T, 256, 3, 1)], options)
        nmfa.nmfa_batch_launch(b)
        nmfa.nmfa_batch_sync(b)
        res.append(outs[0][0].cpu().numpy())
        nmfa.nmfa_batch_destroy(b)
    np.testing.assert_array_equal(res[0], res[1])
    assert nmfa.nmfa_autotune_bn(p.handle, 256) in (64, 128)
    p.close()


def test_ragged_c4_like_batch():
    # The ragged workload's shape (N ~ U[16, 1000], half SK, half G(N, 0.5)
    # MAX-CUT, 64 replicas each) at 64 instances and t_f = 200, under a graph
    # with autotuned tiles; sampled instances against their solo runs.
    torch, dev = _dev()
    from paper_1806_08422_gb300 import nmfa
    mix = inst.ragged_batch(64, seed=7)
    problems = [nmfa.Problem(J, precision="bf16") for _, _, J in mix]
    T = torch.as_tensor(inst.schedule(200), device=dev)
    specs = [(T, 64, 11, k) for k in range(len(mix))]
    b, outs = _batch(problems, specs, nmfa.NMFA_BATCH_GRAPH | nmfa.NMFA_BATCH_AUTOTUNE)
    nmfa.nmfa_batch_launch(b)
    nmfa.nmfa_batch_sync(b)
    for k in (0, 17, 33, 63):
        sa, ea = _alone(problems[k], *specs[k])
        np.testing.assert_array_equal(outs[k][0].cpu().numpy(), sa)
        np.testing.assert_array_equal(outs[k][1].cpu().numpy(), ea)
        J = mix[k][2]
        assert ea[5] == oracle.energy_i64(J, sa[5])
    nmfa.nmfa_batch_destroy(b)
    for p in problems:
        p.close()


# --------------------------------------------------------------------------
# FP8-E4M3 storage of J (exact for +-1 and small integers): the run must be
# bit-identical to the same instance stored in BF16, alone and inside a mixed
# batch (BF16 and FP8 instances, 64- and 128-replica tiles in one batch).
# --------------------------------------------------------------------------
def test_fp8_storage_matches_bf16():
    torch, dev = _dev()
    from paper_1806_08422_gb300 import nmfa
    J = inst.sk(500, 21)
    T = torch.as_tensor(inst.schedule(120), device=dev)
    a = nmfa.Problem(J, precision="bf16")
    f = nmfa.Problem(J, precision="bf16_fp8j")
    assert f.info()["device_bytes"] < a.info()["device_bytes"]
    sa, ea = _alone(a, T, 192, 4, 2)
    sf, ef = _alone(f, T, 192, 4, 2)
    np.testing.assert_array_equal(sa, sf)
    np.testing.assert_array_equal(ea, ef)
    for r in (0, 100):
        assert ef[r] == oracle.energy_i64(J, sf[r])
    a.close()
    f.close()


def _e4m3_exact_couplings(n, seed):
    # symmetric couplings drawn from exact E4M3 values: zero, subnormals (k 2^-9),
    # fractions, integers and the largest finite value
    vals = np.array([0.0, 2.0 ** -9, 3 * 2.0 ** -9, 7 * 2.0 ** -9, 2.0 ** -6, 0.0625, 0.5, 1.5, 1.0, 3.0, 7.5,
                     15.0, 26.0, 448.0])
    rng = np.random.default_rng(seed)
    U = np.triu(rng.choice(vals, size=(n, n)) * rng.choice([-1.0, 1.0], size=(n, n)), 1)
    return U + U.T


@pytest.mark.parametrize("n,R,tf", [(300, 192, 60), (1000, 64, 40), (2048, 2048, 20)])
def test_fp8_converted_in_kernel_matches_bf16(n, R, tf):
    # FP8-stored couplings reach the tensor cores through the kernel's converter warps
    # (E4M3 slice -> BF16 operand in shared memory; single runs, and batches with
    # NMFA_BATCH_FP8_IN_KERNEL); the run equals the same couplings stored in BF16 bit
    # for bit, for every exact E4M3 value; both storages take the same tile widths
    # (64, 64 and 256 here), and a forced 128 gives the same run.  A default batch
    # widens these sizes once to BF16 and equals them too.
    torch, dev = _dev()
    from paper_1806_08422_gb300 import nmfa
    J = _e4m3_exact_couplings(n, 40 + n)
    T = torch.as_tensor(inst.schedule(tf), device=dev)
    a = nmfa.Problem(J, precision="bf16")
    f = nmfa.Problem(J, precision="bf16_fp8j")
    assert f.info()["device_bytes"] < a.info()["device_bytes"]
    res = {}
    for name, p in (("bf16", a), ("fp8", f)):
        sb = torch.empty((R, n), dtype=torch.int8, device=dev)
        eb = torch.empty(R, dtype=torch.float64, device=dev)  # real-valued couplings: FP64 energies
        b = nmfa.nmfa_batch_create([p.handle], [nmfa.make_job(T, 0.15, 0.15, R, seed=9, stream_id=1, signs=sb,
                                                              energy=eb)], nmfa.NMFA_BATCH_FP8_IN_KERNEL)
        res[name + "_plan"] = nmfa.nmfa_batch_plan(b)
        nmfa.nmfa_batch_launch(b)
        nmfa.nmfa_batch_sync(b)
        nmfa.nmfa_batch_destroy(b)
        res[name + "_batch"] = (sb.cpu().numpy(), eb.cpu().numpy())
        s = torch.empty((R, n), dtype=torch.int8, device=dev)
        e = torch.empty(R, dtype=torch.float64, device=dev)
        p.run_device(T, 0.15, 0.15, R, seed=9, stream_id=1, signs=s, energy=e)
        p.sync()
        res[name] = (s.cpu().numpy(), e.cpu().numpy())
    assert res["fp8_plan"] == res["bf16_plan"] == [(256 if n == 2048 else 64, 1, 1)], res
    if n != 2048:
        sb = torch.empty((R, n), dtype=torch.int8, device=dev)
        eb = torch.empty(R, dtype=torch.float64, device=dev)
        b = nmfa.nmfa_batch_create([f.handle], [nmfa.make_job(T, 0.15, 0.15, R, seed=9, stream_id=1, signs=sb,
                                                              energy=eb)],
                                   nmfa.NMFA_BATCH_BN128 | nmfa.NMFA_BATCH_FP8_IN_KERNEL)
        assert nmfa.nmfa_batch_plan(b) == [(128, 1, 1)]
        nmfa.nmfa_batch_launch(b)
        nmfa.nmfa_batch_sync(b)
        nmfa.nmfa_batch_destroy(b)
        np.testing.assert_array_equal(sb.cpu().numpy(), res["bf16"][0])
        np.testing.assert_array_equal(eb.cpu().numpy(), res["bf16"][1])
    if n == 2048:
        assert res["fp8_plan"] == [(256, 1, 1)] == res["bf16_plan"]
    np.testing.assert_array_equal(res["fp8"][0], res["bf16"][0])
    np.testing.assert_array_equal(res["fp8"][1], res["bf16"][1])
    np.testing.assert_array_equal(res["fp8_batch"][0], res["fp8"][0])  # batched = alone
    sb = torch.empty((R, n), dtype=torch.int8, device=dev)
    eb = torch.empty(R, dtype=torch.float64, device=dev)
    b = nmfa.nmfa_batch_create([f.handle], [nmfa.make_job(T, 0.15, 0.15, R, seed=9, stream_id=1, signs=sb,
                                                          energy=eb)], 0)
    nmfa.nmfa_batch_launch(b)
    nmfa.nmfa_batch_sync(b)
    nmfa.nmfa_batch_destroy(b)
    np.testing.assert_array_equal(sb.cpu().numpy(), res["bf16"][0])
    np.testing.assert_array_equal(eb.cpu().numpy(), res["bf16"][1])
    for r in (0, R - 1):
        assert abs(res["fp8"][1][r] - oracle.energy(J, res["fp8"][0][r])) <= 1e-12 * np.abs(np.triu(J, 1)).sum()
    a.close()
    f.close()


def test_mixed_precision_and_width_batch():
    torch, dev = _dev()
    from paper_1806_08422_gb300 import nmfa
    defs = [(inst.sk(300, 31), "bf16", 64), (inst.gnp_maxcut(450, 0.5, 32), "bf16_fp8j", 160),
            (inst.sk(129, 33), "bf16_fp8j", 64), (inst.moebius(200), "bf16", 300)]
    problems = [nmfa.Problem(J, precision=pr) for J, pr, _ in defs]
    T = torch.as_tensor(inst.schedule(90), device=dev)
    specs = [(T, R, 50 + k, k) for k, (_, _, R) in enumerate(defs)]
    alone = [_alone(p, *sp) for p, sp in zip(problems, specs)]
    b, outs = _batch(problems, specs, nmfa.NMFA_BATCH_GRAPH)
    nmfa.nmfa_batch_launch(b)
    nmfa.nmfa_batch_sync(b)
    for (s, e), (sa, ea) in zip(outs, alone):
        np.testing.assert_array_equal(s.cpu().numpy(), sa)
        np.testing.assert_array_equal(e.cpu().numpy(), ea)
    nmfa.nmfa_batch_destroy(b)
    for p in problems:
        p.close()


def test_fp8_problems_widened_once_per_batch():
    # FP8-stored problems of n_pad <= 4096 are widened to BF16 once, at batch
    # creation: the batch holds a BF16 copy per problem (2 n_pad^2 bytes of its
    # workspace, one copy for two jobs of the same problem), their jobs share the BF16
    # launch of their tile width with BF16-stored problems, and every run equals its
    # solo run; an FP8 problem above n_pad = 4096 is read as stored (no copy).
    torch, dev = _dev()
    from paper_1806_08422_gb300 import nmfa
    T = torch.as_tensor(inst.schedule(30), device=dev)
    J1, J2 = inst.sk(1000, 91), inst.sk(300, 92)
    problems = [nmfa.Problem(J1, precision="bf16_fp8j"), nmfa.Problem(J1, precision="bf16"),
                nmfa.Problem(J2, precision="bf16_fp8j")]
    jobs = [(problems[0], (T, 256, 5, 0)), (problems[1], (T, 256, 5, 0)), (problems[0], (T, 256, 6, 1)),
            (problems[2], (T, 256, 7, 2))]
    alone = [_alone(p, *sp) for p, sp in jobs]
    # one tile width (64 replicas) for every job, so the launches are per storage only
    b, outs = _batch([p for p, _ in jobs], [sp for _, sp in jobs], nmfa.NMFA_BATCH_BN64)
    assert len(nmfa.nmfa_batch_plan(b)) == 1  # one launch: the FP8 jobs run on the BF16 kernel
    ws = nmfa.nmfa_batch_info(b)["workspace_bytes"]
    b_in, _ = _batch([p for p, _ in jobs], [sp for _, sp in jobs],
                     nmfa.NMFA_BATCH_BN64 | nmfa.NMFA_BATCH_FP8_IN_KERNEL)
    assert len(nmfa.nmfa_batch_plan(b_in)) == 2
    assert ws >= 2 * (1024 * 1024 + 384 * 384) + nmfa.nmfa_batch_info(b_in)["workspace_bytes"] - (1 << 20)
    nmfa.nmfa_batch_destroy(b_in)
    nmfa.nmfa_batch_launch(b)
    nmfa.nmfa_batch_sync(b)
    for (s, e), (sa, ea) in zip(outs, alone):
        np.testing.assert_array_equal(s.cpu().numpy(), sa)
        np.testing.assert_array_equal(e.cpu().numpy(), ea)
    np.testing.assert_array_equal(outs[0][0].cpu().numpy(), outs[1][0].cpu().numpy())  # FP8 = BF16 storage
    nmfa.nmfa_batch_destroy(b)
    big = nmfa.Problem(inst.sk(4200, 93), precision="bf16_fp8j")
    b, outs = _batch([big], [(T, 64, 8, 0)], 0)
    b_in, _ = _batch([big], [(T, 64, 8, 0)], nmfa.NMFA_BATCH_FP8_IN_KERNEL)
    assert nmfa.nmfa_batch_info(b)["workspace_bytes"] == nmfa.nmfa_batch_info(b_in)["workspace_bytes"]
    nmfa.nmfa_batch_destroy(b_in)
    nmfa.nmfa_batch_launch(b)
    nmfa.nmfa_batch_sync(b)
    s, e = _alone(big, T, 64, 8, 0)
    np.testing.assert_array_equal(outs[0][0].cpu().numpy(), s)
    np.testing.assert_array_equal(outs[0][1].cpu().numpy(), e)
    nmfa.nmfa_batch_destroy(b)
    for p in problems + [big]:
        p.close()


def test_withheld_tile_times_out_and_the_device_recovers():
    # Failure detection without a GPU fault: one row-block tile of a group is left
    # out of the plan, so its peers wait for an epoch flag that nothing sets.  Their
    # bounded waits give up, the launch reports NMFA_ETIMEOUT, and the next launch
    # on the same device gives the same results as before.
    torch, dev = _dev()
    from paper_1806_08422_gb300 import nmfa
    J = inst.sk(300, 41)
    p = nmfa.Problem(J, precision="bf16")
    T_dev = torch.as_tensor(inst.schedule(20), device=dev)
    ref_s, ref_e = _alone(p, T_dev, 96, 3, 1)
    b, _ = _batch([p], [(T_dev, 96, 3, 1)], nmfa.NMFA_BATCH_DEBUG_WITHHOLD_TILE)
    nmfa.nmfa_batch_launch(b)
    with pytest.raises(nmfa.NmfaError) as ei:
        nmfa.nmfa_batch_sync(b)
    assert ei.value.code == nmfa.NMFA_ETIMEOUT
    nmfa.nmfa_batch_destroy(b)
    s, e = _alone(p, T_dev, 96, 3, 1)
    np.testing.assert_array_equal(s, ref_s)
    np.testing.assert_array_equal(e, ref_e)
    b, outs = _batch([p], [(T_dev, 96, 3, 1)], 0)
    nmfa.nmfa_batch_launch(b)
    nmfa.nmfa_batch_sync(b)
    np.testing.assert_array_equal(outs[0][0].cpu().numpy(), ref_s)
    nmfa.nmfa_batch_destroy(b)
    p.close()


def test_256_replica_tiles_match_64_replica_tiles():
    # A run whose 128-replica tiles would need two waves takes 256-replica tiles
    # (one accumulator, bias written after the update); its signs and Eq. (1)
    # energies are bit-identical to the same run on 64-replica tiles.
    torch, dev = _dev()
    from paper_1806_08422_gb300 import nmfa
    n, R = 2048, 2048
    J = inst.sk(n, 52)
    p = nmfa.Problem(J, precision="bf16")
    T_dev = torch.as_tensor(inst.schedule(25), device=dev)
    b, outs = _batch([p], [(T_dev, R, 6, 2)], 0)
    assert nmfa.nmfa_batch_info(b)["groups"] == R // 256
    nmfa.nmfa_batch_launch(b)
    nmfa.nmfa_batch_sync(b)
    s256, e256 = outs[0][0].cpu().numpy(), outs[0][1].cpu().numpy()
    nmfa.nmfa_batch_destroy(b)
    b, outs = _batch([p], [(T_dev, R, 6, 2)], nmfa.NMFA_BATCH_BN64)
    assert nmfa.nmfa_batch_info(b)["groups"] == R // 64
    nmfa.nmfa_batch_launch(b)
    nmfa.nmfa_batch_sync(b)
    np.testing.assert_array_equal(outs[0][0].cpu().numpy(), s256)
    np.testing.assert_array_equal(outs[0][1].cpu().numpy(), e256)
    nmfa.nmfa_batch_destroy(b)
    s, e = _alone(p, T_dev, R, 6, 2)
    np.testing.assert_array_equal(s, s256)
    for r in (0, 777, R - 1):
        assert e256[r] == oracle.energy_i64(J, s256[r])
    p.close()


@pytest.mark.parametrize("n,R,storage", [(300, 200, "bf16"), (1000, 300, "bf16_fp8j"), (129, 64, "bf16")])
def test_forced_256_replica_tiles_match_128_replica_tiles(n, R, storage):
    # NMFA_BATCH_BN256 forces 256-replica tiles (one accumulator; short K sweeps of
    # one to eight slices; a replica block that is partly padding): signs and Eq. (1)
    # energies equal those of 128-replica tiles bit for bit, and the energies are
    # exact against the oracle.
    torch, dev = _dev()
    from paper_1806_08422_gb300 import nmfa
    J = inst.sk(n, 90 + n)
    p = nmfa.Problem(J, precision=storage)
    T = torch.as_tensor(inst.schedule(40), device=dev)
    res = {}
    for name, options, bn in (("bn256", nmfa.NMFA_BATCH_BN256, 256), ("bn128", nmfa.NMFA_BATCH_BN128, 128)):
        b, outs = _batch([p], [(T, R, 5, 2)], options)
        assert nmfa.nmfa_batch_plan(b) == [(bn, 1, 1)], (name, nmfa.nmfa_batch_plan(b))
        nmfa.nmfa_batch_launch(b)
        nmfa.nmfa_batch_sync(b)
        res[name] = (outs[0][0].cpu().numpy(), outs[0][1].cpu().numpy())
        nmfa.nmfa_batch_destroy(b)
    np.testing.assert_array_equal(res["bn256"][0], res["bn128"][0])
    np.testing.assert_array_equal(res["bn256"][1], res["bn128"][1])
    for r in (0, R - 1):
        assert res["bn256"][1][r] == oracle.energy_i64(J, res["bn256"][0][r])
    p.close()


@pytest.mark.parametrize("options", [0, 1])
def test_variant_launches_side_by_side_or_in_turn(options):
    # A batch with several tile variants runs one persistent launch per variant: side
    # by side when all their CTAs fit the SMs together (first batch: a 64-, a 128- and
    # an FP8 128-replica launch of a few tiles each), one after the other when they
    # do not (second batch: 256-replica tiles on 128 CTAs beside 128-replica tiles
    # on 64).  Every run equals its solo run either way, with and without a graph.
    torch, dev = _dev()
    from paper_1806_08422_gb300 import nmfa
    T = torch.as_tensor(inst.schedule(40), device=dev)
    for defs in ([(inst.sk(300, 81), "bf16", 64), (inst.sk(1500, 82), "bf16", 256), (inst.sk(1500, 83), "bf16_fp8j", 256)],
                 [(inst.sk(2048, 84), "bf16", 2048), (inst.sk(2048, 85), "bf16", 512)]):
        problems = [nmfa.Problem(J, precision=pr) for J, pr, _ in defs]
        specs = [(T, R, 60 + k, k) for k, (_, _, R) in enumerate(defs)]
        alone = [_alone(p, *sp) for p, sp in zip(problems, specs)]
        b, outs = _batch(problems, specs, options | nmfa.NMFA_BATCH_FP8_IN_KERNEL)
        assert len(nmfa.nmfa_batch_plan(b)) == len(defs)
        nmfa.nmfa_batch_launch(b)
        nmfa.nmfa_batch_sync(b)
        for (s, e), (sa, ea) in zip(outs, alone):
            np.testing.assert_array_equal(s.cpu().numpy(), sa)
            np.testing.assert_array_equal(e.cpu().numpy(), ea)
        nmfa.nmfa_batch_destroy(b)
        for p in problems:
            p.close()


@pytest.mark.parametrize("options", [0, 1])
def test_set_stream_ids_reruns_with_fresh_noise(options):
    # A created batch is re-targeted at other noise streams (plan and workspace kept,
    # descriptors uploaded again): each execution equals the solo runs on the streams
    # it was given, for jobs on different tile widths, with and without a CUDA graph.
    torch, dev = _dev()
    from paper_1806_08422_gb300 import nmfa
    problems = [nmfa.Problem(inst.sk(300, 61), precision="bf16"), nmfa.Problem(inst.sk(2000, 62), precision="bf16")]
    T = torch.as_tensor(inst.schedule(50), device=dev)
    specs = [(T, 64, 21, 0), (T, 512, 22, 0)]
    b, outs = _batch(problems, specs, options)
    assert len(nmfa.nmfa_batch_plan(b)) == 2
    for ids in ([0, 0], [1, 2], [2, 1]):
        if ids != [0, 0]:
            nmfa.nmfa_batch_set_stream_ids(b, ids)
        nmfa.nmfa_batch_launch(b)
        nmfa.nmfa_batch_sync(b)
        for p, (Td, R, seed, _), sid, (s, e) in zip(problems, specs, ids, outs):
            sa, ea = _alone(p, Td, R, seed, sid)
            np.testing.assert_array_equal(s.cpu().numpy(), sa)
            np.testing.assert_array_equal(e.cpu().numpy(), ea)
    with pytest.raises(RuntimeError):
        nmfa.nmfa_batch_set_stream_ids(b, [1])
    nmfa.nmfa_batch_destroy(b)
    for p in problems:
        p.close()


# --------------------------------------------------------------------------
# CTA pairs (NMFA_BATCH_PAIR128): 128-replica tiles of problems whose row blocks pair
# up run as clusters of two CTAs sharing one cta_group::2 MMA (M = 256).  One-CTA
# tiles of every width sweep K from their own row block, so 128- and 64-replica tiles
# give bit-identical results; a pair sweeps K from its even row block for both of its
# tiles, so its runs agree with one-CTA runs to the BF16 path's rounding.  Pair runs
# are independent of what else the batch holds, and their energies are exact.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n,R", [(256, 128), (1000, 384), (2000, 1024)])
def test_cta_pairs_match_single_cta_tiles(n, R):
    torch, dev = _dev()
    from paper_1806_08422_gb300 import nmfa
    J = inst.sk(n, 70 + n)
    p = nmfa.Problem(J, precision="bf16")
    other = nmfa.Problem(inst.sk(300, 71), precision="bf16")
    T = torch.as_tensor(inst.schedule(60), device=dev)
    res = {}
    for name, options, plan in (("pair", nmfa.NMFA_BATCH_PAIR128, [(128, 2, 2)]),
                                ("one", nmfa.NMFA_BATCH_BN128, [(128, 1, 1)]), ("bn64", nmfa.NMFA_BATCH_BN64, [(64, 1, 1)])):
        b, outs = _batch([p], [(T, R, 8, 3)], options)
        assert nmfa.nmfa_batch_plan(b) == plan, (name, nmfa.nmfa_batch_plan(b))
        nmfa.nmfa_batch_launch(b)
        nmfa.nmfa_batch_sync(b)
        res[name] = (outs[0][0].cpu().numpy(), outs[0][1].cpu().numpy())
        nmfa.nmfa_batch_destroy(b)
    # one-CTA widths: bit for bit, and equal to the default run alone
    np.testing.assert_array_equal(res["one"][0], res["bn64"][0])
    np.testing.assert_array_equal(res["one"][1], res["bn64"][1])
    s, e = _alone(p, T, R, 8, 3)
    np.testing.assert_array_equal(s, res["one"][0])
    # pairs: the same run beside another job is bit-identical; exact energies; the
    # energy distribution agrees with the one-CTA run's
    b, outs = _batch([p, other], [(T, R, 8, 3), (T, 64, 9, 0)], nmfa.NMFA_BATCH_PAIR128)
    nmfa.nmfa_batch_launch(b)
    nmfa.nmfa_batch_sync(b)
    np.testing.assert_array_equal(outs[0][0].cpu().numpy(), res["pair"][0])
    np.testing.assert_array_equal(outs[0][1].cpu().numpy(), res["pair"][1])
    nmfa.nmfa_batch_destroy(b)
    for r in (0, R // 2 + 1, R - 1):
        assert res["pair"][1][r] == oracle.energy_i64(J, res["pair"][0][r])
    mp, mo = float(res["pair"][1].mean()), float(res["one"][1].mean())
    assert abs(mp - mo) <= 0.02 * abs(mo), (mp, mo)
    p.close()
    other.close()
