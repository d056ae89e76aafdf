"""The serving loop: requests of different sizes arriving while others run are
admitted, batched into shared persistent launches, and each request's result must
be the same as running it alone (attempt k uses noise stream k)."""
import numpy as np
import pytest

from paper_1806_08422_gb300 import instances as inst

pytestmark = pytest.mark.gpu


def _solo_best(J, T_np, R, seed, stream_id):
    import torch
    from paper_1806_08422_gb300 import nmfa
    dev = torch.device("cuda", 0)
    p = nmfa.Problem(J, precision="bf16_fp8j")
    e = torch.empty(R, dtype=torch.float64, device=dev)
    s = torch.empty((R, p.n), dtype=torch.int8, device=dev)
    p.run_device(torch.as_tensor(T_np, device=dev), 0.15, 0.15, R, seed=seed, stream_id=stream_id, signs=s, energy=e)
    p.sync()
    ee = e.cpu().numpy()
    k = int(np.argmin(ee))
    out = (float(ee[k]), s.cpu().numpy()[k].copy())
    p.close()
    return out


def test_server_results_equal_solo_runs():
    import time
    from paper_1806_08422_gb300 import nmfa
    T = inst.schedule(150)
    defs = [(inst.sk(200, 1), 64, 5), (inst.moebius(64), 128, 6), (inst.gnp_maxcut(700, 0.5, 2), 64, 7),
            (inst.sk(90, 3), 256, 8), (inst.sk(1300, 4), 64, 9)]
    srv = nmfa.nmfa_server_create(0, 2, 3)
    tickets = []
    for k, (J, R, seed) in enumerate(defs):
        # reachable target for the first three, unreachable for the rest (-> 3 attempts)
        target = 1e18 if k < 3 else -1e18
        tickets.append(nmfa.nmfa_server_submit(srv, J, T, R, target, seed=seed))
        time.sleep(0.01)  # staggered arrivals while earlier requests run
    nmfa.nmfa_server_drain(srv, 300.0)
    for k, ((J, R, seed), t) in enumerate(zip(defs, tickets)):
        res = nmfa.nmfa_server_poll(srv, t, n=J.shape[0])
        assert res["state"] == 3 and res["error"] == 0
        if k < 3:
            assert res["success"] == 1 and res["attempts"] == 1 and res["time_to_target"] > 0
            e, s = _solo_best(J, T, R, seed, 0)
            assert res["best_energy"] == e
            np.testing.assert_array_equal(res["best_signs"], s)
        else:
            assert res["success"] == 0 and res["attempts"] == 3
            best = min(_solo_best(J, T, R, seed, a)[0] for a in range(3))
            assert res["best_energy"] == best
    st = nmfa.nmfa_server_stats(srv)
    # nine runs in all (three requests once, two three times); whether two of them share
    # a launch depends on arrival timing here (the test below shows it deterministically)
    assert st["outstanding"] == 0 and 2 <= st["launches"] <= 9 and st["max_requests_per_launch"] >= 1, st
    nmfa.nmfa_server_destroy(srv)


def test_server_memory_budget_admits_in_order():
    from paper_1806_08422_gb300 import nmfa
    T = inst.schedule(40)
    srv = nmfa.nmfa_server_create(8 << 20, 1, 1)  # tight budget: about one request at a time
    tickets = [nmfa.nmfa_server_submit(srv, inst.sk(600, k), T, 64, 1e18, seed=k) for k in range(6)]
    nmfa.nmfa_server_drain(srv, 300.0)
    res = [nmfa.nmfa_server_poll(srv, t) for t in tickets]
    assert all(r["state"] == 3 and r["success"] == 1 for r in res)
    admits = [r["t_admit"] for r in res]
    assert admits == sorted(admits)
    import time
    for _ in range(200):  # the reaper thread releases memory shortly after completion
        if nmfa.nmfa_server_stats(srv)["mem_used"] == 0:
            break
        time.sleep(0.01)
    assert nmfa.nmfa_server_stats(srv)["mem_used"] == 0
    nmfa.nmfa_server_destroy(srv)


def test_request_arriving_mid_launch_starts_before_that_launch_ends():
    # Continuous batching: a long request A is on the GPU when B arrives; B starts in a
    # second launch on the SMs A leaves free, before A's launch has ended, and its
    # result is that of B run alone.  Requests batched behind a busy slot share a launch.
    import time
    from paper_1806_08422_gb300 import nmfa
    JA, JB = inst.sk(1000, 11), inst.sk(200, 12)
    TA, TB = inst.schedule(20000), inst.schedule(150)
    srv = nmfa.nmfa_server_create(0, 2, 1)
    ta = nmfa.nmfa_server_submit(srv, JA, TA, 128, 1e18, seed=3)
    for _ in range(2000):  # until A's launch is on the GPU
        if nmfa.nmfa_server_poll(srv, ta)["state"] == 2:
            break
        time.sleep(0.001)
    assert nmfa.nmfa_server_poll(srv, ta)["state"] == 2
    tb = nmfa.nmfa_server_submit(srv, JB, TB, 64, 1e18, seed=4)
    nmfa.nmfa_server_drain(srv, 300.0)
    ra, rb = nmfa.nmfa_server_poll(srv, ta), nmfa.nmfa_server_poll(srv, tb, n=200)
    assert ra["state"] == 3 and rb["state"] == 3 and ra["error"] == 0 and rb["error"] == 0
    assert rb["t_submit"] > ra["t_first_start"]
    assert rb["t_first_start"] < ra["t_done"], (rb["t_first_start"], ra["t_done"])
    e, s = _solo_best(JB, TB, 64, 4, 0)
    assert rb["best_energy"] == e
    np.testing.assert_array_equal(rb["best_signs"], s)
    nmfa.nmfa_server_destroy(srv)
    # one launch slot: requests that arrive while it is busy share the next launch
    srv = nmfa.nmfa_server_create(0, 1, 1)
    ts = [nmfa.nmfa_server_submit(srv, JA, inst.schedule(3000), 64, 1e18, seed=5)]
    ts += [nmfa.nmfa_server_submit(srv, inst.sk(150, 20 + k), TB, 64, 1e18, seed=6 + k) for k in range(4)]
    nmfa.nmfa_server_drain(srv, 300.0)
    assert all(nmfa.nmfa_server_poll(srv, t)["state"] == 3 for t in ts)
    st = nmfa.nmfa_server_stats(srv)
    assert st["launches"] < 5 and st["max_requests_per_launch"] >= 2, st
    nmfa.nmfa_server_destroy(srv)


def test_reruns_reuse_their_batch():
    # A request that misses its target reruns on the next noise stream; alone on the
    # server its reruns reuse the batch of its first attempt (no new plan), and its
    # best energy is the best of the solo runs on streams 0, 1, 2.
    from paper_1806_08422_gb300 import nmfa
    J, T = inst.sk(400, 14), inst.schedule(120)
    srv = nmfa.nmfa_server_create(0, 1, 3)
    t = nmfa.nmfa_server_submit(srv, J, T, 128, -1e18, seed=7)
    nmfa.nmfa_server_drain(srv, 300.0)
    res = nmfa.nmfa_server_poll(srv, t, n=400)
    assert res["state"] == 3 and res["error"] == 0 and res["attempts"] == 3 and res["success"] == 0
    st = nmfa.nmfa_server_stats(srv)
    assert st["launches"] == 3 and st["batches_reused"] == 2, st
    solo = [_solo_best(J, T, 128, 7, a) for a in range(3)]
    k = min(range(3), key=lambda a: solo[a][0])
    assert res["best_energy"] == solo[k][0]
    np.testing.assert_array_equal(res["best_signs"], solo[k][1])
    nmfa.nmfa_server_destroy(srv)
