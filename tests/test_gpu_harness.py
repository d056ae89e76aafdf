"""The evaluation harnesses on the GPU against the oracle.

Time to solution (Sec. III, Fig. 4: success probability of independent runs and the
TTS metric of Hamerly et al.) and the schedule calibration (Fig. 2 caption, Sec. II:
alpha = sigma = 0.15; Fig. 3: the 16-spin Moebius ladder with the schedule compressed
to 100 steps reaches its ground energy -20).  Success probabilities of the GPU runs
must fall inside the 95 % Wilson interval of the oracle's, runs paired by noise
stream (same seed, stream and replica index on both sides).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1806_08422_gb300 import instances as inst
from tests.helpers import wilson

pytestmark = pytest.mark.gpu


def test_tts_harness_success_probability_matches_oracle():
    from paper_1806_08422_gb300 import tts
    n, samples, t_f, seed = 20, 2000, 200, 1
    Js, energies, wall = tts.sample_energies("sk", n, samples, t_f, seed)
    assert len(Js) == tts.CLASSES["sk"] and wall > 0
    targets, agree = [], []
    for k, (J, ev) in enumerate(zip(Js, energies)):
        e0, _, _ = oracle.brute_force(J)
        targets.append(e0)
        assert ev.min() >= e0  # no sample beats the exhaustive ground state
        ref = oracle.run(J, inst.schedule(t_f), 0.15, 0.15, samples, seed=seed, stream=k)["energy_i64"]
        k_ref = int(np.sum(ref <= e0))
        lo, hi = wilson(k_ref, samples)
        p = float(np.mean(ev <= e0))
        assert lo <= p <= hi, (k, p, k_ref / samples, lo, hi)
        agree.append(float(np.mean((ev <= e0) == (ref <= e0))))
    # pairing: most runs reach the same outcome on both sides
    assert np.mean(agree) > 0.9, agree
    # the harness's own summary with these targets: p per instance and TTS99 from tau
    res = tts.run_class("sk", n, samples, t_f, seed, targets=targets)
    tau = res["tau_us"] * 1e-6
    for k, row in enumerate(res["per_instance"]):
        assert row["p"] == float(np.mean(energies[k] <= targets[k]))
        assert row["tts99_us"] == pytest.approx(tts.tts99(tau, row["p"]) * 1e6, rel=1e-12)
    ps = [r["p"] for r in res["per_instance"]]
    assert res["p"]["median"] == pytest.approx(float(np.median(ps)), rel=1e-12)
    assert 0.0 < res["p"]["q25"] <= res["p"]["median"] <= res["p"]["q75"] <= 1.0


def test_calibration_sweep_ladder_reaches_ground_state():
    from paper_1806_08422_gb300 import calibrate
    scheds = {k: calibrate.SCHEDULES[k] for k in ("default", "cold-end")}
    rows = calibrate.sweep(scheds, alphas=(0.15,), sigmas=(0.15,), n=256, replicas=64, t_f=200,
                           ladder_replicas=1000, seed=3)
    assert len(rows) == 2
    ladder = inst.moebius(16)
    for r in rows:
        # Fig. 3: the compressed 100-step schedule reaches the ladder's ground energy
        assert r["ladder16_p_ground"] >= 0.9, r
        assert r["ladder16_best"] == -20
        T = inst.schedule(100, r["knots"])
        ref = oracle.run(ladder, T, r["sigma"], r["alpha"], r["ladder16_replicas"], seed=r["seed"],
                         stream=r["ladder16_stream"])["energy_i64"]
        lo, hi = wilson(int(np.sum(ref <= -20)), len(ref))
        assert lo <= r["ladder16_p_ground"] <= hi, (r["schedule"], r["ladder16_p_ground"], lo, hi)
        # energy densities of the SK leg: no replica below the Parisi ground-state density
        assert -0.7633 * 1.05 < r["sk_best_density"] <= r["sk_mean_density"] < 0.0
        assert r["sk_mean_vs_table_I"] == pytest.approx(r["sk_mean_density"] / calibrate.TABLE_I_DENSITY - 1.0)
