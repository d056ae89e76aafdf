"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test names the passage of arXiv 1806.08422 it checks.  None of them re-types
the oracle's own formula: they use published known-answer vectors, closed forms,
exhaustive search, invariances, and special cases that reduce to textbook loops.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_1806_08422_gb300 import instances as inst

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(x, 16) for x in line.split()])
    return rows


# --------------------------------------------------------------------------
# Noise stream (Algorithm 1's field: N(0, sigma); Sec. II: sigma is a standard
# deviation).  Philox4x32-10 from its published known-answer vectors.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("row", _kat_rows())
def test_philox_known_answers(row):
    out = oracle.philox4x32_10(row[:4], row[4:6])
    assert [int(x) for x in out] == row[6:]


def test_uniform_grid_endpoints():
    assert oracle.uniform(0) == 2.0 ** -24
    assert oracle.uniform(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert oracle.uniform(1 << 9) == 3 * 2.0 ** -24  # next odd multiple
    # exactly representable in binary32
    for w in (0, 12345 << 9, 0xFFFFFFFF, 0x80000000):
        u = oracle.uniform(w)
        assert float(np.float32(u)) == u


def test_gauss_is_standard_normal():
    z = np.array([oracle.gauss(7, 3, r, t, i) for r in range(8) for t in range(25)
                  for i in range(100)])
    assert abs(z.mean()) < 0.05
    assert abs(z.std() - 1.0) < 0.03
    assert stats.kstest(z, "norm").pvalue > 1e-3


def test_gauss_streams_differ():
    a = [oracle.gauss(0, 0, 0, 0, i) for i in range(64)]
    for args in [(1, 0, 0, 0), (0, 1, 0, 0), (0, 0, 1, 0), (0, 0, 0, 1), (0, 0, 4, 0)]:
        b = [oracle.gauss(args[0], args[1], args[2], args[3], i) for i in range(64)]
        assert a != b


# --------------------------------------------------------------------------
# Row norms (Algorithm 1's field; Sec. II: the root mean square of the terms
# acting on a spin).  Closed forms for the paper's instance classes.
# --------------------------------------------------------------------------
def test_row_norms_closed_forms():
    n = 50
    np.testing.assert_array_equal(oracle.row_norms(inst.sk(n, 1)), np.full(n, math.sqrt(n - 1)))
    J = inst.gnp_maxcut(n, 0.5, 2)
    np.testing.assert_allclose(oracle.row_norms(J), np.sqrt(J.sum(1)), rtol=0, atol=1e-14)
    h = inst.random_fields(n, 2.0, 3)
    np.testing.assert_allclose(oracle.row_norms(inst.moebius(n), h),
                               np.sqrt(h ** 2 + 3.0), rtol=1e-15)


# --------------------------------------------------------------------------
# Step 1 of Algorithm 1 from s = 0:  s_1 = -alpha tanh((h_i/d_i + sigma z)/T_1)
# (Algorithm 1).  With sigma = 0 this is a closed form; with sigma > 0 the
# recovered z must be the stream's draw for (r, t=0, i) and standard normal.
# --------------------------------------------------------------------------
def test_step1_closed_form_sigma0():
    n, R = 40, 3
    J = inst.sk(n, 5)
    h = inst.random_fields(n, 1.5, 6)
    T = np.array([0.7, 0.3])
    out = oracle.run(J, T[:1], sigma=0.0, alpha=0.15, replicas=R, h=h, want_state=True)
    d = np.sqrt(h ** 2 + (n - 1))
    expect = -0.15 * np.tanh((h / d) / 0.7)
    for r in range(R):
        np.testing.assert_allclose(out["state"][r], expect, rtol=1e-14, atol=1e-16)


def test_step1_recovers_noise_stream():
    n, R, alpha, sigma, T0 = 64, 12, 0.15, 0.15, 0.9
    J = inst.sk(n, 8)
    h = inst.random_fields(n, 0.5, 9)
    out = oracle.run(J, [T0, 0.1], sigma, alpha, R, seed=11, stream=4, h=h, want_state=False,
                     want_phi=True)
    # two steps: the last Phi belongs to step t = 1 (0-based); rerun one step for t=0
    one = oracle.run(J, [T0], sigma, alpha, R, seed=11, stream=4, h=h, want_state=True)
    d = np.sqrt(h ** 2 + (n - 1))
    z = (T0 * np.arctanh(-one["state"] / alpha) - h / d) / sigma
    zref = np.array([[oracle.gauss(11, 4, r, 0, i) for i in range(n)] for r in range(R)])
    np.testing.assert_allclose(z, zref, rtol=0, atol=1e-9)
    assert stats.kstest(z.ravel(), "norm").pvalue > 1e-3
    assert abs(z.std() - 1.0) < 0.1  # a variance reading (sigma^2) would give 0.15
    assert out["phi"].shape == (R, n)


# --------------------------------------------------------------------------
# Invariants of Algorithm 1: |s_i(t)| <= 1 - (1 - alpha)^t from s = 0, since
# |tanh| < 1 and each step is a convex combination (Algorithm 1's alpha-mix).
# --------------------------------------------------------------------------
def test_state_bound():
    n, alpha = 30, 0.15
    J = inst.sk(n, 12)
    T = inst.schedule(60)
    for tf in (1, 2, 5, 20, 60):
        st = oracle.run(J, T[:tf], 0.15, alpha, 6, seed=3, want_state=True)["state"]
        assert np.all(np.abs(st) <= 1.0 - (1.0 - alpha) ** tf + 1e-15)


# --------------------------------------------------------------------------
# High temperature (Algorithm 1 with T_t huge): |tanh x| <= |x| and, by
# Cauchy-Schwarz, (|h_i| + sum_j |J_ij| |s_j|) / d_i <= sqrt(n) for |s_j| <= 1, so
# |Phi_i| <= sqrt(n) + sigma |z| and every state stays below (sqrt(n) + sigma z_max) / T
# (the uniforms of the stream are >= 2^-24, so |z| <= sqrt(48 ln 2)).  The state is
# O(1/T): it shrinks tenfold when T grows tenfold.
# --------------------------------------------------------------------------
def test_high_temperature_state_is_order_one_over_T():
    n, R, tf, sigma = 40, 6, 30, 0.15
    J = inst.sk(n, 21)
    h = inst.random_fields(n, 0.5, 22)
    zmax = np.sqrt(48.0 * np.log(2.0))
    peaks = []
    for Tval in (1e4, 1e5, 1e6):
        st = oracle.run(J, [Tval] * tf, sigma, 0.15, R, seed=4, h=h, want_state=True)["state"]
        assert np.all(np.abs(st) <= (np.sqrt(n) + sigma * zmax) / Tval)
        peaks.append(np.abs(st).max())
    assert 9.0 < peaks[0] / peaks[1] < 11.0 and 9.0 < peaks[1] / peaks[2] < 11.0


# --------------------------------------------------------------------------
# Spin-flip symmetry at h = 0: negating every noise draw negates the whole
# trajectory exactly (tanh odd, coupling linear, IEEE negation exact), so the
# signs flip and Eq. (1) is unchanged.
# --------------------------------------------------------------------------
def test_noise_negation_symmetry():
    n, R = 48, 5
    J = inst.sk(n, 13)
    T = inst.schedule(80)
    a = oracle.run(J, T, 0.15, 0.15, R, seed=5, want_state=True)
    b = oracle.run(J, T, 0.15, 0.15, R, seed=5, noise_sign=-1, want_state=True)
    np.testing.assert_array_equal(a["state"], -b["state"])
    nz = a["state"] != 0
    np.testing.assert_array_equal(a["signs"][nz], -b["signs"][nz])
    np.testing.assert_array_equal(a["energy_i64"], b["energy_i64"])


def test_sigma0_zero_fixed_point_and_tiebreak():
    n = 20
    J = inst.sk(n, 14)
    out = oracle.run(J, inst.schedule(30), 0.0, 0.15, 2, want_state=True)
    assert np.all(out["state"] == 0.0)
    assert np.all(out["signs"] == 1)  # s = 0 reads out as +1
    assert out["energy_i64"][0] == int(np.triu(J, 1).sum())


def test_sigma0_negation_of_s0_and_h():
    n, R = 36, 3
    J = inst.sk(n, 15)
    T = inst.schedule(50)
    rng = np.random.default_rng(0)
    s0 = rng.uniform(-1, 1, size=(R, n))
    a = oracle.run(J, T, 0.0, 0.15, R, s0=s0, want_state=True)["state"]
    b = oracle.run(J, T, 0.0, 0.15, R, s0=-s0, want_state=True)["state"]
    np.testing.assert_array_equal(a, -b)
    h = inst.random_fields(n, 1.0, 16)
    c = oracle.run(J, T, 0.0, 0.15, R, h=h, want_state=True)["state"]
    e = oracle.run(J, T, 0.0, 0.15, R, h=-h, want_state=True)["state"]
    np.testing.assert_array_equal(c, -e)
    assert np.any(c != 0)


# --------------------------------------------------------------------------
# Special cases that reduce to textbook routines (Sec. II: NMFA generalises
# mean-field annealing, Bilbro et al. 1989).
#   sigma = 0, alpha = 1: synchronous deterministic mean-field annealing
#       s <- -tanh((J s + h) / (d T_t)), written here with a BLAS product.
#   sigma = 0, alpha = 1, T -> 0: zero-temperature synchronous sign dynamics
#       s <- -sgn(J s + h), checked in exact integer arithmetic.
# --------------------------------------------------------------------------
def test_mean_field_annealing_special_case():
    n, R, steps = 60, 4, 25
    J = inst.sk(n, 17)
    h = inst.random_fields(n, 0.8, 18)
    T = np.geomspace(3.0, 0.5, steps)
    rng = np.random.default_rng(1)
    s0 = rng.uniform(-0.5, 0.5, size=(R, n))
    got = oracle.run(J, T, 0.0, 1.0, R, h=h, s0=s0, want_state=True)["state"]
    d = np.sqrt(h ** 2 + (J ** 2).sum(1))
    s = s0.copy()
    for t in range(steps):
        s = -np.tanh(((s @ J.T) + h) / d / T[t])
    np.testing.assert_allclose(got, s, rtol=0, atol=1e-10)


def test_zero_temperature_sign_dynamics():
    n, R, steps = 40, 6, 12
    J = inst.sk(n, 19)
    Ji = J.astype(np.int64)
    rng = np.random.default_rng(2)
    s0 = rng.choice([-1.0, 1.0], size=(R, n))
    got = oracle.run(J, np.full(steps, 1e-300), 0.0, 1.0, R, s0=s0, want_state=True)["state"]
    s = s0.astype(np.int64)
    for _ in range(steps):
        s = -np.sign(s @ Ji.T)
    np.testing.assert_array_equal(got, s.astype(np.float64))


def test_alpha_mix_memory_over_several_steps():
    # Algorithm 1 with the paper's alpha = 0.15 < 1 (Sec. II): the (1 - alpha) s memory
    # term carried over twelve steps, against an independent loop that forms every
    # field with compensated sums (math.fsum) and applies the update with numpy.  Once
    # with sigma = 0 and once with sigma = 0.15, the draws given to the loop as inputs
    # (the stream itself is pinned by the known-answer and step-1 tests above).
    n, R, steps, alpha = 40, 3, 12, 0.15
    J = inst.sk(n, 23)
    h = inst.random_fields(n, 0.4, 24)
    T = np.geomspace(4.0, 2.0, steps)
    s0 = np.random.default_rng(25).uniform(-0.6, 0.6, size=(R, n))
    d = np.array([math.sqrt(math.fsum([h[i] ** 2] + [J[i, j] ** 2 for j in range(n)])) for i in range(n)])
    for sigma in (0.0, 0.15):
        got = oracle.run(J, T, sigma, alpha, R, seed=9, stream=2, h=h, s0=s0, want_state=True)["state"]
        s = s0.copy()
        for t in range(steps):
            phi = np.empty((R, n))
            for r in range(R):
                for i in range(n):
                    phi[r, i] = math.fsum([h[i]] + [J[i, j] * s[r, j] for j in range(n)]) / d[i]
                    phi[r, i] += sigma * oracle.gauss(9, 2, r, t, i)
            s = alpha * -np.tanh(phi / T[t]) + (1.0 - alpha) * s
        np.testing.assert_allclose(got, s, rtol=0, atol=1e-12)
        # the memory term matters here: alpha = 1 (no memory) lands far away
        nomem = oracle.run(J, T, sigma, 1.0, R, seed=9, stream=2, h=h, s0=s0, want_state=True)["state"]
        assert np.abs(nomem - s).max() > 0.1


def test_run_continues_from_its_state():
    # Algorithm 1's loop carries only the state from one step to the next, and the
    # draw of step t depends on t alone: k steps, then the remaining steps from that
    # state with the step index continued, equal the whole run bit for bit.
    n, R = 50, 5
    J = inst.sk(n, 26)
    h = inst.random_fields(n, 0.3, 27)
    T = inst.schedule(40)
    whole = oracle.run(J, T, 0.15, 0.15, R, seed=4, stream=3, h=h, want_state=True)["state"]
    part = oracle.run(J, T[:17], 0.15, 0.15, R, seed=4, stream=3, h=h, want_state=True)["state"]
    rest = oracle.run(J, T[17:], 0.15, 0.15, R, seed=4, stream=3, h=h, s0=part, want_state=True, t_first=17)
    np.testing.assert_array_equal(rest["state"], whole)
    # without the continued step index the draws repeat steps 0.. and the runs differ
    wrong = oracle.run(J, T[17:], 0.15, 0.15, R, seed=4, stream=3, h=h, s0=part, want_state=True)["state"]
    assert np.abs(wrong - whole).max() > 1e-3


def test_coupling_product_against_compensated_sum():
    # Algorithm 1's field with sigma = 0 from a given state: Phi = (h + J s)/d.
    n, R = 70, 3
    J = inst.random_real_couplings(n, 20, density=0.6)
    h = inst.random_fields(n, 0.3, 21)
    rng = np.random.default_rng(3)
    s0 = rng.uniform(-1, 1, size=(R, n))
    phi = oracle.run(J, [1.0], 0.0, 0.15, R, h=h, s0=s0, want_phi=True)["phi"]
    for r in range(R):
        for i in range(n):
            num = math.fsum([h[i]] + [J[i, j] * s0[r, j] for j in range(n)])
            den = math.sqrt(math.fsum([h[i] ** 2] + [J[i, j] ** 2 for j in range(n)]))
            assert abs(phi[r, i] - num / den) <= 1e-13 * (1 + abs(num / den))


def test_isolated_spin_has_zero_field():
    # d_i = 0 (no couplings and no field): the normalised field reads as 0,
    # so only the noise acts.
    J = inst.moebius(8)
    J = np.pad(J, ((0, 1), (0, 1)))  # spin 8 is isolated
    out = oracle.run(J, [0.5], 0.0, 0.15, 2, want_phi=True, want_state=True)
    assert np.all(out["phi"][:, 8] == 0.0)
    assert np.all(np.isfinite(out["state"]))


# --------------------------------------------------------------------------
# Eq. (1) energy and readout.
# --------------------------------------------------------------------------
def _golden_closed_forms():
    rows = []
    with open(os.path.join(GOLDEN, "closed_form_ground_energies.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                g, n, e, c = line.split()
                rows.append((g, int(n), int(e), int(c)))
    return rows


def _graph(g, n):
    return {"complete": inst.complete, "ring": inst.ring, "moebius": inst.moebius}[g](n)


@pytest.mark.parametrize("row", [r for r in _golden_closed_forms() if r[1] <= 20])
def test_brute_force_matches_closed_form(row):
    g, n, e_min, cut = row
    J = _graph(g, n)
    e, best, count = oracle.brute_force(J)
    assert e == e_min
    assert oracle.energy_i64(J, best) == e_min
    n_edges = int(np.triu(J, 1).sum())
    assert (n_edges - e_min) // 2 == cut  # MAX-CUT value, Table I's convention


def test_ring_has_two_ground_states():
    e, best, count = oracle.brute_force(inst.ring(10))
    assert count == 2


def test_complete_graph_energy_closed_form():
    rng = np.random.default_rng(4)
    for n in (3, 8, 13):
        J = inst.complete(n)
        for _ in range(5):
            s = rng.choice([-1, 1], size=n).astype(np.int8)
            M = int(s.sum())
            assert oracle.energy_i64(J, s) == (M * M - n) // 2
            assert oracle.energy(J, s) == (M * M - n) / 2


def test_energy_gauge_and_permutation_invariance():
    n = 25
    rng = np.random.default_rng(5)
    J = inst.random_real_couplings(n, 22)
    h = inst.random_fields(n, 1.0, 23)
    s = rng.choice([-1, 1], size=n).astype(np.int8)
    g = rng.choice([-1, 1], size=n)
    e = oracle.energy(J, s, h)
    e_gauge = oracle.energy(J * np.outer(g, g), (g * s).astype(np.int8), h * g)
    assert abs(e - e_gauge) <= 1e-12 * (np.abs(J).sum() + np.abs(h).sum())
    p = rng.permutation(n)
    e_perm = oracle.energy(J[np.ix_(p, p)], s[p], h[p])
    assert abs(e - e_perm) <= 1e-12 * (np.abs(J).sum() + np.abs(h).sum())


def test_brute_force_small_sk_with_field():
    # Ground state of a random integer instance: no single flip lowers H.
    n = 14
    J = inst.sk(n, 24)
    h = np.round(inst.random_fields(n, 3.0, 25))
    e, best, _ = oracle.brute_force(J, h)
    assert oracle.energy_i64(J, best, h) == e
    for k in range(n):
        s2 = best.copy()
        s2[k] = -s2[k]
        assert oracle.energy_i64(J, s2, h) >= e


# --------------------------------------------------------------------------
# CSR form: the sum over stored entries equals the dense sum exactly (adding
# zero terms does not change an IEEE sum), so both forms agree bit for bit.
# --------------------------------------------------------------------------
def test_csr_equals_dense():
    n, R = 40, 4
    J = inst.regular3(n, 26)
    T = inst.schedule(40)
    a = oracle.run(J, T, 0.15, 0.15, R, seed=9, want_state=True)
    b = oracle.run(None, T, 0.15, 0.15, R, seed=9, want_state=True, csr=inst.to_csr(J))
    np.testing.assert_array_equal(a["state"], b["state"])
    np.testing.assert_array_equal(a["energy_i64"], b["energy_i64"])


def test_moebius_csr_generator_matches_dense_ladder():
    # the direct CSR construction (used for ladders too large for a dense matrix)
    for n in (4, 6, 16, 100, 2000):
        for x, y in zip(inst.moebius_csr(n), inst.to_csr(inst.moebius(n))):
            np.testing.assert_array_equal(x, y)


# --------------------------------------------------------------------------
# Fig. 3 (qualitative, no numbers survive): a 16-spin Moebius ladder with the
# schedule compressed to 100 steps; spins leave 0, saturate near +-1 and the
# energy falls, often to the ground energy -20.
# --------------------------------------------------------------------------
def test_fig3_moebius16_qualitative():
    J = inst.moebius(16)
    out = oracle.run(J, inst.schedule(100), 0.15, 0.15, 200, seed=1, want_state=True)
    assert np.median(np.abs(out["state"])) > 0.9
    e = out["energy_i64"]
    assert e.min() == -20
    assert np.mean(e <= -16) > 0.5


def test_gset_roundtrip_and_cut_value(tmp_path):
    # Table I reports MAX-CUT values: cut = (W - H)/2; a ring of 10 has a perfect
    # cut of 10 edges at the ground energy -10.
    J = inst.ring(10)
    path = str(tmp_path / "ring.gset")
    inst.write_gset(path, J)
    n, J2 = inst.read_gset(path)
    assert n == 10 and np.array_equal(J, J2)
    e, best, _ = oracle.brute_force(J2)
    assert inst.cut_value(J2, e) == 10.0
    Jm = inst.moebius(16)
    e, _, _ = oracle.brute_force(Jm)
    assert inst.cut_value(Jm, e) == 22.0


# --------------------------------------------------------------------------
# Time to solution (Sec. III: the common TTS metric of Hamerly et al.): the time
# to reach the target once with 99 % confidence, TTS99 = tau ln(0.01) / ln(1 - p)
# for a success probability p < 0.99 per run of duration tau, and tau once p >= 0.99.
# Values computed by hand.
# --------------------------------------------------------------------------
def test_tts99_hand_values():
    from paper_1806_08422_gb300.tts import tts99
    assert tts99(1.0, 0.9) == pytest.approx(2.0, rel=1e-15)            # ln 0.01 / ln 0.1 = 2
    assert tts99(1.0, 0.5) == pytest.approx(6.643856189774724, rel=1e-14)  # log2(100)
    assert tts99(3.0, 0.99) == 3.0 and tts99(3.0, 1.0) == 3.0          # one run suffices
    assert tts99(2e-6, 0.0) == math.inf                                 # never succeeds
    # a rare success: ln(0.01)/ln(1-p) ~ ln(100)/p for small p
    assert tts99(1.0, 1e-6) == pytest.approx(math.log(100.0) / 1e-6, rel=1e-6)
    assert tts99(1.0, 0.989) > tts99(1.0, 0.99)
