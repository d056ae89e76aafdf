"""Energy readout of the tensor path (Eq. 1 at the sign vectors, Algorithm 1's last
lines).

For integer couplings and fields with max_i (sum_j |J_ij| + 2 |h_i|) < 2^24 the
persistent kernel ends every run with one more product J s~ of the sign vectors and
forms the energies itself; the energies must equal the oracle's energy of the
returned sign vectors exactly (int64, and the same integers in FP64).  Other runs
(t_f = 0, real-valued couplings, rows at or above the 2^24 bound) take the separate
energy kernel and must agree just as exactly.
"""
import numpy as np
import pytest

import oracle
from paper_1806_08422_gb300 import instances as inst

from helpers import Gpu

pytestmark = pytest.mark.gpu

TENSOR = ["bf16", "bf16_fp8j"]


def check_energies(J, h, out, R):
    ref = np.array([oracle.energy_i64(J, out["signs"][r], h) for r in range(R)], dtype=np.int64)
    np.testing.assert_array_equal(out["energy_i64"], ref)
    np.testing.assert_array_equal(out["energy"], ref.astype(np.float64))


@pytest.mark.parametrize("prec", TENSOR)
@pytest.mark.parametrize("n,R", [(300, 64), (257, 200), (640, 300)])
def test_fused_energy_with_fields(prec, n, R):
    """Integer fields enter through the 2h start of the accumulator; n and R ragged
    against the 128-spin tiles and the replica blocks."""
    J = inst.sk(n, 100 + n)
    h = np.random.default_rng(n).integers(-3, 4, size=n).astype(np.float64)
    g = Gpu(J, h=h, precision=prec)
    out = g.run(inst.schedule(60), 0.15, 0.15, R, seed=21)
    check_energies(J, h, out, R)
    g.close()


@pytest.mark.parametrize("prec", TENSOR)
def test_fused_energy_maxcut_and_ladder(prec):
    for J in (inst.gnp_maxcut(390, 0.5, 31), inst.moebius(200), inst.regular3(258, 32)):
        n = J.shape[0]
        g = Gpu(J, precision=prec)
        out = g.run(inst.schedule(80), 0.15, 0.15, 130, seed=22)
        check_energies(J, None, out, 130)
        g.close()


def test_energy_without_steps():
    """t_f = 0: the signs of the zero state are all +1 and the energy is sum_{i<j} J_ij
    + sum_i h_i (the separate energy kernel)."""
    n, R = 200, 40
    J = inst.sk(n, 41)
    h = np.random.default_rng(41).integers(-2, 3, size=n).astype(np.float64)
    g = Gpu(J, h=h, precision="bf16")
    out = g.run(np.zeros(0), 0.15, 0.15, R, seed=1)
    assert np.all(out["signs"] == 1)
    assert np.all(out["energy_i64"] == int(np.triu(J, 1).sum() + h.sum()))
    g.close()


@pytest.mark.parametrize("n,fused", [(1000, True), (1100, False)])
def test_energy_near_exactness_bound(n, fused):
    """J = +-2^14: rows sum to (n - 1) 2^14, just below 2^24 for n = 1000 (kernel-formed
    energies, accumulator partial sums close to the bound) and above it for n = 1100
    (the separate FP64 energy kernel).  Both must be exact."""
    J = inst.sk(n, 50 + n) * 16384.0
    assert (((n - 1) * 16384) < 2 ** 24) == fused
    g = Gpu(J, precision="bf16")
    out = g.run(inst.schedule(40), 0.15, 0.15, 96, seed=3)
    check_energies(J, None, out, 96)
    g.close()


def test_real_valued_bf16_energies_stay_fp64():
    """Couplings exact in BF16 but not integers: no integer energies, and the FP64
    energies come from the FP64 couplings."""
    n, R = 150, 24
    J = np.round(inst.random_real_couplings(n, 61, density=0.6) * 4.0) / 4.0
    J = np.clip(J, -8.0, 8.0)
    h = np.round(inst.random_fields(n, 1.0, 62) * 2.0) / 2.0
    g = Gpu(J, h=h, precision="bf16")
    out = g.run(inst.schedule(40), 0.15, 0.15, R, seed=4)
    assert out["energy_i64"] is None
    mag = np.abs(np.triu(J, 1)).sum() + np.abs(h).sum()
    for r in range(R):
        assert abs(out["energy"][r] - oracle.energy(J, out["signs"][r], h)) <= 1e-12 * mag
    g.close()
