"""Shared helpers for the parity tests: run the CUDA path through the C ABI with
torch-allocated device buffers, and compute the oracle-side tolerance scale."""
from __future__ import annotations

import math

import numpy as np

import oracle


def phi_scale(J, s0, h, sigma, seed, stream, t=0, r_first=0):
    """Forward-error scale of Phi for one step from state s0 (R, n) of replicas
    r_first.. : scale_i = (|h_i| + sum_j |J_ij s_j|) / d_i + sigma |z|."""
    J = np.asarray(J, dtype=np.float64)
    R, n = s0.shape
    hh = np.zeros(n) if h is None else np.asarray(h, dtype=np.float64)
    d = np.sqrt(hh ** 2 + (J ** 2).sum(1))
    mag = np.abs(s0) @ np.abs(J).T + np.abs(hh)[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        base = np.where(d[None, :] > 0, mag / d[None, :], 0.0)
    z = np.array([[oracle.gauss(seed, stream, r_first + r, t, i) for i in range(n)] for r in range(R)])
    return base + sigma * np.abs(z)


# Rounding allowances of the update s <- alpha (-tanh(Phi / T)) + (1 - alpha) s per path:
#   mul   relative error of Phi * (1/T) (the FP32 paths multiply by a binary32 1/T);
#   tanh  absolute error of the tanh the path uses (FP64 tanh and FP32 tanhf are within
#         two units in the last place of |tanh| <= 1; the BF16 tensor path uses the MUFU
#         tanh.approx.f32, whose error is about 2^-11 over the whole range);
#   round the remaining binary32/binary64 roundings (alpha, 1 - alpha, s0, products, sum).
UPDATE_EPS = {
    "fp64": {"mul": 2.0 ** -50, "tanh": 2.0 ** -50, "round": 2.0 ** -50},
    "fp32": {"mul": 2.0 ** -21, "tanh": 2.0 ** -21, "round": 2.0 ** -21},
    "bf16": {"mul": 2.0 ** -21, "tanh": 2.0 ** -10, "round": 2.0 ** -21},
}


def update_tol(prec, alpha, T, phi, phi_err=0.0):
    """Elementwise bound on |s_gpu - s_exact| after one step of Algorithm 1's update
    s = alpha (-tanh(Phi / T)) + (1 - alpha) s_prev from the same s_prev, when the
    GPU's Phi differs from the exact one by at most `phi_err` (tanh has slope <= 1,
    so that error enters as phi_err / T)."""
    e = UPDATE_EPS[prec]
    return alpha * ((phi_err + np.abs(phi) * e["mul"]) / T + e["tanh"]) + e["round"]


def wilson(k, n, zq=1.959963984540054):
    p = k / n
    den = 1 + zq * zq / n
    c = (p + zq * zq / (2 * n)) / den
    half = zq * math.sqrt(p * (1 - p) / n + zq * zq / (4 * n * n)) / den
    return c - half, c + half


class Gpu:
    """Device-side driver of one problem through nmfa_debug_run / nmfa_run_device."""

    def __init__(self, J=None, h=None, precision="fp32", csr=None, n=None):
        import torch

        from paper_1806_08422_gb300 import nmfa

        self.torch = torch
        self.nmfa = nmfa
        self.p = nmfa.Problem(J, h=h, precision=precision, csr=csr, n=n)
        self.n = self.p.n

    def run(self, T, sigma, alpha, replicas, seed=0, stream_id=0, noise_sign=1, s0=None, want_state=False,
            want_phi=False, want_energy=True):
        torch = self.torch
        dev = torch.device("cuda", 0)
        Td = torch.as_tensor(np.asarray(T, dtype=np.float64), device=dev)
        n = self.n
        signs = torch.empty((replicas, n), dtype=torch.int8, device=dev)
        energy = torch.empty(replicas, dtype=torch.float64, device=dev) if want_energy else None
        integer = self.p.info()["integer_valued"]
        ei = torch.empty(replicas, dtype=torch.int64, device=dev) if (want_energy and integer) else None
        s0d = None if s0 is None else torch.as_tensor(np.ascontiguousarray(s0, dtype=np.float64), device=dev)
        so = torch.empty((replicas, n), dtype=torch.float64, device=dev) if want_state else None
        po = torch.empty((replicas, n), dtype=torch.float64, device=dev) if want_phi else None
        self.p.debug_run(Td, sigma, alpha, replicas, seed=seed, stream_id=stream_id, noise_sign=noise_sign,
                         s0=s0d, s_out=so, phi_out=po, signs=signs, energy=energy, energy_i64=ei)
        self.p.sync()
        out = {"signs": signs.cpu().numpy(),
               "energy": None if energy is None else energy.cpu().numpy(),
               "energy_i64": None if ei is None else ei.cpu().numpy(),
               "state": None if so is None else so.cpu().numpy(),
               "phi": None if po is None else po.cpu().numpy()}
        return out

    def close(self):
        self.p.close()
