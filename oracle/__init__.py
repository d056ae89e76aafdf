"""FP64 CPU oracle for noisy mean-field annealing (Algorithm 1, arXiv 1806.08422).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path (the CUDA
library in ``paper_1806_08422_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``nmfa_oracle.c`` (plain C, binary64, no fused multiply-add);
this module only compiles it with gcc and marshals numpy arrays through ctypes.

Function map (paper passages in the C file's comments):
  philox4x32_10  -- counter-based generator of Salmon et al. (SC'11)
  gauss          -- the N(0,1) draw for (replica, step, spin); Box-Muller
  row_norms      -- d_i of Algorithm 1's field update (Sec. II)
  run_dense/run_csr -- Algorithm 1, with readout and Eq. (1) energies
  energy/energy_i64 -- Eq. (1), unordered pairs counted once
  brute_force    -- exhaustive ground state for small n
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nmfa_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libnmfa_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/libnmfa_oracle.so (gcc, -ffp-contract=off)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    # a per-process temporary name and an atomic rename: several processes (e.g. the
    # ranks of a multi-process test) may build at once
    tmp = "%s.%d.tmp" % (_LIB_PATH, os.getpid())
    base = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", "-fvisibility=hidden", _SRC, "-o", tmp]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:] + ["-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i32, i64, u32, u64, f64 = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                   ctypes.c_uint64, ctypes.c_double)
        lib.orc_philox4x32_10.argtypes = [P, P, P]
        lib.orc_philox4x32_10.restype = None
        lib.orc_uniform.argtypes = [u32]
        lib.orc_uniform.restype = f64
        lib.orc_gauss.argtypes = [u64, u32, i64, i32, i32]
        lib.orc_gauss.restype = f64
        lib.orc_row_norms.argtypes = [i32, P, P, P]
        lib.orc_row_norms.restype = None
        lib.orc_row_norms_csr.argtypes = [i32, P, P, P, P, P]
        lib.orc_row_norms_csr.restype = None
        lib.orc_energy.argtypes = [i32, P, P, P]
        lib.orc_energy.restype = f64
        lib.orc_energy_i64.argtypes = [i32, P, P, P]
        lib.orc_energy_i64.restype = i64
        lib.orc_run_dense.argtypes = [i32, P, P, P, i32, f64, f64, i32, i64, i32, u64, u32,
                                      i32, P, P, P, P, i32]
        lib.orc_run_dense.restype = ctypes.c_int
        lib.orc_run_csr.argtypes = [i32, P, P, P, P, P, i32, f64, f64, i32, i64, i32, u64,
                                    u32, i32, P, P, P, P, i32]
        lib.orc_run_csr.restype = ctypes.c_int
        lib.orc_brute_force.argtypes = [i32, P, P, P, P]
        lib.orc_brute_force.restype = f64
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def philox4x32_10(ctr, key) -> np.ndarray:
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def uniform(word: int) -> float:
    return _load().orc_uniform(int(word) & 0xFFFFFFFF)


def gauss(seed: int, stream: int, r: int, t: int, i: int) -> float:
    return _load().orc_gauss(seed, stream, r, t, i)


def row_norms(J, h=None) -> np.ndarray:
    J = _f64(J)
    n = J.shape[0]
    h = _f64(h)
    d = np.zeros(n)
    _load().orc_row_norms(n, _ptr(h), _ptr(J), _ptr(d))
    return d


def energy(J, signs, h=None) -> float:
    J = _f64(J)
    s = np.ascontiguousarray(signs, dtype=np.int8)
    h = _f64(h)
    return _load().orc_energy(J.shape[0], _ptr(h), _ptr(J), _ptr(s))


def energy_i64(J, signs, h=None) -> int:
    J = _f64(J)
    if not np.all(J == np.round(J)) or (h is not None and not np.all(h == np.round(h))):
        raise ValueError("energy_i64 needs integer-valued h and J")
    s = np.ascontiguousarray(signs, dtype=np.int8)
    h = _f64(h)
    return int(_load().orc_energy_i64(J.shape[0], _ptr(h), _ptr(J), _ptr(s)))


def is_integer_problem(J, h=None) -> bool:
    ok = bool(np.all(J == np.round(J)) and np.all(np.abs(J) < 2**31))
    if h is not None:
        ok = ok and bool(np.all(h == np.round(h)) and np.all(np.abs(h) < 2**31))
    return ok


def run(J, T, sigma, alpha, replicas, seed=0, stream=0, h=None, noise_sign=1, s0=None,
        want_state=False, want_phi=False, nthreads=0, csr=None, r_first=0, t_first=0):
    """Algorithm 1 over replicas r_first .. r_first+replicas-1, its steps drawn as
    steps t_first .. t_first+len(T)-1 of the noise stream.  Returns a dict with
    signs (R, n) int8, energy (R,) float64, energy_i64 (R,) int64 or None,
    and, on request, state (R, n) and phi (R, n) (the last step's Phi).

    `csr=(row_ptr, col, val)` selects the sparse form (J may then be None, unless
    energies are wanted, which always use the dense matrix when given)."""
    lib = _load()
    T = _f64(T)
    t_f = int(T.shape[0])
    h = _f64(h)
    s0 = _f64(s0)
    if csr is not None:
        row_ptr = np.ascontiguousarray(csr[0], dtype=np.int64)
        col = np.ascontiguousarray(csr[1], dtype=np.int32)
        val = _f64(csr[2])
        n = int(row_ptr.shape[0] - 1)
    else:
        J = _f64(J)
        n = int(J.shape[0])
    if s0 is not None:
        assert s0.shape == (replicas, n)
    signs = np.zeros((replicas, n), dtype=np.int8)
    state = np.zeros((replicas, n)) if want_state else None
    phi = np.zeros((replicas, n)) if want_phi else None
    if csr is not None:
        rc = lib.orc_run_csr(n, _ptr(h), _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(T),
                             t_f, float(sigma), float(alpha), int(replicas), int(r_first), int(t_first),
                             int(seed),
                             int(stream), int(noise_sign), _ptr(s0), _ptr(state),
                             _ptr(phi), _ptr(signs), int(nthreads))
    else:
        rc = lib.orc_run_dense(n, _ptr(h), _ptr(J), _ptr(T), t_f, float(sigma),
                               float(alpha), int(replicas), int(r_first), int(t_first), int(seed),
                               int(stream),
                               int(noise_sign), _ptr(s0), _ptr(state), _ptr(phi),
                               _ptr(signs), int(nthreads))
    if rc != 0:
        raise MemoryError("oracle run failed (%d)" % rc)
    out = {"signs": signs, "state": state, "phi": phi, "energy": None, "energy_i64": None}
    Jd = J
    if Jd is None and csr is not None:
        Jd = csr_to_dense(n, row_ptr, col, val)
    out["energy"] = np.array([energy(Jd, signs[r], h) for r in range(replicas)])
    if is_integer_problem(Jd, h):
        out["energy_i64"] = np.array([energy_i64(Jd, signs[r], h) for r in range(replicas)],
                                     dtype=np.int64)
    return out


def csr_to_dense(n, row_ptr, col, val) -> np.ndarray:
    J = np.zeros((n, n))
    for i in range(n):
        for k in range(int(row_ptr[i]), int(row_ptr[i + 1])):
            J[i, int(col[k])] = val[k]
    return J


def brute_force(J, h=None):
    """Exhaustive minimum of Eq. (1): (E_min, one minimiser, count of minimisers)."""
    J = _f64(J)
    n = J.shape[0]
    if n > 30:
        raise ValueError("brute force is for n <= 30")
    h = _f64(h)
    best = np.zeros(n, dtype=np.int8)
    cnt = ctypes.c_int64(0)
    e = _load().orc_brute_force(n, _ptr(h), _ptr(J), _ptr(best), ctypes.byref(cnt))
    return e, best, int(cnt.value)
