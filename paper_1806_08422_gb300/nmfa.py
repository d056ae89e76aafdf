"""Thin ctypes binding of libnmfa.so (include/nmfa.h), same names as the C ABI.

Argument marshalling only: every step of the annealing runs in the library's CUDA
kernels.  Host-buffer calls take numpy arrays; device calls take torch CUDA tensors
(torch supplies device memory and streams).  If the compiled library is missing the
import of this module's functions fails loudly; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnmfa.so")

NMFA_OK = 0
NMFA_EINVAL = -1
NMFA_ENOTSYM = -2
NMFA_EDIAG = -3
NMFA_ENOMEM = -4
NMFA_ECUDA = -5
NMFA_ETIMEOUT = -6
NMFA_EUNSUPPORTED = -7

NMFA_FP64 = 0
NMFA_FP32 = 1
NMFA_BF16 = 2
NMFA_BF16_FP8J = 3
PRECISIONS = {"fp64": NMFA_FP64, "fp32": NMFA_FP32, "bf16": NMFA_BF16, "bf16_fp8j": NMFA_BF16_FP8J}

# Every symbol include/nmfa.h declares, with (restype, argtypes).
_P = ctypes.c_void_p
_i32, _i64, _u32, _u64, _f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
SIGNATURES = {
    "nmfa_create": (ctypes.c_int, [_i32, _P, _P, _i32, ctypes.POINTER(_P)]),
    "nmfa_create_csr": (ctypes.c_int, [_i32, _P, _P, _P, _P, _i32, ctypes.POINTER(_P)]),
    "nmfa_destroy": (None, [_P]),
    "nmfa_run": (ctypes.c_int, [_P, _P, _i32, _f64, _f64, _i32, _u64, _u32, _P, _P, _P]),
    "nmfa_run_device": (ctypes.c_int, [_P, _P, _i32, _f64, _f64, _i32, _u64, _u32, _P, _P, _P, _P]),
    "nmfa_run_device_noalloc": (ctypes.c_int, [_P, _P, _i32, _f64, _f64, _i32, _u64, _u32, _P, _P, _P, _P]),
    "nmfa_sync": (ctypes.c_int, [_P]),
    "nmfa_batch_create": (ctypes.c_int, [_P, _P, _i32, _i32, ctypes.POINTER(_P)]),
    "nmfa_batch_launch": (ctypes.c_int, [_P, _P]),
    "nmfa_batch_sync": (ctypes.c_int, [_P]),
    "nmfa_batch_info": (ctypes.c_int, [_P, _P, _P, _P]),
    "nmfa_batch_destroy": (None, [_P]),
    "nmfa_batch_plan": (ctypes.c_int, [_P, _P, _P, _P, _i32, _P]),
    "nmfa_autotune_bn": (ctypes.c_int, [_P, _i32, _P]),
    "nmfa_server_create": (ctypes.c_int, [_P, ctypes.POINTER(_P)]),
    "nmfa_server_submit": (ctypes.c_int, [_P, _P, ctypes.POINTER(_u64)]),
    "nmfa_server_poll": (ctypes.c_int, [_P, _u64, _P, _P]),
    "nmfa_server_drain": (ctypes.c_int, [_P, _f64]),
    "nmfa_server_stats": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "nmfa_batch_set_stream_ids": (ctypes.c_int, [_P, _P, _i32]),
    "nmfa_server_destroy": (None, [_P]),
    "nmfa_debug_run": (ctypes.c_int, [_P, _P, _i32, _f64, _f64, _i32, _u64, _u32, _i32, _P, _P, _P, _P, _P,
                                      _P, _P]),
    "nmfa_problem_info": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "nmfa_profile_enable": (ctypes.c_int, [_P, _i32]),
    "nmfa_last_kernel_ms": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float)]),
    "nmfa_measure_alu_peaks": (ctypes.c_int, [_P, _P]),
    "nmfa_tune_replicas_per_cta": (ctypes.c_int, [_P, _i32]),
    "nmfa_debug_withhold_arrival": (ctypes.c_int, [_P, _i32]),
    "nmfa_launch_count": (_u64, []),
    "nmfa_last_error": (ctypes.c_char_p, []),
    "nmfa_version": (ctypes.c_char_p, []),
}

_lib = None


class NmfaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("NMFA error %d: %s" % (code, msg))
        self.code = code


def load(path: str = LIB_PATH):
    """Load libnmfa.so (built by paper_1806_08422_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libnmfa.so is not built (run paper_1806_08422_gb300.build.build())")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc):
    if rc != NMFA_OK:
        raise NmfaError(rc, load().nmfa_last_error().decode())


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _t_ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


# ---------------------------------------------------------------- C names
def nmfa_create(J, h=None, precision="bf16"):
    J = np.ascontiguousarray(J, dtype=np.float64)
    h = None if h is None else np.ascontiguousarray(h, dtype=np.float64)
    out = ctypes.c_void_p()
    _check(load().nmfa_create(J.shape[0], _np_ptr(h), _np_ptr(J), PRECISIONS.get(precision, precision),
                              ctypes.byref(out)))
    return out


def nmfa_create_csr(n, row_ptr, col, val, h=None, precision="fp32"):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    vl = np.ascontiguousarray(val, dtype=np.float64)
    h = None if h is None else np.ascontiguousarray(h, dtype=np.float64)
    out = ctypes.c_void_p()
    _check(load().nmfa_create_csr(int(n), _np_ptr(h), _np_ptr(rp), _np_ptr(cl), _np_ptr(vl),
                                  PRECISIONS.get(precision, precision), ctypes.byref(out)))
    return out


def nmfa_destroy(handle):
    load().nmfa_destroy(handle)


def nmfa_run(handle, n, T, sigma, alpha, replicas, seed=0, stream_id=0, want_i64=False):
    """Host buffers in and out; returns (signs (R, n) int8, energy (R,), energy_i64 or None)."""
    T = np.ascontiguousarray(T, dtype=np.float64)
    signs = np.empty((replicas, n), dtype=np.int8)
    energy = np.empty(replicas, dtype=np.float64)
    ei = np.empty(replicas, dtype=np.int64) if want_i64 else None
    _check(load().nmfa_run(handle, _np_ptr(T), T.shape[0], float(sigma), float(alpha), int(replicas), int(seed),
                           int(stream_id), _np_ptr(signs), _np_ptr(energy), _np_ptr(ei)))
    return signs, energy, ei


def nmfa_run_device(handle, T_dev, sigma, alpha, replicas, seed=0, stream_id=0, signs=None, energy=None,
                    energy_i64=None, stream=None):
    _check(load().nmfa_run_device(handle, _t_ptr(T_dev), int(T_dev.numel()), float(sigma), float(alpha),
                                  int(replicas), int(seed), int(stream_id), _t_ptr(signs), _t_ptr(energy),
                                  _t_ptr(energy_i64), _stream_ptr(stream)))


def nmfa_run_device_noalloc(handle, T_dev, sigma, alpha, replicas, seed=0, stream_id=0, signs=None, energy=None,
                            energy_i64=None, stream=None):
    """nmfa_run_device for a BF16 or FP8-stored problem without any allocation (static
    scratch); capturable into a CUDA graph after a first call outside the capture."""
    _check(load().nmfa_run_device_noalloc(handle, _t_ptr(T_dev), int(T_dev.numel()), float(sigma), float(alpha),
                                          int(replicas), int(seed), int(stream_id), _t_ptr(signs), _t_ptr(energy),
                                          _t_ptr(energy_i64), _stream_ptr(stream)))


def nmfa_debug_run(handle, T_dev, sigma, alpha, replicas, seed=0, stream_id=0, noise_sign=1, s0=None,
                   s_out=None, phi_out=None, signs=None, energy=None, energy_i64=None, stream=None):
    _check(load().nmfa_debug_run(handle, _t_ptr(T_dev), int(T_dev.numel()), float(sigma), float(alpha),
                                 int(replicas), int(seed), int(stream_id), int(noise_sign), _t_ptr(s0),
                                 _t_ptr(s_out), _t_ptr(phi_out), _t_ptr(signs), _t_ptr(energy),
                                 _t_ptr(energy_i64), _stream_ptr(stream)))


def nmfa_sync(handle):
    _check(load().nmfa_sync(handle))


def nmfa_problem_info(handle):
    n, p, iv, b = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check(load().nmfa_problem_info(handle, ctypes.byref(n), ctypes.byref(p), ctypes.byref(iv),
                                    ctypes.byref(b)))
    return {"n": n.value, "precision": p.value, "integer_valued": bool(iv.value), "device_bytes": b.value}


def nmfa_profile_enable(handle, on=True):
    _check(load().nmfa_profile_enable(handle, 1 if on else 0))


def nmfa_last_kernel_ms(handle):
    ms = ctypes.c_float()
    _check(load().nmfa_last_kernel_ms(handle, ctypes.byref(ms)))
    return ms.value


def nmfa_measure_alu_peaks(stream=None):
    """Measured FP32 and FP64 FMA throughput (TFLOP/s) and MUFU tanh throughput
    (Tops/s) of the current device."""
    out = (ctypes.c_double * 3)()
    _check(load().nmfa_measure_alu_peaks(ctypes.cast(out, ctypes.c_void_p), _stream_ptr(stream)))
    return {"fp32_fma_tflops": out[0], "fp64_fma_tflops": out[1], "mufu_tanh_tops": out[2]}


def nmfa_tune_replicas_per_cta(handle, rc):
    _check(load().nmfa_tune_replicas_per_cta(handle, int(rc)))


def nmfa_debug_withhold_arrival(handle, step):
    _check(load().nmfa_debug_withhold_arrival(handle, int(step)))


def nmfa_launch_count():
    return int(load().nmfa_launch_count())


def nmfa_last_error():
    return load().nmfa_last_error().decode()


def nmfa_version():
    return load().nmfa_version().decode()


class nmfa_job(ctypes.Structure):
    _fields_ = [("T_dev", ctypes.c_void_p), ("t_f", ctypes.c_int32), ("sigma", ctypes.c_double),
                ("alpha", ctypes.c_double), ("replicas", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("stream_id", ctypes.c_uint32), ("signs_dev", ctypes.c_void_p), ("energy_dev", ctypes.c_void_p),
                ("energy_i64_dev", ctypes.c_void_p)]


NMFA_BATCH_GRAPH = 1
NMFA_BATCH_AUTOTUNE = 2
NMFA_BATCH_BN64 = 4
NMFA_BATCH_BN128 = 16
NMFA_BATCH_PAIR128 = 32
NMFA_BATCH_BN256 = 64
NMFA_BATCH_DEBUG_WITHHOLD_TILE = 8
NMFA_BATCH_FP8_IN_KERNEL = 128


def make_job(T_dev, sigma, alpha, replicas, seed=0, stream_id=0, signs=None, energy=None, energy_i64=None):
    return nmfa_job(T_dev.data_ptr(), int(T_dev.numel()), float(sigma), float(alpha), int(replicas), int(seed),
                    int(stream_id), None if signs is None else signs.data_ptr(),
                    None if energy is None else energy.data_ptr(),
                    None if energy_i64 is None else energy_i64.data_ptr())


def nmfa_batch_create(handles, jobs, options=0):
    n = len(handles)
    harr = (ctypes.c_void_p * n)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    jarr = (nmfa_job * n)(*jobs)
    out = ctypes.c_void_p()
    _check(load().nmfa_batch_create(harr, jarr, n, int(options), ctypes.byref(out)))
    return out


def nmfa_batch_launch(batch, stream=None):
    _check(load().nmfa_batch_launch(batch, _stream_ptr(stream)))


def nmfa_batch_sync(batch):
    _check(load().nmfa_batch_sync(batch))


def nmfa_batch_set_stream_ids(batch, stream_ids):
    ids = (ctypes.c_uint32 * len(stream_ids))(*[int(x) for x in stream_ids])
    _check(load().nmfa_batch_set_stream_ids(batch, ids, len(stream_ids)))


def nmfa_batch_info(batch):
    g, n, b = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check(load().nmfa_batch_info(batch, ctypes.byref(g), ctypes.byref(n), ctypes.byref(b)))
    return {"grid": g.value, "groups": n.value, "workspace_bytes": b.value}


def nmfa_batch_destroy(batch):
    load().nmfa_batch_destroy(batch)


def nmfa_batch_plan(batch):
    """[(replicas per tile, CTAs per MMA, CTAs per cluster)] for each persistent launch
    of the batch."""
    bn, cp, cc, cnt = (ctypes.c_int32 * 8)(), (ctypes.c_int32 * 8)(), (ctypes.c_int32 * 8)(), ctypes.c_int32()
    _check(load().nmfa_batch_plan(batch, bn, cp, cc, 8, ctypes.byref(cnt)))
    return [(bn[k], cp[k], cc[k]) for k in range(min(cnt.value, 8))]


def nmfa_autotune_bn(handle, replicas):
    bn = ctypes.c_int32()
    _check(load().nmfa_autotune_bn(handle, int(replicas), ctypes.byref(bn)))
    return bn.value


class nmfa_server_config(ctypes.Structure):
    _fields_ = [("memory_budget_bytes", ctypes.c_int64), ("max_inflight", ctypes.c_int32),
                ("max_attempts", ctypes.c_int32)]


class nmfa_request(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("h", ctypes.c_void_p), ("J", ctypes.c_void_p), ("precision", ctypes.c_int32),
                ("T", ctypes.c_void_p), ("t_f", ctypes.c_int32), ("sigma", ctypes.c_double),
                ("alpha", ctypes.c_double), ("replicas", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("target_energy", ctypes.c_double)]


class nmfa_result(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("attempts", ctypes.c_int32), ("success", ctypes.c_int32),
                ("error", ctypes.c_int32), ("best_energy", ctypes.c_double), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_first_start", ctypes.c_double), ("t_done", ctypes.c_double),
                ("time_to_target", ctypes.c_double), ("spin_updates", ctypes.c_int64)]


def nmfa_server_create(memory_budget_bytes=0, max_inflight=2, max_attempts=4):
    cfg = nmfa_server_config(int(memory_budget_bytes), int(max_inflight), int(max_attempts))
    out = ctypes.c_void_p()
    _check(load().nmfa_server_create(ctypes.byref(cfg), ctypes.byref(out)))
    return out


def nmfa_server_submit(server, J, T, replicas, target_energy, h=None, precision="bf16_fp8j", sigma=0.15,
                       alpha=0.15, seed=0):
    J = np.ascontiguousarray(J, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    h = None if h is None else np.ascontiguousarray(h, dtype=np.float64)
    q = nmfa_request(J.shape[0], None if h is None else h.ctypes.data, J.ctypes.data,
                     PRECISIONS.get(precision, precision), T.ctypes.data, T.shape[0], float(sigma), float(alpha),
                     int(replicas), int(seed), float(target_energy))
    ticket = ctypes.c_uint64()
    _check(load().nmfa_server_submit(server, ctypes.byref(q), ctypes.byref(ticket)))
    return ticket.value


def nmfa_server_poll(server, ticket, n=None):
    res = nmfa_result()
    signs = np.zeros(n, dtype=np.int8) if n else None
    _check(load().nmfa_server_poll(server, int(ticket), ctypes.byref(res), _np_ptr(signs)))
    d = {k: getattr(res, k) for k, _ in nmfa_result._fields_}
    if signs is not None:
        d["best_signs"] = signs
    return d


def nmfa_server_drain(server, timeout_s=600.0):
    _check(load().nmfa_server_drain(server, float(timeout_s)))


def nmfa_server_stats(server):
    la, mu, out, mb, ru = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check(load().nmfa_server_stats(server, ctypes.byref(la), ctypes.byref(mu), ctypes.byref(out), ctypes.byref(mb),
                                    ctypes.byref(ru)))
    return {"launches": la.value, "mem_used": mu.value, "outstanding": out.value, "max_requests_per_launch": mb.value,
            "batches_reused": ru.value}


def nmfa_server_destroy(server):
    load().nmfa_server_destroy(server)


# ---------------------------------------------------------------- convenience
class Problem:
    """Owning wrapper around an nmfa_problem handle."""

    def __init__(self, J=None, h=None, precision="bf16", csr=None, n=None):
        if csr is not None:
            self.n = int(n if n is not None else len(csr[0]) - 1)
            self.handle = nmfa_create_csr(self.n, csr[0], csr[1], csr[2], h=h, precision=precision)
        else:
            self.n = int(np.asarray(J).shape[0])
            self.handle = nmfa_create(J, h=h, precision=precision)
        self.precision = precision

    def info(self):
        return nmfa_problem_info(self.handle)

    def run(self, T, sigma=0.15, alpha=0.15, replicas=1, seed=0, stream_id=0, want_i64=None):
        if want_i64 is None:
            want_i64 = self.info()["integer_valued"]
        return nmfa_run(self.handle, self.n, T, sigma, alpha, replicas, seed, stream_id, want_i64)

    def run_device(self, T_dev, sigma=0.15, alpha=0.15, replicas=1, seed=0, stream_id=0, signs=None,
                   energy=None, energy_i64=None, stream=None):
        nmfa_run_device(self.handle, T_dev, sigma, alpha, replicas, seed, stream_id, signs, energy, energy_i64,
                        stream)

    def debug_run(self, T_dev, sigma, alpha, replicas, **kw):
        nmfa_debug_run(self.handle, T_dev, sigma, alpha, replicas, **kw)

    def sync(self):
        nmfa_sync(self.handle)

    def close(self):
        if getattr(self, "handle", None) is not None:
            nmfa_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
