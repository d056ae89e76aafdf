"""CPU-only checks of the C ABI: the library builds, loads and exports every symbol
include/nmfa.h declares, and argument checking happens before any device work."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1806_08422_gb300 import build as nbuild
from paper_1806_08422_gb300 import instances as inst
from paper_1806_08422_gb300 import nmfa

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "nmfa.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nmfa_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    nbuild.build()
    return nmfa.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    assert set(_declared()) == set(nmfa.SIGNATURES)


def _create(J, h=None, precision=nmfa.NMFA_FP32):
    lib = nmfa.load()
    out = ctypes.c_void_p()
    J = np.ascontiguousarray(J, dtype=np.float64)
    hp = None if h is None else np.ascontiguousarray(h, dtype=np.float64).ctypes.data_as(ctypes.c_void_p)
    rc = lib.nmfa_create(J.shape[0], hp, J.ctypes.data_as(ctypes.c_void_p), precision, ctypes.byref(out))
    return rc, out


def test_rejects_asymmetric(lib):
    J = inst.sk(6, 1)
    J[0, 1] = -J[0, 1]
    rc, out = _create(J)
    assert rc == nmfa.NMFA_ENOTSYM and not out.value
    assert "symmetric" in nmfa.nmfa_last_error()


def test_rejects_diagonal(lib):
    J = inst.sk(6, 1)
    J[2, 2] = 1.0
    assert _create(J)[0] == nmfa.NMFA_EDIAG


def test_rejects_bad_sizes_and_values(lib):
    assert lib.nmfa_create(0, None, None, 0, ctypes.byref(ctypes.c_void_p())) == nmfa.NMFA_EINVAL
    J = inst.sk(4, 2)
    J[0, 1] = J[1, 0] = np.nan
    assert _create(J)[0] == nmfa.NMFA_EINVAL
    assert _create(inst.sk(4, 2), precision=9)[0] == nmfa.NMFA_EINVAL


def test_rejects_unrepresentable_couplings(lib):
    J = inst.sk(8, 3) * 0.1  # 0.1 is exact in neither BF16 nor E4M3
    assert _create(J, precision=nmfa.NMFA_BF16)[0] == nmfa.NMFA_EUNSUPPORTED
    assert _create(J, precision=nmfa.NMFA_BF16_FP8J)[0] == nmfa.NMFA_EUNSUPPORTED
    J = inst.sk(8, 3) * 300.0  # exact in BF16, beyond E4M3's range
    assert _create(J, precision=nmfa.NMFA_BF16_FP8J)[0] == nmfa.NMFA_EUNSUPPORTED


def test_csr_checks(lib):
    row_ptr, col, val = inst.to_csr(inst.moebius(8))
    out = ctypes.c_void_p()

    def make(rp, cl, vl, prec=nmfa.NMFA_FP32):
        rp = np.ascontiguousarray(rp, dtype=np.int64)
        cl = np.ascontiguousarray(cl, dtype=np.int32)
        vl = np.ascontiguousarray(vl, dtype=np.float64)
        return lib.nmfa_create_csr(8, None, rp.ctypes.data_as(ctypes.c_void_p), cl.ctypes.data_as(ctypes.c_void_p),
                                   vl.ctypes.data_as(ctypes.c_void_p), prec, ctypes.byref(out))

    bad = col.copy()
    bad[0] = 99
    assert make(row_ptr, bad, val) == nmfa.NMFA_EINVAL
    v2 = val.copy()
    v2[0] = 2.0
    assert make(row_ptr, col, v2) == nmfa.NMFA_ENOTSYM
    assert make(row_ptr, col, val, nmfa.NMFA_BF16) == nmfa.NMFA_EUNSUPPORTED


def test_null_handle(lib):
    assert lib.nmfa_run(None, None, 0, 0.15, 0.15, 1, 0, 0, None, None, None) == nmfa.NMFA_EINVAL
    assert lib.nmfa_sync(None) == nmfa.NMFA_EINVAL
    lib.nmfa_destroy(None)


def test_no_device_is_an_error_not_a_fallback(lib):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        pytest.skip("a GPU is present")
    rc, out = _create(inst.sk(8, 4))
    assert rc == nmfa.NMFA_ECUDA and not out.value


def test_version_and_counter(lib):
    assert "sm_103a" in nmfa.nmfa_version()
    assert nmfa.nmfa_launch_count() >= 0


def test_alu_peaks_rejects_null_output(lib):
    # argument checking comes before any device work
    assert lib.nmfa_measure_alu_peaks(None, None) == nmfa.NMFA_EINVAL
    assert "NULL" in nmfa.nmfa_last_error()
