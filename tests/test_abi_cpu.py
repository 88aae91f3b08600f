"""C-ABI checks that need no GPU: the library builds and loads, exports every
function include/fcpd.h declares, and rejects bad arguments before touching
the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2006_06281_gb300 import build as libbuild
from paper_2006_06281_gb300 import cpd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return cpd.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "fcpd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cpd_[A-Za-z_]+)\s*\(", text)))


def test_header_and_binding_agree():
    assert declared_functions() == sorted(cpd.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_library_targets_sm103a_only():
    # the build passes exactly one -gencode, for sm_103a
    assert libbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_static_calls(lib):
    assert lib.cpd_abi_version() == 1
    assert lib.cpd_status_string(5) == b"CPD_ENUMERIC"
    assert lib.cpd_status_string(99) == b"CPD_UNKNOWN"
    p = cpd.CpdParams()
    lib.cpd_params_default(C.byref(p))
    assert (p.D, p.precision, p.w, p.beta, p.lam, p.K, p.max_iter) == (3, 1, 0.1, 2.0, 2.0, 0, 50)


def _setup(lib, X, p):
    h = C.c_void_p()
    st = lib.cpd_setup(X.ctypes.data if X is not None else None, 0 if X is None else X.shape[0],
                       C.byref(p) if p is not None else None, None, C.byref(h))
    return st, h


@pytest.mark.parametrize("field,value", [("D", 2), ("precision", 7), ("w", 1.0), ("w", -0.1),
                                         ("beta", 0.0), ("lam", -1.0), ("K", -1), ("flags", 32), ("flags", 33),
                                         ("tol", -1.0), ("max_iter", -1),
                                         ("sigma2_init", float("nan"))])
def test_setup_rejects_bad_params_without_device_work(lib, field, value):
    X = np.zeros((4, 3), dtype=np.float32)
    p = cpd.make_params()
    setattr(p, field, value)
    st, h = _setup(lib, X, p)
    assert st == cpd.EINVAL
    assert h.value is None
    assert lib.cpd_last_error() != b""


def test_spectral_trim_is_rejected_for_fp64_and_batches(lib):
    X = np.zeros((4, 3), dtype=np.float64)
    p = cpd.make_params(precision=cpd.FP64, flags=cpd.FLAG_SPECTRAL_TRIM)
    st, h = _setup(lib, X, p)
    assert st == cpd.EINVAL and h.value is None
    assert b"FP64" in lib.cpd_last_error()
    X32 = np.zeros((4, 3), dtype=np.float32)
    p = cpd.make_params(flags=cpd.FLAG_SPECTRAL_TRIM)
    b = C.c_void_p()
    M = (C.c_int64 * 1)(4)
    ptr = (C.c_void_p * 1)(X32.ctypes.data)
    assert lib.cpd_batch_create(1, ptr, M, ptr, M, C.byref(p), 0.0, None, C.byref(b)) == cpd.EINVAL
    assert b.value is None


def test_get_trim_rejects_null_arguments(lib):
    k = C.c_int64()
    n = C.c_int32()
    assert lib.cpd_get_trim(None, C.byref(k), C.byref(n)) == cpd.EINVAL
    assert lib.cpd_pass_b_pieces(None, C.byref(n)) == cpd.EINVAL


def test_setup_rejects_bad_shapes(lib):
    p = cpd.make_params()
    X = np.zeros((4, 3), dtype=np.float32)
    assert _setup(lib, None, p)[0] == cpd.EINVAL
    assert _setup(lib, X, None)[0] == cpd.EINVAL
    h = C.c_void_p()
    assert lib.cpd_setup(X.ctypes.data, 0, C.byref(p), None, C.byref(h)) == cpd.EINVAL
    assert lib.cpd_setup(X.ctypes.data, 46341, C.byref(p), None, C.byref(h)) == cpd.EINVAL
    p.K = 5
    assert lib.cpd_setup(X.ctypes.data, 4, C.byref(p), None, C.byref(h)) == cpd.EINVAL


def test_other_entry_points_reject_null_context(lib):
    Y = np.zeros((4, 3), dtype=np.float32)
    d = C.c_double()
    i = C.c_int32()
    assert lib.cpd_iterate(None, Y.ctypes.data, 4, 1, None, None, None) == cpd.EINVAL
    assert lib.cpd_reset(None) == cpd.EINVAL
    assert lib.cpd_get_state(None, C.byref(d), C.byref(i), C.byref(i)) == cpd.EINVAL
    assert lib.cpd_get_W(None, Y.ctypes.data) == cpd.EINVAL
    assert lib.cpd_mstep(None, Y.ctypes.data, 1.0, Y.ctypes.data, None) == cpd.EINVAL
    assert lib.cpd_set_ground_truth(None, None, 0.0) == cpd.EINVAL
    assert lib.cpd_get_history(None, 0, None, None, None) == cpd.EINVAL
    ys = (C.c_void_p * 1)(Y.ctypes.data)
    ns = (C.c_int64 * 1)(4)
    s2 = (C.c_double * 1)()
    assert lib.cpd_iterate_shared(None, 1, ys, ns, 1, ys, s2) == cpd.EINVAL
    lib.cpd_destroy(None)   # ignored


def test_estep_rejects_bad_arguments(lib):
    T = np.zeros((4, 3), dtype=np.float32)
    out = np.zeros((4, 3), dtype=np.float32)
    e = lib.cpd_estep
    assert e(None, 4, T.ctypes.data, 4, 1, 1.0, 0.1, out.ctypes.data, None, None, None, None) == cpd.EINVAL
    assert e(T.ctypes.data, 0, T.ctypes.data, 4, 1, 1.0, 0.1, out.ctypes.data, None, None, None, None) == cpd.EINVAL
    assert e(T.ctypes.data, 4, T.ctypes.data, 4, 3, 1.0, 0.1, out.ctypes.data, None, None, None, None) == cpd.EINVAL
    assert e(T.ctypes.data, 4, T.ctypes.data, 4, 1, 0.0, 0.1, out.ctypes.data, None, None, None, None) == cpd.EINVAL
    assert e(T.ctypes.data, 4, T.ctypes.data, 4, 1, 1.0, 1.0, out.ctypes.data, None, None, None, None) == cpd.EINVAL
    assert e(T.ctypes.data, 4, T.ctypes.data, 4, 1, 1.0, 0.1, None, None, None, None, None) == cpd.EINVAL


def test_register_rejects_missing_outputs(lib):
    X = np.zeros((4, 3), dtype=np.float32)
    p = cpd.make_params()
    assert lib.cpd_register(X.ctypes.data, 4, X.ctypes.data, 4, C.byref(p), None, None, None, None,
                            None) == cpd.EINVAL


def test_injected_allocation_failure_is_reported_before_device_work(lib, monkeypatch):
    monkeypatch.setenv("CPD_FAULT", "alloc")
    X = np.zeros((4, 3), dtype=np.float32)
    st, h = _setup(lib, X, cpd.make_params())
    assert st == cpd.ENOMEM and h.value is None
    assert b"CPD_FAULT=alloc" in lib.cpd_last_error()


def test_binding_raises_typed_errors(lib):
    with pytest.raises(cpd.CpdError) as ei:
        cpd.Context(np.zeros((4, 3), dtype=np.float32), K=9)
    assert ei.value.status == cpd.EINVAL


def test_batch_entry_points_reject_bad_arguments(lib):
    X = np.zeros((10, 3), dtype=np.float32)
    arr = (C.c_void_p * 2)(X.ctypes.data, X.ctypes.data)
    null = (C.c_void_p * 2)(X.ctypes.data, None)
    n = (C.c_int64 * 2)(10, 10)
    bad_n = (C.c_int64 * 2)(10, 0)
    h = C.c_void_p()
    p32, p64 = cpd.make_params(cpd.FP32), cpd.make_params(cpd.FP64)
    create = lib.cpd_batch_create
    assert create(0, arr, n, arr, n, C.byref(p32), 0.0, None, C.byref(h)) == cpd.EINVAL
    assert create(2, arr, n, arr, n, C.byref(p64), 0.0, None, C.byref(h)) == cpd.EINVAL
    assert b"FP32" in lib.cpd_last_error()
    assert create(2, arr, n, arr, n, C.byref(p32), 100.0, None, C.byref(h)) == cpd.EINVAL
    assert create(2, arr, n, arr, n, C.byref(p32), -1.0, None, C.byref(h)) == cpd.EINVAL
    assert create(2, null, n, arr, n, C.byref(p32), 0.0, None, C.byref(h)) == cpd.EINVAL
    assert b"pair 1" in lib.cpd_last_error()
    assert create(2, arr, n, arr, bad_n, C.byref(p32), 0.0, None, C.byref(h)) == cpd.EINVAL
    assert create(2, arr, n, arr, n, C.byref(p32), 0.0, None, None) == cpd.EINVAL
    assert h.value is None
    i = C.c_int32()
    assert lib.cpd_batch_iterate(None, 1) == cpd.EINVAL
    assert lib.cpd_batch_state(None, None, None, None) == cpd.EINVAL
    assert lib.cpd_batch_get_T(None, 0, X.ctypes.data) == cpd.EINVAL
    assert lib.cpd_batch_info(None, 0, None, None, None) == cpd.EINVAL
    assert lib.cpd_batch_launch_shape(None, C.byref(i), None, None) == cpd.EINVAL
    assert lib.cpd_batch_reset(None) == cpd.EINVAL
    lib.cpd_batch_destroy(None)   # ignored


def test_batch_injected_allocation_failure(lib, monkeypatch):
    monkeypatch.setenv("CPD_FAULT", "alloc")
    X = np.zeros((10, 3), dtype=np.float32)
    arr = (C.c_void_p * 1)(X.ctypes.data)
    n = (C.c_int64 * 1)(10)
    h = C.c_void_p()
    assert lib.cpd_batch_create(1, arr, n, arr, n, C.byref(cpd.make_params()), 0.0, None, C.byref(h)) == cpd.ENOMEM
    assert h.value is None
