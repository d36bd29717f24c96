"""The C-ABI library builds, loads and exports every symbol include/tlfe.h
declares; argument validation answers with status codes without any GPU
(these calls return before touching the device)."""

import ctypes as C
import os
import re
import shutil

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("CUDA toolkit not available")
    from paper_2602_17002_gb300 import build_lib, tlfe
    build_lib.build()
    return tlfe.load()


def declared_symbols():
    with open(os.path.join(ROOT, "include", "tlfe.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tlfe_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    from paper_2602_17002_gb300 import tlfe
    names = declared_symbols()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(tlfe.EXPORTS)
    assert lib.tlfe_version().decode().startswith("tlfe")


def _desc(tlfe, X, blocks, mats, precision=1):
    cb = (tlfe.tlfe_block * len(blocks))(*blocks)
    cm = (tlfe.tlfe_material * len(mats))(*mats)
    d = tlfe.tlfe_mesh_desc(X.shape[0], X.ctypes.data, len(blocks), C.addressof(cb), len(mats), C.addressof(cm),
                            None, precision, 0, 0)
    return d, cb, cm


def test_validation_errors_need_no_gpu(lib):
    from paper_2602_17002_gb300 import tlfe
    h = C.c_void_p()
    assert lib.tlfe_create_mesh(None, None, C.byref(h)) == 1
    X = np.zeros((4, 3))
    X[1, 0] = X[2, 1] = X[3, 2] = 1.0
    conn = np.array([[0, 1, 2, 7]], np.int32)  # node 7 does not exist
    mat = tlfe.tlfe_material(0, 1e6, 1e6, 0.0, 0.0, 1e3)
    d, cb, cm = _desc(tlfe, X, [tlfe.tlfe_block(0, 1, 1, conn.ctypes.data, None)], [mat])
    assert lib.tlfe_create_mesh(C.byref(d), None, C.byref(h)) == 1
    assert "out of range" in lib.tlfe_last_error().decode()
    conn = np.array([[0, 1, 2, 3]], np.int32)
    d, cb, cm = _desc(tlfe, X, [tlfe.tlfe_block(0, 1, 3, conn.ctypes.data, None)], [mat])  # T4 with 3 points
    assert lib.tlfe_create_mesh(C.byref(d), None, C.byref(h)) == 7
    bad = tlfe.tlfe_material(0, 1e6, 1e6, -1.0, 0.0, 1e3)  # negative damping
    d, cb, cm = _desc(tlfe, X, [tlfe.tlfe_block(0, 1, 1, conn.ctypes.data, None)], [bad])
    assert lib.tlfe_create_mesh(C.byref(d), None, C.byref(h)) == 1
    body = np.array([3], np.int32)  # body id beyond n_bodies
    d, cb, cm = _desc(tlfe, X, [tlfe.tlfe_block(0, 1, 1, conn.ctypes.data, body.ctypes.data)], [mat])
    assert lib.tlfe_create_mesh(C.byref(d), None, C.byref(h)) == 1
    d, cb, cm = _desc(tlfe, X, [tlfe.tlfe_block(0, 1, 1, conn.ctypes.data, None)], [mat], precision=5)
    assert lib.tlfe_create_mesh(C.byref(d), None, C.byref(h)) == 1


def test_null_handles_and_oversized_noalloc_are_rejected(lib):
    assert lib.tlfe_internal_force(None, None, None, None, None) == 1
    assert lib.tlfe_vjp(None, None, None, None, None, None, None, None) == 1
    assert lib.tlfe_sync(None, None, None) == 1
    assert lib.tlfe_destroy_mesh(None) == 0
    one = C.c_double(0.0)
    assert lib.tlfe_norm_noalloc(C.byref(one), C.c_int64(4096 * 4096 + 1), C.byref(one), None) == 1
    assert "exceeds the maximum" in lib.tlfe_last_error().decode()
    assert lib.tlfe_norm_noalloc(None, C.c_int64(-1), C.byref(one), None) == 1


def test_wait_timeout_selftest_validates_its_arguments(lib):
    """The timeout diagnostic rejects a NULL mesh before touching the device."""
    assert lib.tlfe_selftest_wait_timeout(None, C.c_int64(16), None) == 1
    assert "mesh is NULL" in lib.tlfe_last_error().decode()
