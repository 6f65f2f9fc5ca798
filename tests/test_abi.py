"""CPU checks of the C ABI: the library builds, loads, exports every symbol
the header declares, and rejects bad arguments on the host before any CUDA
call (so these run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2208_07731_gb300 import build
    build.build()
    import paper_2208_07731_gb300 as isdf
    return isdf.lib()


def declared_symbols():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"ISDF_API[^;(]*?\b(isdf_\w+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 11
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(lib):
    assert lib.isdf_status_string(0) == b"ok"
    assert b"Hermitian" in lib.isdf_status_string(3)


def test_host_side_validation(lib):
    P = ctypes.c_void_p
    dummy = P(256)
    # n_phi < 1
    assert lib.isdf_weights(dummy, 4, 0, dummy, 4, 4, 10, 0, 0, 2.0, dummy, None) == 1
    # ld < n
    assert lib.isdf_weights(dummy, 2, 4, dummy, 4, 4, 10, 0, 0, 2.0, dummy, None) == 1
    # bad dtype / kind / alpha
    assert lib.isdf_weights(dummy, 4, 4, dummy, 4, 4, 10, 7, 0, 2.0, dummy, None) == 1
    assert lib.isdf_weights(dummy, 4, 4, dummy, 4, 4, 10, 0, 9, 2.0, dummy, None) == 1
    assert lib.isdf_weights(dummy, 4, 4, dummy, 4, 4, 10, 0, 0, -1.0, dummy, None) == 1
    # misaligned pointers
    assert lib.isdf_weights(P(258), 4, 4, dummy, 4, 4, 10, 0, 0, 2.0, dummy, None) == 1
    # empty grid is a no-op
    assert lib.isdf_weights(None, 4, 4, None, 4, 4, 0, 0, 0, 2.0, None, None) == 0
    n = ctypes.c_size_t(0)
    assert lib.isdf_kmeans_workspace(0, 4, 4, 4, ctypes.byref(n)) == 1
    assert lib.isdf_kmeans_workspace(8, 8, 8, 16, ctypes.byref(n)) == 0 and n.value > 0
    cell = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    # n_mu > n_r
    assert lib.isdf_kmeans(dummy, 2, 2, 2, cell, 9, dummy, 1, 0, dummy, None, None, None, None, dummy, n.value,
                           None) == 1
    # too many centroids for this build
    assert lib.isdf_kmeans(dummy, 128, 128, 128, cell, 9000, dummy, 1, 0, dummy, None, None, None, None, dummy,
                           n.value, None) == 8
    # missing workspace
    assert lib.isdf_kmeans(dummy, 8, 8, 8, cell, 16, dummy, 1, 0, dummy, None, None, None, None, None, 0, None) == 7
    bad_cell = (ctypes.c_double * 3)(1.0, 0.0, 1.0)
    assert lib.isdf_kmeans(dummy, 8, 8, 8, bad_cell, 16, dummy, 1, 0, dummy, None, None, None, None, dummy, n.value,
                           None) == 1
    plan = P(0)
    assert lib.isdf_plan_create(ctypes.byref(plan), None, 4, dummy, 4, 100, 4, 4, 0, dummy, 8, 0, 64, None) == 1
    assert lib.isdf_plan_create(ctypes.byref(plan), dummy, 4, dummy, 4, 100, 4, 4, 0, dummy, 200, 0, 64, None) == 1
    assert lib.isdf_plan_create(ctypes.byref(plan), dummy, 4, dummy, 4, 100, 4, 4, 0, dummy, 8, 5, 64, None) == 1
    assert lib.isdf_fit_theta(None, 0, 1, dummy, 8, None) == 1
    assert lib.isdf_fit_theta_host(None, 0, 1, dummy, 8, None) == 1
    assert lib.isdf_plan_status(None, None) == 1
    assert lib.isdf_fit_error(None, 0, 1, dummy, None) == 1
    lab, ix = P(512), P(1024)
    # cluster residual: null labels, n_psi < 1, ld < n, bad dtype, misaligned sums
    assert lib.isdf_cluster_residual(dummy, 4, 4, dummy, 4, 4, ctypes.c_int64(10), 0, None, ix, 2, dummy, lab,
                                     None) == 1
    assert lib.isdf_cluster_residual(dummy, 4, 4, dummy, 4, 0, ctypes.c_int64(10), 0, lab, ix, 2, dummy, lab,
                                     None) == 1
    assert lib.isdf_cluster_residual(dummy, 3, 4, dummy, 4, 4, ctypes.c_int64(10), 0, lab, ix, 2, dummy, lab,
                                     None) == 1
    assert lib.isdf_cluster_residual(dummy, 4, 4, dummy, 4, 4, ctypes.c_int64(10), 5, lab, ix, 2, dummy, lab,
                                     None) == 1
    assert lib.isdf_cluster_residual(dummy, 4, 4, dummy, 4, 4, ctypes.c_int64(10), 0, lab, ix, 2, P(260), lab,
                                     None) == 1
    ex = P(0)
    cell3 = (ctypes.c_double * 3)(4.0, 4.0, 4.0)
    # exchange: bad grid, kernel, omega, cell; axis lengths with a factor 7 or above 256 are unsupported
    assert lib.isdf_exchange_create(ctypes.byref(ex), 0, 8, 8, cell3, 4, 2, 2, 0, 0, 0, 0.0, None, 64, None) == 1
    assert lib.isdf_exchange_create(ctypes.byref(ex), 8, 8, 8, cell3, 4, 2, 2, 0, 0, 5, 0.0, None, 64, None) == 1
    assert lib.isdf_exchange_create(ctypes.byref(ex), 8, 8, 8, cell3, 4, 2, 2, 0, 0, 1, 0.0, None, 64, None) == 1
    assert lib.isdf_exchange_create(ctypes.byref(ex), 8, 8, 8, bad_cell, 4, 2, 2, 0, 0, 0, 0.0, None, 64, None) == 1
    assert lib.isdf_exchange_create(ctypes.byref(ex), 8, 7, 8, cell3, 4, 2, 2, 0, 0, 0, 0.0, None, 64, None) == 8
    assert lib.isdf_exchange_create(ctypes.byref(ex), 8, 512, 8, cell3, 4, 2, 2, 0, 0, 0, 0.0, None, 64, None) == 8
    assert lib.isdf_exchange_potential(None, dummy, 4, dummy, 4, None) == 1
    assert lib.isdf_exchange_apply(None, dummy, 4, dummy, 4, dummy, dummy, 4, 0, 1, dummy, 4, None) == 1
    assert lib.isdf_exchange_status(None) == 1
    # batch: null arrays, zero count, a null pair pointer
    arr = (P * 2)(256, 0)
    lds = (ctypes.c_int64 * 2)(4, 4)
    bt = P(0)
    assert lib.isdf_batch_create(ctypes.byref(bt), 2, None, lds, arr, lds, 100, 4, 4, 0, dummy, 8, 0, 64,
                                 None) == 1
    assert lib.isdf_batch_create(ctypes.byref(bt), 0, arr, lds, arr, lds, 100, 4, 4, 0, dummy, 8, 0, 64, None) == 1
    assert lib.isdf_batch_create(ctypes.byref(bt), 2, arr, lds, arr, lds, 100, 4, 4, 0, dummy, 8, 0, 64, None) == 1
    assert lib.isdf_batch_update(None, dummy, None) == 1
    assert lib.isdf_batch_plan(None, 0) is None
    # QRCP: n_mu > p, null A, bad dtype, too many grid rows
    assert lib.isdf_qrcp_points(dummy, 4, 4, dummy, 4, 4, 100, 0, dummy, dummy, 8, 9, ix, ix, None) == 1
    assert lib.isdf_qrcp_points(dummy, 4, 4, dummy, 4, 4, 100, 0, None, dummy, 8, 4, ix, ix, None) == 1
    assert lib.isdf_qrcp_points(dummy, 4, 4, dummy, 4, 4, 100, 3, dummy, dummy, 8, 4, ix, ix, None) == 1
    assert lib.isdf_qrcp_points(dummy, 4, 4, dummy, 4, 4, 1 << 23, 0, dummy, dummy, 8, 4, ix, ix, None) == 8
    # empty grid is a no-op
    assert lib.isdf_cluster_residual(dummy, 4, 4, dummy, 4, 4, ctypes.c_int64(0), 0, lab, ix, 2, dummy, lab,
                                     None) == 0
    # status of a K-means call and the wait budget need their objects
    lib.isdf_kmeans_status.argtypes = [P, P]
    lib.isdf_plan_set_wait_budget.argtypes = [P, ctypes.c_int64]
    assert lib.isdf_kmeans_status(None, None) == 1
    assert lib.isdf_plan_set_wait_budget(None, 100) == 1
    # the allocation-free K-means checks its arguments like isdf_kmeans before the scratch size:
    # an invalid call on a large grid is INVALID_ARG, a valid one beyond the fixed array UNSUPPORTED
    I32 = ctypes.c_int32
    lib.isdf_kmeans_noalloc.argtypes = [P, I32, I32, I32, P, I32, P, I32, I32, P, P, P, P, P, P]
    big = (256, 256, 256)
    assert lib.isdf_kmeans_noalloc(None, *big, cell, 64, dummy, 1, 0, dummy, None, None, None, None, None) == 1
    assert lib.isdf_kmeans_noalloc(dummy, *big, cell, 64, None, 1, 0, dummy, None, None, None, None, None) == 1
    assert lib.isdf_kmeans_noalloc(dummy, *big, bad_cell, 64, dummy, 1, 0, dummy, None, None, None, None,
                                   None) == 1
    assert lib.isdf_kmeans_noalloc(dummy, *big, cell, 64, dummy, 1, 8, dummy, None, None, None, None, None) == 1
    assert lib.isdf_kmeans_noalloc(dummy, 4, 4, 4, cell, 65, dummy, 1, 0, dummy, None, None, None, None,
                                   None) == 1
    assert lib.isdf_kmeans_noalloc(dummy, *big, cell, 64, dummy, 1, 0, dummy, None, None, None, None, None) == 8


def test_oracle_builds_and_loads():
    import oracle.oracle as o
    lib = o.load()
    assert hasattr(lib, "oracle_kmeans") and hasattr(lib, "oracle_weights")


def test_product_path_has_no_oracle_imports():
    # the CUDA path never reaches the oracle: no module of the package imports it
    pkg = os.path.join(ROOT, "paper_2208_07731_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            text = open(os.path.join(pkg, f)).read()
            assert not re.search(r"^\s*(import|from)\s+oracle", text, re.M), f
