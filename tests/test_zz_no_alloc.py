"""The K-means entry point that allocates nothing (isdf_kmeans_noalloc), for
callers that cannot call cudaMalloc because another framework's allocator
owns the device memory or because their loop must not allocate mid-step.

It must give exactly what isdf_kmeans gives (the K-means results are
bit-exact, so the tolerance is equality), on two calls in a row that share the
library's fixed scratch array, and must refuse problems larger than that
array before launching anything. This file is collected last so that a run
stopping at the first failure has already run every other test; it also
passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def isdf():
    from paper_2208_07731_gb300 import build
    build.build()
    import paper_2208_07731_gb300 as m
    L = m.lib()
    P, I32 = ctypes.c_void_p, ctypes.c_int32
    L.isdf_kmeans_noalloc.argtypes = [P, I32, I32, I32, P, I32, P, I32, I32, P, P, P, P, P, P]
    L.isdf_kmeans_noalloc.restype = I32
    return m


def _p(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def noalloc(isdf, w, shape, cell, n_mu, init, iters, flags=0, labels=True, objective=True):
    n_r = int(np.prod(shape))
    idx = torch.full((n_mu,), -7, dtype=torch.int64, device=DEV)
    cen = torch.full((n_mu, 3), -1.0, dtype=torch.float64, device=DEV)
    obj = torch.full((iters + 1,), -1.0, dtype=torch.float64, device=DEV) if objective else None
    lab = torch.full((n_r,), -3, dtype=torch.int32, device=DEV) if labels else None
    stats = torch.zeros(4, dtype=torch.int64, device=DEV)
    cellh = (ctypes.c_double * 3)(*cell)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = isdf.lib().isdf_kmeans_noalloc(_p(w), *shape, cellh, n_mu, _p(init), iters, flags, _p(idx), _p(cen),
                                        _p(obj), _p(lab), _p(stats), stream)
    return rc, {"idx": idx, "centroids": cen, "objective": obj, "labels": lab, "stats": stats}


def _case(seed, shape, n_mu):
    rng = np.random.default_rng(seed)
    n_r = int(np.prod(shape))
    w = torch.from_numpy(rng.random(n_r) ** 2).to(DEV)
    init = torch.from_numpy(np.sort(rng.choice(n_r, n_mu, replace=False))).to(DEV)
    return w, init


def test_noalloc_matches_kmeans_on_two_calls_in_a_row(isdf):
    cases = [((24, 24, 24), (10.0, 10.0, 10.0), 128, 30, 0, 11),
             ((10, 7, 13), (3.0, 2.1, 3.9), 17, 12, 1, 12)]
    for shape, cell, n_mu, iters, flags, seed in cases:
        w, init = _case(seed, shape, n_mu)
        ref = isdf.kmeans(w, shape, cell, n_mu, init, iters, early_stop=bool(flags))
        rc, got = noalloc(isdf, w, shape, cell, n_mu, init, iters, flags)
        torch.cuda.synchronize()
        assert rc == 0
        for k in ("idx", "centroids", "objective", "labels", "stats"):
            assert torch.equal(got[k], ref[k]), k


def test_noalloc_repeated_identical_calls(isdf):
    shape, cell, n_mu, iters = (16, 16, 16), (8.0, 8.0, 8.0), 64, 20
    w, init = _case(3, shape, n_mu)
    _, a = noalloc(isdf, w, shape, cell, n_mu, init, iters)
    _, b = noalloc(isdf, w, shape, cell, n_mu, init, iters)
    torch.cuda.synchronize()
    for k in a:
        assert torch.equal(a[k], b[k]), k


def test_noalloc_after_a_failed_call_and_without_labels(isdf):
    # a call that leaves an error flag in the shared array (an init index outside the grid: every
    # idx -1, stats[2] = -2), then a good call that must equal isdf_kmeans exactly; then a call with
    # labels and objective NULL, where the labels live in the shared array too
    shape, cell, n_mu, iters = (16, 12, 10), (8.0, 6.0, 5.0), 48, 15
    w, init = _case(21, shape, n_mu)
    bad = init.clone()
    bad[3] = int(np.prod(shape)) + 5
    rc, got = noalloc(isdf, w, shape, cell, n_mu, bad, iters)
    torch.cuda.synchronize()
    assert rc == 0 and bool((got["idx"] == -1).all()) and got["stats"][2].item() == -2
    ref = isdf.kmeans(w, shape, cell, n_mu, init, iters)
    rc, got = noalloc(isdf, w, shape, cell, n_mu, init, iters)
    torch.cuda.synchronize()
    assert rc == 0
    for k in ("idx", "centroids", "objective", "labels", "stats"):
        assert torch.equal(got[k], ref[k]), k
    rc, got = noalloc(isdf, w, shape, cell, n_mu, init, iters, labels=False, objective=False)
    torch.cuda.synchronize()
    assert rc == 0
    for k in ("idx", "centroids", "stats"):
        assert torch.equal(got[k], ref[k]), k


def test_noalloc_rejects_problems_beyond_the_scratch_size(isdf):
    # 256^3 points need far more than the fixed 32 MiB array: refused before any launch. The
    # pointers are valid, so the refusal is the size check and not an argument error
    w = torch.zeros(8, dtype=torch.float64, device=DEV)
    init = torch.arange(64, dtype=torch.int64, device=DEV)
    rc, got = noalloc(isdf, w, (256, 256, 256), (10.0, 10.0, 10.0), 64, init, 1)
    assert rc == 8  # ISDF_ERR_UNSUPPORTED
    assert bool((got["idx"] == -7).all())
    # an invalid call (no weights) is reported as such first
    rc, _ = noalloc(isdf, None, (256, 256, 256), (10.0, 10.0, 10.0), 64, init, 1)
    assert rc == 1  # ISDF_ERR_INVALID_ARG
