"""Pins for the oracle's weighted K-means (Sec. 2.2, Eq. opt second form,
Eq. r_k, Algorithm 1): exact rational brute force on tiny grids, closed forms,
the Lloyd descent property and exact invariances."""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2208_07731_gb300 import workload as W


def _rational_lloyd(wts, shape, h, init, iters):
    """Pure-Python Lloyd in exact rational arithmetic (tiny inputs only)."""
    nx, ny, nz = shape
    pts = [(Fraction(ix) * h, Fraction(iy) * h, Fraction(iz) * h)
           for ix in range(nx) for iy in range(ny) for iz in range(nz)]
    wf = [Fraction(x) for x in wts]
    cen = [pts[r] for r in init]
    labels = None
    for _ in range(iters + 1):
        labels = []
        for p in pts:
            d = [sum((p[k] - c[k]) ** 2 for k in range(3)) for c in cen]
            labels.append(min(range(len(cen)), key=lambda m: (d[m], m)))
        if _ == iters:
            break
        new = []
        for m in range(len(cen)):
            sw = sum(wf[r] for r in range(len(pts)) if labels[r] == m)
            if sw == 0:
                new.append(cen[m])
                continue
            new.append(tuple(sum(wf[r] * pts[r][k] for r in range(len(pts)) if labels[r] == m) / sw
                             for k in range(3)))
        cen = new
    return labels, cen


def test_rational_brute_force():
    # dyadic weights and spacing: every w*x is exact, so the oracle's centroid
    # is the correctly rounded exact weighted mean
    rng = np.random.default_rng(5)
    shape = (4, 3, 5)
    h = Fraction(1, 2)
    n_r = 60
    wts = rng.integers(1, 64, size=n_r) / 8.0
    init = np.array([3, 17, 31, 44, 58], dtype=np.int64)
    labels, cen = _rational_lloyd(wts, shape, h, init, 6)
    res = O.kmeans(wts, shape, [2.0, 1.5, 2.5], 5, init, 6)
    assert list(res["labels"]) == labels
    exp = np.array([[float(c) for c in cc] for cc in cen])
    assert np.array_equal(res["centroids"], exp)


def test_single_cluster_is_weighted_mean():
    rng = np.random.default_rng(1)
    shape, cell = (6, 5, 7), [3.0, 2.5, 3.5]
    w = rng.random(210)
    res = O.kmeans(w, shape, cell, 1, np.array([11]), 3)
    x = O.grid_coords(shape, cell)
    np.testing.assert_allclose(res["centroids"][0], (w[:, None] * x).sum(0) / w.sum(), rtol=1e-14)
    # the snapped point is the grid point nearest to the weighted mean
    d = ((x - res["centroids"][0]) ** 2).sum(1)
    assert res["idx"][0] == int(np.argmin(d))


def test_uniform_weights_converge_to_subcube_centres():
    n, h = 8, 0.5
    shape, cell = (n, n, n), [n * h] * 3
    init = np.array([(a * n + b) * n + c for a in (1, 6) for b in (1, 6) for c in (1, 6)], dtype=np.int64)
    res = O.kmeans(np.ones(n ** 3), shape, cell, 8, init, 5)
    exp = np.array([[a, b, c] for a in (1.5 * h, 5.5 * h) for b in (1.5 * h, 5.5 * h) for c in (1.5 * h, 5.5 * h)])
    assert np.array_equal(res["centroids"], exp)
    # all eight sub-cubes have 64 members
    assert np.array_equal(np.bincount(res["labels"], minlength=8), np.full(8, 64))


def test_every_point_its_own_cluster():
    shape, cell = (3, 4, 2), [1.5, 2.0, 1.0]
    n_r = 24
    w = np.linspace(0.5, 2.0, n_r)
    res = O.kmeans(w, shape, cell, n_r, np.arange(n_r), 4)
    assert np.array_equal(res["idx"], np.arange(n_r))
    assert res["objective"][-1] < 1e-25  # fixed-point truncation of w*x leaves ~1e-16 offsets


@pytest.fixture(scope="module")
def tiny_run():
    w = W.WORKLOADS["tiny"]
    phi, psi = W.make_pair(w)
    wt = O.weights(phi.numpy(), psi.numpy())
    init = W.init_indices(wt, w.n_mu, 1000 + w.seed)
    return w, wt, init


def test_objective_non_increasing(tiny_run):
    w, wt, init = tiny_run
    res = O.kmeans(wt, (w.n,) * 3, (w.L,) * 3, w.n_mu, init, w.iters)
    J = res["objective"]
    assert np.all(J[1:] <= J[:-1] * (1 + 1e-12))
    assert J[-1] < J[0]
    assert len(set(res["idx"].tolist())) == w.n_mu and res["empty"] == 0


def test_power_of_two_weight_scaling_is_exact(tiny_run):
    w, wt, init = tiny_run
    a = O.kmeans(wt, (w.n,) * 3, (w.L,) * 3, w.n_mu, init, 20)
    b = O.kmeans(wt * 2.0 ** 37, (w.n,) * 3, (w.L,) * 3, w.n_mu, init, 20)
    assert np.array_equal(a["idx"], b["idx"])
    assert np.array_equal(a["centroids"], b["centroids"])
    assert np.array_equal(a["labels"], b["labels"])


def test_converged_state_is_a_lloyd_fixed_point(tiny_run):
    w, wt, init = tiny_run
    res = O.kmeans(wt, (w.n,) * 3, (w.L,) * 3, w.n_mu, init, 500, early_stop=True)
    assert res["n_iter"] < 500
    x = O.grid_coords((w.n,) * 3, (w.L,) * 3)
    lab, c = res["labels"], res["centroids"]
    # labels are the nearest centroids (brute force, lowest index on ties)
    d = ((x[:, None, :] - c[None, :, :]) ** 2).sum(-1)
    assert np.array_equal(lab, np.argmin(d, axis=1))
    # centroids are the weighted means of their members (Eq. r_k)
    sw = np.bincount(lab, weights=wt, minlength=w.n_mu)
    for k in range(3):
        np.testing.assert_allclose(c[:, k], np.bincount(lab, weights=wt * x[:, k], minlength=w.n_mu) / sw,
                                   rtol=1e-13)
    # the snapped point of each cluster is its nearest member
    for m in range(0, w.n_mu, 9):
        mem = np.nonzero(lab == m)[0]
        assert res["idx"][m] == mem[np.argmin(d[mem, m])]


def test_early_stop_matches_full_run(tiny_run):
    w, wt, init = tiny_run
    full = O.kmeans(wt, (w.n,) * 3, (w.L,) * 3, w.n_mu, init, 300)
    early = O.kmeans(wt, (w.n,) * 3, (w.L,) * 3, w.n_mu, init, 300, early_stop=True)
    assert np.array_equal(full["idx"], early["idx"])
    assert np.array_equal(full["centroids"], early["centroids"])


def test_fixed_point_scale_closed_form():
    # N_r = 13824 -> 14 bits; wmax = 0.75 -> 2^0; L = 10 -> 2^4: s = 126 - 18
    assert O.fixed_point_scale(13824, 0.75, [10.0, 10.0, 10.0]) == 108
    # N_r = 1 -> 1 bit; wmax = 0 -> 2^0; max(L, 1) = 1 = 0.5 * 2^1 -> 1 bit: s = 126 - 2
    assert O.fixed_point_scale(1, 0.0, [0.5, 0.5, 0.5]) == 124


def test_invalid_arguments():
    with pytest.raises(ValueError):
        O.kmeans(np.array([1.0, -1.0]), (2, 1, 1), [1.0, 1.0, 1.0], 1, np.array([0]), 1)
    with pytest.raises(ValueError):
        O.kmeans(np.array([1.0, 1.0]), (2, 1, 1), [1.0, 1.0, 1.0], 1, np.array([5]), 1)


# ---------------------------------------------------------------- single steps (lock-step checks)
def test_single_steps_against_rational_lloyd():
    # the one-step functions restate Algorithm 1's steps: one update from the exact labels of pass t
    # gives the exact rational centroids of pass t + 1 (dyadic inputs), the assignment of every point
    # gives the rational labels, and the snap gives each cluster's nearest member
    rng = np.random.default_rng(9)
    shape = (4, 3, 5)
    h = Fraction(1, 2)
    cell = [2.0, 1.5, 2.5]
    wts = rng.integers(1, 64, size=60) / 8.0
    init = np.array([2, 19, 30, 47, 55], dtype=np.int64)
    for t in range(4):
        lab_t, cen_t = _rational_lloyd(wts, shape, h, init, t)
        _, cen_t1 = _rational_lloyd(wts, shape, h, init, t + 1)
        c_t = np.array([[float(c) for c in cc] for cc in cen_t])
        c_t1 = np.array([[float(c) for c in cc] for cc in cen_t1])
        got = O.kmeans_update(wts, shape, cell, np.array(lab_t), c_t)
        assert np.array_equal(got, c_t1), t
        lab, dist = O.kmeans_assign(shape, cell, c_t, np.arange(60))
        assert list(lab) == lab_t
        pts = O.grid_coords(shape, cell)
        assert np.array_equal(dist, ((pts - c_t[lab]) ** 2).sum(1))


def test_single_steps_reproduce_full_run():
    w = W.small_workload(n=10, n_orb=3, n_mu=24, iters=8, seed=3)
    phi, psi = W.make_pair(w)
    wt = O.weights(phi.numpy(), psi.numpy())
    shape, cell = (w.n,) * 3, (w.L,) * 3
    init = W.init_indices(wt, w.n_mu, 11)
    x = O.grid_coords(shape, cell)
    c = x[init]
    for t in range(6):
        ref = O.kmeans(wt, shape, cell, w.n_mu, init, t)
        assert np.array_equal(ref["centroids"], c), t
        lab, _ = O.kmeans_assign(shape, cell, c, np.arange(w.n_r))
        assert np.array_equal(lab, ref["labels"]), t
        idx, empty = O.kmeans_snap(shape, cell, c, lab)
        assert np.array_equal(idx, ref["idx"]) and empty == ref["empty"]
        c = O.kmeans_update(wt, shape, cell, lab, c)


def test_single_update_weighted_mean_and_empty_cluster():
    # one cluster holding every point: the update is the weighted mean (closed form); a label that no
    # point carries keeps its centroid, and the snap reports that cluster empty
    rng = np.random.default_rng(4)
    shape, cell = (5, 4, 6), [2.5, 2.0, 3.0]
    w = rng.random(120)
    x = O.grid_coords(shape, cell)
    c_in = np.array([[0.1, 0.2, 0.3], [9.0, 9.0, 9.0]])
    got = O.kmeans_update(w, shape, cell, np.zeros(120, np.int32), c_in)
    exp = (w[:, None] * x).sum(0) / w.sum()
    assert np.allclose(got[0], exp, rtol=1e-13, atol=0) and np.array_equal(got[1], c_in[1])
    idx, empty = O.kmeans_snap(shape, cell, got, np.zeros(120, np.int32))
    assert empty == 1 and idx[1] == -1
    assert idx[0] == int(np.argmin(((x - got[0]) ** 2).sum(1)))
