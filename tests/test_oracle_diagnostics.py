"""Pins of the decomposition diagnostics (Appendix A) against explicitly formed Z:
the least-squares residual from scipy's lstsq and the projection residual of
Eq. errorISDF / Eq. proj computed row by row."""
import numpy as np
import scipy.linalg as sla

import oracle as O
from paper_2208_07731_gb300 import workload as W


def _small(seed=3, n_orb=8, n_mu=40, n=8):   # N_mu <= N^2 keeps M = C C^H definite
    w = W.small_workload(n=n, L=6.0, n_orb=n_orb, n_mu=n_mu, iters=8, ecut=6.0, seed=seed)
    phi, psi = W.make_pair(w)
    p, q = phi.numpy(), psi.numpy()
    wt = O.weights(p, q)
    km = O.kmeans(wt, (w.n,) * 3, (w.L,) * 3, w.n_mu, W.init_indices(wt, w.n_mu, 11), w.iters)
    return p, q, km


def test_isdf_error_matches_explicit_least_squares():
    p, q, km = _small()
    idx = km["idx"]
    Z = O.explicit_Z(p, q)
    C = Z[idx]
    X, *_ = sla.lstsq(C.T, Z.T)          # Theta^T minimises ||C^T Theta^T - Z^T||
    res2 = np.linalg.norm(Z - X.T @ C) ** 2
    d = O.isdf_error(p, q, idx, block=100)
    assert abs(d["z2"] - np.linalg.norm(Z) ** 2) < 1e-12 * d["z2"]
    assert abs(d["residual2"] - res2) < 1e-9 * d["z2"]
    assert 0 < d["error"] < 1


def test_isdf_error_vanishes_when_the_points_span_Z():
    # N = 2: Z has rank 4, so 4 points with independent rows reconstruct it exactly
    w = W.small_workload(n=3, L=3.0, n_orb=2, n_mu=4, iters=1, ecut=6.0, seed=2)
    phi, psi = W.make_pair(w)
    idx = np.array([0, 7, 13, 22])
    d = O.isdf_error(phi.numpy(), psi.numpy(), idx)
    assert d["residual2"] < 1e-12 * d["z2"]


def test_cluster_residual_matches_explicit_projections():
    p, q, km = _small(seed=5)
    labels, idx = km["labels"], km["idx"]
    Z = O.explicit_Z(p, q)
    R = 0.0
    for r in range(Z.shape[0]):
        zmu = Z[idx[labels[r]]]
        proj = (Z[r] @ zmu.conj()) / (zmu @ zmu.conj()) * zmu
        R += np.linalg.norm(Z[r] - proj) ** 2
    d = O.cluster_residual(p, q, labels, idx)
    assert abs(d["R"] - R) < 1e-10 * d["z2"]
    # the selected points themselves project exactly
    assert O.cluster_residual(p[idx], q[idx], np.arange(len(idx)), np.arange(len(idx)))["R"] < 1e-12 * d["z2"]
