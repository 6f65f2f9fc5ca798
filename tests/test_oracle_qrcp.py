"""Pins of the randomized-QRCP comparator (Sec. 2.1, Eq. QRCP): the sketch equals
Z G with an explicitly formed Z and Khatri-Rao random columns; the pivots equal
LAPACK's column-pivoted QR (scipy) on the same matrix; |R_kk| is non-increasing
and equals LAPACK's |diag R|; a matrix of exact rank k leaves no residual after
k pivots."""
import numpy as np
import scipy.linalg as sla

import oracle as O
from paper_2208_07731_gb300 import workload as W


def _crandn(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)


def test_sketch_is_Z_times_khatri_rao_columns():
    w = W.small_workload(n=6, L=5.0, n_orb=3, n_mu=4, iters=1, ecut=4.0, seed=2)
    phi, psi = (x.numpy() for x in W.make_pair(w))
    rng = np.random.default_rng(1)
    A, B = _crandn(rng, 3, 7), _crandn(rng, 3, 7)
    Z = O.explicit_Z(phi, psi)                                   # columns (i, j), i major
    G = np.stack([np.kron(A[:, k], B[:, k].conj()) for k in range(7)], axis=1)
    np.testing.assert_allclose(O.qrcp_sketch(phi, psi, A, B), Z @ G, rtol=1e-12, atol=1e-14)


def test_pivots_match_lapack_qrcp():
    rng = np.random.default_rng(3)
    S = _crandn(rng, 400, 24) * np.exp(rng.standard_normal((400, 1)))   # rows of varying norm
    got = O.qrcp_points(S, 20)
    Q, R, P = sla.qr(S.T, pivoting=True, mode="economic")
    assert np.array_equal(got["idx"], P[:20])
    np.testing.assert_allclose(got["rdiag"], np.abs(np.diag(R))[:20], rtol=1e-10)
    assert np.all(np.diff(got["rdiag"]) <= 1e-12 * got["rdiag"][0])


def test_exact_rank_is_exhausted():
    rng = np.random.default_rng(4)
    S = _crandn(rng, 300, 5) @ _crandn(rng, 5, 12)                      # rank 5
    got = O.qrcp_points(S, 6)
    assert got["rdiag"][5] < 1e-12 * got["rdiag"][0]
    assert len(set(got["idx"][:5].tolist())) == 5
