"""GPU parity of the randomized-QRCP comparator (Sec. 2.1, Eq. QRCP;
isdf_qrcp_points) against the oracle on the same seeded sketch matrices:
identical pivots (both sides decide in FP64; near ties within 1e-9 would be
resolved by the lowest index on the GPU) and |R_kk| to 1e-10. At the medium
size, where the oracle's greedy loop is too slow, the first pivot against the
oracle's sketch and size-independent properties."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2208_07731_gb300 import workload as W

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def isdf():
    from paper_2208_07731_gb300 import build
    build.build()
    import paper_2208_07731_gb300 as m
    return m


def _crandn(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)


def test_qrcp_tiny_matches_oracle(isdf):
    w = W.WORKLOADS["tiny"]
    phi, psi = W.make_pair(w)
    rng = np.random.default_rng(31)
    p = w.n_mu + 8
    A, B = _crandn(rng, w.n_orb, p), _crandn(rng, w.n_orb, p)
    ref = O.qrcp_points(O.qrcp_sketch(phi.numpy(), psi.numpy(), A, B), w.n_mu)
    got = isdf.qrcp_points(phi.to(DEV), psi.to(DEV), torch.from_numpy(A), torch.from_numpy(B), w.n_mu)
    assert np.array_equal(got["idx"].cpu().numpy(), ref["idx"])
    np.testing.assert_allclose(got["rdiag"].cpu().numpy(), ref["rdiag"], rtol=1e-10)


def test_qrcp_unequal_widths_c64_strided(isdf):
    rng = np.random.default_rng(32)
    n_r, n_phi, n_psi, p, n_mu = 2000 + 17, 12, 20, 40, 32
    a = _crandn(rng, n_r, n_phi + 3).astype(np.complex64)
    b = _crandn(rng, n_r, n_psi).astype(np.complex64)
    A, B = _crandn(rng, n_phi, p), _crandn(rng, n_psi, p)
    ref = O.qrcp_points(O.qrcp_sketch(a[:, :n_phi], b, A, B), n_mu)
    got = isdf.qrcp_points(torch.from_numpy(a).to(DEV)[:, :n_phi], torch.from_numpy(b).to(DEV),
                           torch.from_numpy(A), torch.from_numpy(B), n_mu)
    assert np.array_equal(got["idx"].cpu().numpy(), ref["idx"])
    np.testing.assert_allclose(got["rdiag"].cpu().numpy(), ref["rdiag"], rtol=1e-10)


def test_qrcp_medium_properties(isdf):
    w = W.WORKLOADS["medium"]
    phi, psi = W.make_pair(w)
    rng = np.random.default_rng(33)
    p = w.n_mu + 16
    A, B = _crandn(rng, w.n_orb, p), _crandn(rng, w.n_orb, p)
    got = isdf.qrcp_points(phi.to(DEV), psi.to(DEV), torch.from_numpy(A), torch.from_numpy(B), w.n_mu)
    idx, rd = got["idx"].cpu().numpy(), got["rdiag"].cpu().numpy()
    assert len(set(idx.tolist())) == w.n_mu and idx.min() >= 0 and idx.max() < w.n_r
    assert np.all(np.diff(rd) <= 1e-10 * rd[0])
    S = O.qrcp_sketch(phi.numpy(), psi.numpy(), A, B)
    n2 = np.sum(np.abs(S) ** 2, axis=1)
    assert idx[0] == int(np.argmax(n2))
    assert rd[0] == pytest.approx(np.sqrt(n2.max()), rel=1e-12)


def test_qrcp_as_many_points_as_sketch_columns(isdf):
    rng = np.random.default_rng(34)
    n_r, n, p = 700, 6, 30
    a, b = _crandn(rng, n_r, n), _crandn(rng, n_r, n)
    A, B = _crandn(rng, n, p), _crandn(rng, n, p)
    ref = O.qrcp_points(O.qrcp_sketch(a, b, A, B), p)
    got = isdf.qrcp_points(torch.from_numpy(a).to(DEV), torch.from_numpy(b).to(DEV), torch.from_numpy(A),
                           torch.from_numpy(B), p)
    assert np.array_equal(got["idx"].cpu().numpy(), ref["idx"])
    np.testing.assert_allclose(got["rdiag"].cpu().numpy(), ref["rdiag"], rtol=1e-9)
