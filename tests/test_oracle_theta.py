"""Pins for the oracle's interpolation-vector fit (Sec. 2.1, Eqs. theta,
muRownuCol, muRownuColden): the Hadamard identity against an explicitly
formed Z, textbook least squares (scipy lstsq) on Z, the interpolation
property Theta C = I at the selected points, exact reconstruction when the
selected rows span Z, and invariances of Theta."""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from paper_2208_07731_gb300 import workload as W


@pytest.fixture(scope="module")
def tiny():
    w = W.WORKLOADS["tiny"]
    phi, psi = W.make_pair(w)
    phi, psi = phi.numpy(), psi.numpy()
    wt = O.weights(phi, psi)
    init = W.init_indices(wt, w.n_mu, 1000 + w.seed)
    idx = O.kmeans(wt, (w.n,) * 3, (w.L,) * 3, w.n_mu, init, w.iters)["idx"]
    return w, phi, psi, idx


def test_hadamard_identity_against_explicit_Z(tiny):
    w, phi, psi, idx = tiny
    Z = O.explicit_Z(phi, psi)
    C = Z[idx]
    phi_mu, psi_mu = O.gather(phi, psi, idx)
    rows = np.arange(0, w.n_r, 3)
    Y = O.gram_hadamard(phi[rows], psi[rows], phi_mu, psi_mu)
    np.testing.assert_allclose(Y, Z[rows] @ C.conj().T, rtol=0, atol=1e-12 * np.abs(Y).max())
    M = O.form_M(phi_mu, psi_mu)
    np.testing.assert_allclose(M, C @ C.conj().T, rtol=0, atol=1e-12 * np.abs(M).max())
    # C C^H is exactly a row subsample of Z C^H (Sec. 2.4)
    np.testing.assert_allclose(M, O.gram_hadamard(phi[idx], psi[idx], phi_mu, psi_mu), rtol=0, atol=0)
    # M is Hermitian positive definite (a Schur product of two Gram matrices)
    assert np.allclose(M, M.conj().T, atol=0)
    assert np.linalg.eigvalsh(M).min() > 0


def test_theta_matches_textbook_least_squares(tiny):
    w, phi, psi, idx = tiny
    Z = O.explicit_Z(phi, psi)
    C = Z[idx]
    fit = O.fit_theta(phi, psi, idx, block=5000)
    # Theta minimises ||Z - Theta C||_F: Theta^H solves C^H Theta^H = Z^H in least squares
    ref = sla.lstsq(C.conj().T, Z.conj().T)[0].conj().T
    err = np.linalg.norm(fit["theta"] - ref) / np.linalg.norm(ref)
    assert err < 1e-12


def test_interpolation_property_and_normal_equations(tiny):
    w, phi, psi, idx = tiny
    fit = O.fit_theta(phi, psi, idx)
    T = fit["theta"]
    assert np.abs(T[idx] - np.eye(len(idx))).max() < 1e-12
    rows = np.arange(0, w.n_r, 5)
    Y = O.gram_hadamard(phi[rows], psi[rows], fit["phi_mu"], fit["psi_mu"])
    assert np.linalg.norm(Y - T[rows] @ fit["M"]) < 1e-12 * np.linalg.norm(Y)


def test_block_size_independence(tiny):
    w, phi, psi, idx = tiny
    a = O.fit_theta(phi, psi, idx, block=w.n_r)["theta"]
    b = O.fit_theta(phi, psi, idx, block=777)["theta"]
    assert np.linalg.norm(a - b) <= 1e-14 * np.linalg.norm(a)


def test_exact_reconstruction_when_rows_span_Z():
    # N = 2 orbitals: Z has 4 columns, so 4 independent rows span its row space
    # and the fit reproduces Z exactly on every grid point
    rng = np.random.default_rng(3)
    n_r = 40
    phi = rng.standard_normal((n_r, 2)) + 1j * rng.standard_normal((n_r, 2))
    psi = rng.standard_normal((n_r, 2)) + 1j * rng.standard_normal((n_r, 2))
    idx = np.array([2, 11, 23, 37])
    Z = O.explicit_Z(phi, psi)
    T = O.fit_theta(phi, psi, idx)["theta"]
    assert np.linalg.norm(T @ Z[idx] - Z) < 1e-12 * np.linalg.norm(Z)


def test_all_points_selected_gives_identity():
    rng = np.random.default_rng(4)
    phi = rng.standard_normal((8, 4)) + 1j * rng.standard_normal((8, 4))
    psi = rng.standard_normal((8, 4)) + 1j * rng.standard_normal((8, 4))
    idx = np.array([5, 0, 7, 2, 1, 6, 3, 4])
    T = O.fit_theta(phi, psi, idx)["theta"]
    P = np.zeros((8, 8))
    P[idx, np.arange(8)] = 1.0
    assert np.abs(T - P).max() < 1e-12


def test_theta_invariances(tiny):
    w, phi, psi, idx = tiny
    rng = np.random.default_rng(9)
    rows = np.arange(0, w.n_r, 11)
    base = O.fit_theta(phi, psi, idx)["theta"][rows]
    U, _ = np.linalg.qr(rng.standard_normal((w.n_orb, w.n_orb)) + 1j * rng.standard_normal((w.n_orb, w.n_orb)))
    t1 = O.fit_theta(phi @ U, psi, idx)["theta"][rows]
    t2 = O.fit_theta(phi, (0.3 - 1.7j) * psi, idx)["theta"][rows]
    for t in (t1, t2):
        assert np.linalg.norm(t - base) < 1e-11 * np.linalg.norm(base)
    # exchanging the roles of Phi and Psi conjugates Z, hence Theta
    t3 = O.fit_theta(psi, phi, idx)["theta"][rows]
    assert np.linalg.norm(t3 - base.conj()) < 1e-11 * np.linalg.norm(base)
