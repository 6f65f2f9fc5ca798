"""Pins for the oracle's weight function (Sec. 2.2, Eqs. weight function and
weight function 2) against hand-worked values, a normalisation invariant and
the explicit transposed Khatri-Rao product (Appendix A, Eq. Zmu)."""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2208_07731_gb300 import workload as W

GOLD = os.path.join(os.path.dirname(__file__), "golden", "weights_hand.json")


def _cplx(rows):
    return np.array([[complex(a, b) for a, b in row] for row in rows], dtype=np.complex128)


def test_hand_worked_values():
    g = json.load(open(GOLD))
    phi, psi = _cplx(g["phi"]), _cplx(g["psi"])
    for key, exp in g["expected"].items():
        if key == "psm":
            got = O.weights(phi, psi, "psm")
        else:
            got = O.weights(phi, psi, "ssm", float(key[-1]))
        np.testing.assert_allclose(got, exp, rtol=1e-15, atol=0, err_msg=key)


@pytest.fixture(scope="module")
def tiny():
    w = W.WORKLOADS["tiny"]
    phi, psi = W.make_pair(w)
    return w, phi.numpy(), psi.numpy()


def test_ssm_normalisation(tiny):
    # orthonormal orbitals: sum_r w(r) dV = N_phi + N_psi exactly for alpha = 2
    w, phi, psi = tiny
    s = O.weights(phi, psi).sum() * w.dV
    assert abs(s - 2 * w.n_orb) < 1e-11 * 2 * w.n_orb


def test_ssm_is_sum_of_densities(tiny):
    w, phi, psi = tiny
    rho = np.linalg.norm(phi, axis=1) ** 2 + np.linalg.norm(psi, axis=1) ** 2
    np.testing.assert_allclose(O.weights(phi, psi), rho, rtol=1e-13)


def test_psm_equals_row_norm_of_Z(tiny):
    # Eq. Zmu: Z(r).Z*(r) = (sum_i |phi_i|^2)(sum_j |psi_j|^2)
    w, phi, psi = tiny
    rows = np.arange(0, w.n_r, 7)
    Z = O.explicit_Z(phi[rows], psi[rows])
    np.testing.assert_allclose(O.weights(phi[rows], psi[rows], "psm"), np.sum(np.abs(Z) ** 2, axis=1), rtol=1e-13)


def test_alpha_family_against_moduli(tiny):
    w, phi, psi = tiny
    rows = slice(0, 500)
    for a in (1.0, 3.0, 4.0, 2.5):
        exp = np.sum(np.abs(phi[rows]) ** a, axis=1) + np.sum(np.abs(psi[rows]) ** a, axis=1)
        np.testing.assert_allclose(O.weights(phi[rows], psi[rows], "ssm", a), exp, rtol=1e-13)


def test_complex64_input_is_upcast_exactly(tiny):
    w, phi, psi = tiny
    p64, q64 = phi[:300].astype(np.complex64), psi[:300].astype(np.complex64)
    a = O.weights(p64, q64)
    b = O.weights(p64.astype(np.complex128), q64.astype(np.complex128))
    assert np.array_equal(a, b)
