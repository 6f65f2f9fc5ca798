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


# ---------------------------------------------------------------- the sums' reading (exact, rounded once)
def _rn(q):
    """Round a non-negative rational to the nearest double (ties to even) by exact arithmetic."""
    from fractions import Fraction
    if q == 0:
        return 0.0
    lo = float(q)   # Python's float(Fraction) is correctly rounded
    assert Fraction(lo) - q <= Fraction(np.spacing(lo)) / 2
    return lo


def _random_rows(rng, n_rows, n, spread):
    mag = np.exp(rng.uniform(-spread, spread, size=(n_rows, n)))
    return (rng.standard_normal((n_rows, n)) + 1j * rng.standard_normal((n_rows, n))) * mag


def test_alpha2_sum_is_the_correctly_rounded_exact_sum():
    # the SSM weight (alpha = 2) is the exact sum of the squared components rounded once: checked
    # against rational arithmetic on rows whose entries span many binades, complex128 and complex64
    from fractions import Fraction
    rng = np.random.default_rng(31)
    for dtype in (np.complex128, np.complex64):
        phi = _random_rows(rng, 40, 9, 12.0).astype(dtype)
        psi = _random_rows(rng, 40, 6, 12.0).astype(dtype)
        got = O.weights(phi, psi)
        for r in range(40):
            exact = sum(Fraction(float(v)) ** 2 for z in list(phi[r]) + list(psi[r]) for v in (z.real, z.imag))
            assert got[r] == _rn(exact), (dtype, r)
        # PSM: the two exact sums, each rounded, multiplied once
        got = O.weights(phi, psi, "psm")
        for r in range(40):
            sa = _rn(sum(Fraction(float(v)) ** 2 for z in phi[r] for v in (z.real, z.imag)))
            sb = _rn(sum(Fraction(float(v)) ** 2 for z in psi[r] for v in (z.real, z.imag)))
            assert got[r] == sa * sb


def test_sums_do_not_depend_on_column_order():
    rng = np.random.default_rng(32)
    phi = _random_rows(rng, 64, 33, 6.0)
    psi = _random_rows(rng, 64, 17, 6.0)
    pp, qp = rng.permutation(33), rng.permutation(17)
    for kind, a in (("ssm", 2.0), ("ssm", 1.0), ("ssm", 3.0), ("psm", 2.0)):
        assert np.array_equal(O.weights(phi, psi, kind, a), O.weights(phi[:, pp], psi[:, qp], kind, a))
    # the SSM weight with the two sets swapped is the same sum
    assert np.array_equal(O.weights(phi, psi), O.weights(psi, phi))


def test_alpha_terms_summed_exactly():
    # alpha != 2: the FP64 terms |z|^alpha, summed exactly and rounded once
    from fractions import Fraction
    rng = np.random.default_rng(33)
    phi = _random_rows(rng, 20, 7, 4.0)
    psi = _random_rows(rng, 20, 5, 4.0)
    for a in (1.0, 3.0, 2.5):
        got = O.weights(phi, psi, "ssm", a)
        for r in range(20):
            terms = []
            for z in list(phi[r]) + list(psi[r]):
                m = z.real * z.real
                m = m + z.imag * z.imag
                terms.append(np.sqrt(m) if a == 1.0 else (m * np.sqrt(m) if a == 3.0 else m ** (0.5 * a)))
            assert got[r] == _rn(sum(Fraction(float(t)) for t in terms)), (a, r)


def test_all_zero_row_and_single_component():
    phi = np.zeros((3, 4), np.complex128)
    psi = np.zeros((3, 2), np.complex128)
    phi[1, 2] = 3e-100 + 0j          # a lone tiny component: its square, exactly rounded
    psi[2, 0] = 0.0 + 1.5j
    w = O.weights(phi, psi)
    assert w[0] == 0.0 and w[2] == 2.25
    assert w[1] == _rn(__import__("fractions").Fraction(3e-100) ** 2)
