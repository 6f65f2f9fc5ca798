"""Pins of the exchange-application oracle (Sec. 2.3: Eq. v, Eq. v2, Eq. V_mu)
against facts fixed outside it: plane waves are eigenfunctions of the periodic
interaction, the screened (erfc) potential of a Gaussian charge has a closed
form, the bare Coulomb potential satisfies Poisson's equation (checked with an
8th-order finite-difference Laplacian), the ISDF exchange equals the direct
exchange of Eq. v when the decomposition is exact, and the exchange energy of
an orbital set with itself is real and negative."""
import math

import numpy as np
import pytest
from scipy.special import erf

import oracle as O
from paper_2208_07731_gb300 import workload as W


def _coords(shape, cell):
    nx, ny, nz = shape
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    h = [c / n for c, n in zip(cell, shape)]
    return np.stack([ix.ravel() * h[0], iy.ravel() * h[1], iz.ravel() * h[2]], axis=1)


@pytest.mark.parametrize("kind,omega,q", [("coulomb", 0.0, (0.0, 0.0, 0.0)), ("erfc", 0.7, (0.0, 0.0, 0.0)),
                                          ("coulomb", 0.0, (0.11, -0.2, 0.05)), ("erfc", 0.3, (0.3, 0.0, -0.1))])
def test_plane_waves_are_eigenfunctions(kind, omega, q):
    shape, cell = (8, 6, 10), (5.0, 4.0, 6.5)
    x = _coords(shape, cell)
    # the Nyquist index n/2 of an even axis is read as the frequency -n/2 (fftfreq order)
    for m in [(1, 0, 0), (0, -2, 3), (3, 2, -4), (-4, -3, -5), (0, 0, 0)]:
        G = np.array([2 * math.pi * m[a] / cell[a] for a in range(3)])
        zeta = np.exp(1j * (x @ G))[:, None]
        g2 = float(np.sum((G + np.array(q)) ** 2))
        if g2 == 0.0:
            lam = 0.0 if kind == "coulomb" else math.pi / omega ** 2
        elif kind == "coulomb":
            lam = 4 * math.pi / g2                               # Fourier transform of 1/r
        else:
            lam = 4 * math.pi / g2 * (1 - math.exp(-g2 / (4 * omega ** 2)))   # of erfc(omega r)/r
        V = O.poisson(zeta, shape, cell, kind, omega, q)
        np.testing.assert_allclose(V, lam * zeta, rtol=0, atol=1e-12 * max(lam, 1.0))


def test_erfc_potential_of_a_gaussian_charge():
    # rho = unit Gaussian charge (width sigma) at the cell centre; the erfc(omega r)/r potential
    # is [erf(r / sqrt(2 sigma^2)) - erf(r / sqrt(2 sigma^2 + 1/omega^2))] / r (Gaussian convolutions);
    # the kernel is short-ranged, so the periodic images are below 1e-18 here
    n, L, sigma, omega = 64, 20.0, 0.8, 1.0
    shape, cell = (n,) * 3, (L,) * 3
    x = _coords(shape, cell)
    d = x - L / 2
    r = np.sqrt(np.sum(d * d, axis=1))
    rho = np.exp(-r * r / (2 * sigma ** 2)) / (2 * math.pi * sigma ** 2) ** 1.5
    V = O.poisson(rho[:, None], shape, cell, "erfc", omega)[:, 0]
    s2 = math.sqrt(2 * sigma ** 2 + 1 / omega ** 2)
    with np.errstate(invalid="ignore", divide="ignore"):
        ref = (erf(r / (math.sqrt(2) * sigma)) - erf(r / s2)) / r
    ref[r == 0] = math.sqrt(2 / math.pi) / sigma - 2 / (math.sqrt(math.pi) * s2)
    assert np.max(np.abs(V.imag)) < 1e-14
    np.testing.assert_allclose(V.real, ref, rtol=0, atol=1e-11)


def test_coulomb_potential_solves_poisson_equation():
    # -lap V = 4 pi (rho - <rho>) for the bare kernel with the G = 0 term removed
    n, L = 64, 16.0
    shape, cell = (n,) * 3, (L,) * 3
    x = _coords(shape, cell)
    rng = np.random.default_rng(4)
    rho = np.zeros(x.shape[0])
    for c, s, qc in zip(rng.uniform(0, L, (3, 3)), (1.0, 1.2, 1.1), (1.0, -0.5, 0.8)):
        d = (x - c + L / 2) % L - L / 2
        rho += qc * np.exp(-np.sum(d * d, 1) / (2 * s * s)) / (2 * math.pi * s * s) ** 1.5
    V = O.poisson(rho[:, None], shape, cell, "coulomb")[:, 0].real.reshape(shape)
    h = L / n
    c8 = [-205 / 72, 8 / 5, -1 / 5, 8 / 315, -1 / 560]              # 8th-order central second derivative
    lap = np.zeros_like(V)
    for ax in range(3):
        lap += c8[0] * V
        for k in range(1, 5):
            lap += c8[k] * (np.roll(V, k, axis=ax) + np.roll(V, -k, axis=ax))
    lap /= h * h
    src = 4 * math.pi * (rho - rho.mean()).reshape(shape)
    assert np.max(np.abs(-lap - src)) < 2e-5 * np.max(np.abs(src))
    assert abs(V.mean()) < 1e-12 * np.max(np.abs(V))                 # no G = 0 component


def test_erfc_kernel_tends_to_coulomb_for_small_omega():
    shape, cell = (6, 8, 5), (3.0, 4.0, 2.5)
    kc = O.kernel_hat(shape, cell, "coulomb")
    ke = O.kernel_hat(shape, cell, "erfc", 1e-3)
    mask = kc > 0
    np.testing.assert_allclose(ke[mask], kc[mask], rtol=1e-15)
    assert ke[0, 0, 0] == pytest.approx(math.pi / 1e-6)


def test_exchange_apply_brute_force():
    rng = np.random.default_rng(8)
    n_r, n_phi, n_psi, n_mu = 30, 3, 4, 5
    c = lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)
    phi, psi, V = c(n_r, n_phi), c(n_r, n_psi), c(n_r, n_mu)
    idx = np.array([3, 17, 0, 29, 11])
    out = np.zeros((n_r, n_psi), complex)
    for r in range(n_r):
        for j in range(n_psi):
            for mu in range(n_mu):
                for i in range(n_phi):
                    out[r, j] -= V[r, mu] * phi[r, i] * np.conj(phi[idx[mu], i]) * psi[idx[mu], j]
    np.testing.assert_allclose(O.exchange_apply(phi, psi, idx, V), out, rtol=1e-13, atol=1e-13)
    rows = [2, 5, 29]
    np.testing.assert_allclose(O.exchange_apply(phi, psi, idx, V, rows=rows), out[rows], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("kind,omega", [("coulomb", 0.0), ("erfc", 0.4)])
def test_isdf_exchange_equals_direct_when_the_decomposition_is_exact(kind, omega):
    # N = 2: the pair products phi_i* psi_j span 4 functions, so 4 generic points fit them exactly
    w = W.small_workload(n=6, L=5.0, n_orb=2, n_mu=4, iters=1, ecut=4.0, seed=3)
    phi, psi = (x.numpy() for x in W.make_pair(w))
    shape, cell = (w.n,) * 3, (w.L,) * 3
    idx = np.array([1, 40, 97, 150])
    # Theta for Z'(r) = psi_j(r) conj(phi_i(r)) = phi_i*(r) psi_j(r): the pair in the order (psi, phi)
    theta = O.fit_theta(psi, phi, idx)["theta"]
    V = O.poisson(theta, shape, cell, kind, omega)
    isdf = O.exchange_apply(phi, psi, idx, V)
    direct = O.exchange_direct(phi, psi, shape, cell, kind, omega)
    assert np.linalg.norm(isdf - direct) < 1e-10 * np.linalg.norm(direct)


def test_exchange_energy_is_real_and_negative():
    w = W.small_workload(n=6, L=5.0, n_orb=3, n_mu=9, iters=1, ecut=4.0, seed=6)
    phi = W.make_orbitals(w, 0).numpy()
    shape, cell = (w.n,) * 3, (w.L,) * 3
    vx = O.exchange_direct(phi, phi, shape, cell, "coulomb")
    E = np.sum(phi.conj() * vx) * w.dV
    assert abs(E.imag) < 1e-12 * abs(E.real)
    assert E.real < 0
