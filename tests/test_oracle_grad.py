"""Pins for the oracle's adjoint of the Theta fit at fixed interpolation
points: PyTorch CPU autograd through the textbook least-squares formula on an
explicit Z, central finite differences, and the invariants implied by
Theta(Phi U) = Theta(Phi) for unitary U and Theta(a Phi) = Theta(Phi)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2208_07731_gb300 import workload as W


def _small():
    w = W.small_workload(n=6, L=5.0, n_orb=4, n_mu=12, iters=8, ecut=4.0, seed=11)
    phi, psi = W.make_pair(w)
    phi, psi = phi.numpy(), psi.numpy()
    wt = O.weights(phi, psi)
    init = W.init_indices(wt, w.n_mu, 21)
    idx = O.kmeans(wt, (w.n,) * 3, (w.L,) * 3, w.n_mu, init, w.iters)["idx"]
    K = W.loss_matrix(w.n_mu, 31)
    return w, phi, psi, idx, K


def _loss_np(phi, psi, idx, K, dV):
    return O.surrogate_loss(O.fit_theta(phi, psi, idx)["theta"], K, dV)


def _grads(phi, psi, idx, K, dV):
    return O.theta_backward(phi, psi, idx, lambda rows, T: O.surrogate_grad_theta(T, K, dV), block=50)


def test_against_torch_autograd_on_explicit_Z():
    w, phi, psi, idx, K = _small()
    P = torch.tensor(phi, requires_grad=True)
    Q = torch.tensor(psi, requires_grad=True)
    Z = (P[:, :, None] * Q.conj()[:, None, :]).reshape(P.shape[0], -1)
    C = Z[torch.as_tensor(idx)]
    G = C @ C.conj().T
    Theta = torch.linalg.solve(G, (Z @ C.conj().T).T.conj()).T.conj()   # Z C^H (C C^H)^-1
    Kt = torch.tensor(K)
    loss = w.dV * torch.real(torch.sum(Theta.conj() * (Theta @ Kt.T)))
    loss.backward()
    g = _grads(phi, psi, idx, K, w.dV)
    assert abs(loss.item() - _loss_np(phi, psi, idx, K, w.dV)) < 1e-12 * abs(loss.item())
    for ours, ref in ((g["grad_phi"], P.grad.resolve_conj().numpy()), (g["grad_psi"], Q.grad.resolve_conj().numpy())):
        assert np.linalg.norm(ours - ref) < 1e-10 * np.linalg.norm(ref)


def test_central_finite_differences():
    w, phi, psi, idx, K = _small()
    g = _grads(phi, psi, idx, K, w.dV)
    h = 1e-6
    dirs = W.directions((2,) + phi.shape, 8, 77)
    for D in dirs:
        lp = _loss_np(phi + h * D[0], psi + h * D[1], idx, K, w.dV)
        lm = _loss_np(phi - h * D[0], psi - h * D[1], idx, K, w.dV)
        fd = (lp - lm) / (2 * h)
        an = np.real(np.vdot(g["grad_phi"], D[0]) + np.vdot(g["grad_psi"], D[1]))
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3 * np.linalg.norm(g["grad_phi"]))


def test_gauge_invariants():
    w, phi, psi, idx, K = _small()
    g = _grads(phi, psi, idx, K, w.dV)
    for X, Xb in ((phi, g["grad_phi"]), (psi, g["grad_psi"])):
        S = X.conj().T @ Xb
        scale = np.linalg.norm(X) * np.linalg.norm(Xb)
        assert np.linalg.norm(S - S.conj().T) < 1e-11 * scale
        assert abs(np.trace(S)) < 1e-11 * scale


def test_surrogate_gradient_closed_form():
    rng = np.random.default_rng(2)
    T = rng.standard_normal((7, 5)) + 1j * rng.standard_normal((7, 5))
    K = W.loss_matrix(5, 3)
    g = O.surrogate_grad_theta(T, K, 0.5)
    h = 1e-7
    D = rng.standard_normal(T.shape) + 1j * rng.standard_normal(T.shape)
    fd = (O.surrogate_loss(T + h * D, K, 0.5) - O.surrogate_loss(T - h * D, K, 0.5)) / (2 * h)
    assert abs(fd - np.real(np.vdot(g, D))) < 1e-6 * abs(fd)


def test_finite_differences_on_the_nearly_singular_small_case():
    # the 8^3 case of the GPU adjoint test (48 points for 64 orbital products, a nearly singular M): with
    # the oracle's own fits, the non-cancelling central difference at h = 1e-5 is within 1e-6 of the
    # oracle's adjoint on the same 32 directions (at h = 1e-6 FP64 rounding of the fits reaches ~1e-6)
    w = W.small_workload(n=8, L=6.0, n_orb=8, n_mu=48, iters=10, ecut=6.0, seed=5)
    phi, psi = (x.numpy() for x in W.make_pair(w))
    wt = O.weights(phi, psi)
    idx = O.kmeans(wt, (w.n,) * 3, (w.L,) * 3, w.n_mu, W.init_indices(wt, w.n_mu, 17), w.iters)["idx"]
    K = W.loss_matrix(w.n_mu, 23)
    g = O.theta_backward(phi, psi, idx, lambda rows, T: O.surrogate_grad_theta(T, K, w.dV))
    h = 1e-5
    for D in W.directions((2,) + phi.shape, 32, 99):
        tp = O.fit_theta(phi + h * D[0], psi + h * D[1], idx)["theta"]
        tm = O.fit_theta(phi - h * D[0], psi - h * D[1], idx)["theta"]
        fd = w.dV * np.real(np.sum(np.conj(tp - tm) * ((tp + tm) @ K.T))) / (2 * h)
        an = np.real(np.vdot(g["grad_phi"], D[0]) + np.vdot(g["grad_psi"], D[1]))
        assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)
