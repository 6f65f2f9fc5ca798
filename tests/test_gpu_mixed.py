"""GPU parity of the tensor-core (tcgen05, split-FP16) Theta fit against the
CPU FP64 oracle on the same complex64 values upcast to complex128: relative
Frobenius error of Theta and of the reconstructed Z <= 1e-5."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2208_07731_gb300 import workload as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
TOL = 1e-5


@pytest.fixture(scope="module")
def isdf():
    from paper_2208_07731_gb300 import build
    build.build()
    import paper_2208_07731_gb300 as m
    return m


def mixed_small(n_orb=32, n_mu=128, n=24, L=10.0, seed=40):
    return W.Workload(f"mixed{n}", n, L, n_orb, n_mu, "c64", 20, 10.0, (0.25, 0.0, 0.0), "none", seed)


def _setup(w):
    phi, psi = W.make_pair(w)
    phi, psi = phi.to(torch.complex64), psi.to(torch.complex64)
    p64, q64 = phi.numpy(), psi.numpy()
    wt = O.weights(p64, q64)
    init = W.init_indices(wt, w.n_mu, 1000 + w.seed)
    idx = O.kmeans(wt, (w.n,) * 3, (w.L,) * 3, w.n_mu, init, w.iters)["idx"]
    return phi, psi, p64, q64, idx


def recon_error(dT, T_ref, M):
    """||(Theta - Theta_ref) C||_F / ||Theta_ref C||_F = sqrt(tr(dT M dT^H) / tr(T M T^H))."""
    num = np.real(np.sum((dT @ M) * dT.conj()))
    den = np.real(np.sum((T_ref @ M) * T_ref.conj()))
    return float(np.sqrt(max(num, 0.0) / den))


@pytest.mark.parametrize("n_orb,n_mu,max_rows", [(32, 128, 65536), (32, 256, 1000), (64, 192, 4096)])
def test_mixed_theta_small(isdf, n_orb, n_mu, max_rows):
    w = mixed_small(n_orb, n_mu)
    phi, psi, p64, q64, idx = _setup(w)
    plan = isdf.Plan(phi.to(DEV), psi.to(DEV), torch.from_numpy(idx), mode="mixed", max_rows=max_rows)
    th = plan.fit_theta()
    plan.check()
    th = th.cpu().numpy().astype(np.complex128)
    ref = O.fit_theta(p64, q64, idx)
    err = np.linalg.norm(th - ref["theta"]) / np.linalg.norm(ref["theta"])
    assert err < TOL, err
    assert recon_error(th - ref["theta"], ref["theta"], ref["M"]) < TOL
    assert np.abs(th[idx] - np.eye(len(idx))).max() < 10 * TOL


def test_mixed_partial_rows_and_ragged_tail(isdf):
    w = mixed_small(32, 128)
    phi, psi, p64, q64, idx = _setup(w)
    plan = isdf.Plan(phi.to(DEV), psi.to(DEV), torch.from_numpy(idx), mode="mixed", max_rows=777)
    out = torch.zeros((3001, 128 + 4), dtype=torch.complex64, device=DEV)
    plan.fit_theta(10000, 3001, out=out[:, :128])
    plan.check()
    got = out[:, :128].cpu().numpy().astype(np.complex128)
    ref = O.fit_theta(p64, q64, idx)["theta"][10000:13001]
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < TOL
    assert bool((out[:, 128:] == 0).all())


def test_mixed_adjoint_against_fp64_oracle(isdf):
    # tensor-core adjoint (split-FP16 GEMMs, FP32 accumulation) against the FP64 oracle gradient
    w = mixed_small(32, 128)
    phi, psi, p64, q64, idx = _setup(w)
    K = W.loss_matrix(w.n_mu, 5)
    plan = isdf.Plan(phi.to(DEV), psi.to(DEV), torch.from_numpy(idx), mode="mixed", max_rows=5000)
    loss, gphi, gpsi = isdf.surrogate_loss_and_grad(plan, torch.from_numpy(K).to(DEV), w.dV, block=7000)
    plan.check()
    ref = O.theta_backward(p64, q64, idx, lambda rows, T: O.surrogate_grad_theta(T, K, w.dV))
    ref_loss = O.surrogate_loss(O.fit_theta(p64, q64, idx)["theta"], K, w.dV)
    assert abs(loss.item() - ref_loss) < 1e-5 * abs(ref_loss)
    for got, exp in ((gphi, ref["grad_phi"]), (gpsi, ref["grad_psi"])):
        err = np.linalg.norm(got.cpu().numpy() - exp) / np.linalg.norm(exp)
        assert err < 1e-4, err


def test_mixed_adjoint_autograd_grad_theta(isdf):
    # the autograd path (dL/dTheta given, complex64) through the tensor-core adjoint
    w = mixed_small(32, 128)
    phi, psi, p64, q64, idx = _setup(w)
    K = W.loss_matrix(w.n_mu, 6)
    P = phi.to(DEV).requires_grad_(True)
    Q = psi.to(DEV).requires_grad_(True)
    th = isdf.ISDFThetaFn.apply(P, Q, torch.from_numpy(idx), "mixed")
    Kd = torch.from_numpy(K).to(DEV)
    loss = w.dV * torch.real(torch.sum(th.to(torch.complex128).conj() * (th.to(torch.complex128) @ Kd.T)))
    loss.backward()
    ref = O.theta_backward(p64, q64, idx, lambda rows, T: O.surrogate_grad_theta(T, K, w.dV))
    for got, exp in ((P.grad, ref["grad_phi"]), (Q.grad, ref["grad_psi"])):
        err = np.linalg.norm(got.cpu().numpy().astype(np.complex128) - exp) / np.linalg.norm(exp)
        assert err < 1e-4, err
