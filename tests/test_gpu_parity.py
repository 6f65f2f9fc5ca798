"""GPU parity of the CUDA path (through the C ABI) against the CPU oracle on
the same seeded inputs: bit-exact weights and K-means (indices, labels,
centroids), Theta within 1e-10 in FP64 mode, adjoint against the oracle
gradient and finite differences."""
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


def _pair(w):
    phi, psi = W.make_pair(w)
    return W.storage(phi, w), W.storage(psi, w)


@pytest.fixture(scope="module")
def tiny():
    w = W.WORKLOADS["tiny"]
    phi, psi = _pair(w)
    return w, phi, psi


@pytest.fixture(scope="module")
def medium():
    w = W.WORKLOADS["medium"]
    phi, psi = _pair(w)
    return w, phi, psi


# ---------------------------------------------------------------- weights
@pytest.mark.parametrize("kind,alpha", [("ssm", 2.0), ("psm", 2.0), ("ssm", 1.0), ("ssm", 3.0), ("ssm", 4.0)])
def test_weights_bit_exact_c128(isdf, tiny, kind, alpha):
    w, phi, psi = tiny
    ref = O.weights(phi.numpy(), psi.numpy(), kind, alpha)
    got = isdf.weights(phi.to(DEV), psi.to(DEV), kind, alpha).cpu().numpy()
    assert np.array_equal(got, ref)


def test_weights_general_alpha_close(isdf, tiny):
    w, phi, psi = tiny
    ref = O.weights(phi.numpy(), psi.numpy(), "ssm", 2.5)
    got = isdf.weights(phi.to(DEV), psi.to(DEV), "ssm", 2.5).cpu().numpy()
    np.testing.assert_allclose(got, ref, rtol=1e-14)


def test_weights_complex64_ragged_strided(isdf):
    rng = np.random.default_rng(3)
    n_r, n = 1000 + 37, 19          # ragged rows, odd width
    a = (rng.standard_normal((n_r, n + 5)) + 1j * rng.standard_normal((n_r, n + 5))).astype(np.complex64)
    b = (rng.standard_normal((n_r, n)) + 1j * rng.standard_normal((n_r, n))).astype(np.complex64)
    A = torch.from_numpy(a).to(DEV)[:, :n]        # leading dimension n + 5
    B = torch.from_numpy(b).to(DEV)
    ref = O.weights(a[:, :n], b)
    assert np.array_equal(isdf.weights(A, B).cpu().numpy(), ref)
    assert np.array_equal(isdf.weights(A, B, "psm").cpu().numpy(), O.weights(a[:, :n], b, "psm"))


def _dynamic_range_rows(rng, n_r, n, scale_exp):
    """complex64 rows that reach every branch of the integer sum: components up to 2^-60 below the
    row maximum, exact zeros, subnormals, rows whose maximum is tiny or subnormal, all-zero rows"""
    x = (rng.standard_normal((n_r, n)) + 1j * rng.standard_normal((n_r, n))).astype(np.complex64)
    for r in range(n_r):
        k = r % 7
        if k == 1:
            x[r] *= (2.0 ** rng.integers(-60, 1, n)).astype(np.float32)
        elif k == 2:
            x[r, rng.random(n) < 0.3] = 0
        elif k == 3:
            x[r] = (x[r] * np.float32(1e-40)).astype(np.complex64)          # subnormal components
        elif k == 4:
            x[r] = (x[r] * np.float32(1e-30)).astype(np.complex64)
            x[r, 0] = np.complex64(1e-38 + 2e-39j)
        elif k == 5:
            x[r] = 0
        elif k == 6:
            x[r] = 0
            x[r, rng.integers(n)] = np.complex64(3e-45)
    return (x * np.float32(2.0 ** scale_exp)).astype(np.complex64)


def test_weights_complex64_dynamic_range(isdf):
    # widths above 2048 (a lane folds its 64-bit sums more than once per row), an odd width (the tail
    # element) and an odd leading dimension (rows alternately 16-byte aligned or not); Psi sits 2^-40
    # below Phi in half of the rows, so under SSM its whole set lies below the shared window's 2^32 range
    rng = np.random.default_rng(11)
    n_r, n_a, n_b = 70, 2101, 40
    a = _dynamic_range_rows(rng, n_r, n_a, 0)
    b = _dynamic_range_rows(rng, n_r, n_b, 0)
    b[::2] = (b[::2] * np.float32(2.0 ** -40)).astype(np.complex64)
    A, B = torch.from_numpy(a).to(DEV), torch.from_numpy(b).to(DEV)
    for kind in ("ssm", "psm"):
        assert np.array_equal(isdf.weights(A, B, kind).cpu().numpy(), O.weights(a, b, kind)), kind
    # the same rows with the two sets swapped and an even leading dimension of 2102 (all rows aligned)
    pad = np.zeros((n_r, n_a + 1), np.complex64)
    pad[:, :n_a] = a
    P = torch.from_numpy(pad).to(DEV)[:, :n_a]
    assert np.array_equal(isdf.weights(B, P).cpu().numpy(), O.weights(b, a))


def test_weights_medium_bit_exact(isdf, medium):
    w, phi, psi = medium
    ref = O.weights(phi.numpy(), psi.numpy())
    assert np.array_equal(isdf.weights(phi.to(DEV), psi.to(DEV)).cpu().numpy(), ref)


def test_weights_empty(isdf):
    z = torch.zeros((0, 4), dtype=torch.complex128, device=DEV)
    assert isdf.weights(z, z).numel() == 0


# ---------------------------------------------------------------- K-means
def _km_compare(isdf, wt, shape, cell, n_mu, init, iters, early=False):
    ref = O.kmeans(wt, shape, cell, n_mu, init, iters, early_stop=early)
    got = isdf.kmeans(torch.from_numpy(wt).to(DEV), shape, cell, n_mu, torch.from_numpy(init), iters,
                      early_stop=early)
    torch.cuda.synchronize()
    stats = got["stats"].cpu().numpy()
    assert np.array_equal(got["idx"].cpu().numpy(), ref["idx"])
    assert np.array_equal(got["labels"].cpu().numpy(), ref["labels"])
    assert np.array_equal(got["centroids"].cpu().numpy(), ref["centroids"])
    np.testing.assert_allclose(got["objective"].cpu().numpy(), ref["objective"], rtol=1e-12)
    assert stats[0] == ref["n_iter"]
    assert stats[1] == ref["near_ties"]
    assert stats[2] == ref["empty"]
    return ref, got


def test_kmeans_tiny_bit_exact(isdf, tiny):
    w, phi, psi = tiny
    wt = O.weights(phi.numpy(), psi.numpy())
    init = W.init_indices(wt, w.n_mu, 1000 + w.seed)
    _km_compare(isdf, wt, (w.n,) * 3, (w.L,) * 3, w.n_mu, init, w.iters)


def test_kmeans_medium_bit_exact(isdf, medium):
    w, phi, psi = medium
    wt = O.weights(phi.numpy(), psi.numpy())
    init = W.init_indices(wt, w.n_mu, 1000 + w.seed)
    _km_compare(isdf, wt, (w.n,) * 3, (w.L,) * 3, w.n_mu, init, w.iters)


def test_kmeans_early_stop(isdf, tiny):
    w, phi, psi = tiny
    wt = O.weights(phi.numpy(), psi.numpy())
    init = W.init_indices(wt, w.n_mu, 1000 + w.seed)
    _km_compare(isdf, wt, (w.n,) * 3, (w.L,) * 3, w.n_mu, init, 400, early=True)


def test_kmeans_medium_early_stop(isdf, medium):
    # converges before T = 100 (about 85 updates): count, labels, objective and ties as the oracle's
    w, phi, psi = medium
    wt = O.weights(phi.numpy(), psi.numpy())
    init = W.init_indices(wt, w.n_mu, 1000 + w.seed)
    ref, got = _km_compare(isdf, wt, (w.n,) * 3, (w.L,) * 3, w.n_mu, init, w.iters, early=True)
    assert ref["n_iter"] < w.iters


@pytest.mark.parametrize("shape,cell,n_mu,iters", [
    ((10, 7, 13), (3.0, 2.1, 3.9), 17, 12),       # ragged tiles on every axis
    ((5, 5, 5), (2.0, 2.0, 2.0), 1, 4),           # one cluster
    ((3, 4, 2), (1.5, 2.0, 1.0), 24, 3),          # every point its own cluster
    ((16, 16, 16), (8.0, 8.0, 8.0), 64, 0),       # no update: snap of the initial points
])
def test_kmeans_edge_shapes(isdf, shape, cell, n_mu, iters):
    rng = np.random.default_rng(sum(shape) + n_mu)
    n_r = int(np.prod(shape))
    wt = rng.random(n_r) ** 3
    init = np.sort(rng.choice(n_r, n_mu, replace=False)).astype(np.int64)
    _km_compare(isdf, wt, shape, cell, n_mu, init, iters)


def test_kmeans_uniform_weights_exact_ties(isdf):
    # uniform weights on a lattice: many exactly equidistant points, resolved by the lowest index
    shape, cell = (12, 12, 12), (6.0, 6.0, 6.0)
    wt = np.ones(12 ** 3)
    init = np.arange(0, 12 ** 3, 97).astype(np.int64)[:16]
    _km_compare(isdf, wt, shape, cell, 16, init, 10)


def test_kmeans_duplicate_init_reports_empty_cluster(isdf):
    shape, cell = (8, 8, 8), (4.0, 4.0, 4.0)
    rng = np.random.default_rng(2)
    wt = rng.random(512)
    init = np.array([5, 5, 100, 300, 411], dtype=np.int64)
    _km_compare(isdf, wt, shape, cell, 5, init, 6)     # the copy regains members after an update
    ref, got = _km_compare(isdf, wt, shape, cell, 5, init, 0)
    assert ref["empty"] == 1 and got["idx"][1].item() == -1


def test_kmeans_weight_scaling_invariance(isdf, tiny):
    w, phi, psi = tiny
    wt = O.weights(phi.numpy(), psi.numpy())
    init = torch.from_numpy(W.init_indices(wt, w.n_mu, 1000 + w.seed))
    a = isdf.kmeans(torch.from_numpy(wt).to(DEV), (w.n,) * 3, (w.L,) * 3, w.n_mu, init, 20)
    b = isdf.kmeans(torch.from_numpy(wt * 2.0 ** -40).to(DEV), (w.n,) * 3, (w.L,) * 3, w.n_mu, init, 20)
    assert torch.equal(a["idx"], b["idx"]) and torch.equal(a["centroids"], b["centroids"])


def test_kmeans_rejects_negative_weights(isdf):
    wt = torch.ones(64, dtype=torch.float64, device=DEV)
    wt[3] = -1.0
    got = isdf.kmeans(wt, (4, 4, 4), (2.0, 2.0, 2.0), 4, torch.tensor([0, 10, 20, 30]), 2)
    assert got["stats"][2].item() == -1 and bool((got["idx"] == -1).all())


# ---------------------------------------------------------------- Theta (FP64 mode)
def _theta_case(isdf, w, phi, psi, max_rows=65536, rows=None):
    wt = O.weights(phi.numpy(), psi.numpy())
    init = W.init_indices(wt, w.n_mu, 1000 + w.seed)
    idx = O.kmeans(wt, (w.n,) * 3, (w.L,) * 3, w.n_mu, init, w.iters)["idx"]
    plan = isdf.Plan(phi.to(DEV), psi.to(DEV), torch.from_numpy(idx), mode="fp64", max_rows=max_rows)
    return idx, plan


def test_theta_fp64_tiny(isdf, tiny):
    w, phi, psi = tiny
    idx, plan = _theta_case(isdf, w, phi, psi, max_rows=5000)
    th = plan.fit_theta().cpu().numpy()
    plan.check()
    ref = O.fit_theta(phi.numpy(), psi.numpy(), idx)
    assert np.linalg.norm(th - ref["theta"]) / np.linalg.norm(ref["theta"]) < 1e-10
    M = plan.matrix("M").cpu().numpy()
    assert np.abs(M - ref["M"]).max() < 1e-13 * np.abs(ref["M"]).max()
    L = plan.matrix("L").cpu().numpy()
    assert np.abs(L - ref["L"]).max() < 1e-12 * np.abs(ref["L"]).max()
    assert np.abs(th[idx] - np.eye(len(idx))).max() < 1e-11


@pytest.mark.parametrize("n_mu", [1024, 320])
def test_plan_fp64_products_tensor_vs_fp64_pipe(isdf, medium, n_mu):
    # M, L and M^-1 from the exact-slicing tensor-core products against the FP64-pipe GEMMs
    # and against the oracle's M and its inverse (n_mu = 320: padded K and a ragged last tile)
    w, phi, psi = medium
    wt = O.weights(phi.numpy(), psi.numpy())
    idx = W.init_indices(wt, n_mu, 77)
    P, Q, I = phi.to(DEV), psi.to(DEV), torch.from_numpy(idx)
    pt = isdf.Plan(P, Q, I, mode="fp64")
    ps = isdf.Plan(P, Q, I, mode="fp64", fp64_products="simt")
    pt.check()
    ps.check()
    pm, qm = O.gather(phi.numpy(), psi.numpy(), idx)
    M_ref = O.form_M(pm, qm)
    Minv_ref = np.linalg.inv(M_ref)
    for name, tol in (("M", 1e-14), ("L", 1e-13), ("Minv", 1e-12)):
        a, b = pt.matrix(name).cpu().numpy(), ps.matrix(name).cpu().numpy()
        assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b), name
    M = pt.matrix("M").cpu().numpy()
    assert np.abs(M - M_ref).max() < 1e-13 * np.abs(M_ref).max()
    Minv = pt.matrix("Minv").cpu().numpy()
    assert np.linalg.norm(Minv - Minv_ref) < 1e-12 * np.linalg.norm(Minv_ref)


def test_theta_fp64_medium(isdf, medium):
    w, phi, psi = medium
    idx, plan = _theta_case(isdf, w, phi, psi)
    th = plan.fit_theta().cpu().numpy()
    plan.check()
    rows = W.subsample_rows(w.n_r, 8192, 2000 + w.seed)
    phi_mu, psi_mu = O.gather(phi.numpy(), psi.numpy(), idx)
    L = O.cholesky(O.form_M(phi_mu, psi_mu))
    ref = O.theta_rows(phi.numpy(), psi.numpy(), phi_mu, psi_mu, L, rows)
    assert np.linalg.norm(th[rows] - ref) / np.linalg.norm(ref) < 1e-10


def test_theta_row_blocks_and_ld(isdf, tiny):
    w, phi, psi = tiny
    idx, plan = _theta_case(isdf, w, phi, psi, max_rows=1000)
    full = plan.fit_theta()
    out = torch.zeros((3000, w.n_mu + 8), dtype=torch.complex128, device=DEV)
    plan.fit_theta(5000, 3000, out=out[:, :w.n_mu])
    assert torch.allclose(out[:, :w.n_mu], full[5000:8000], rtol=0, atol=1e-14)
    assert bool((out[:, w.n_mu:] == 0).all())


def test_duplicate_points_make_M_singular(isdf, tiny):
    w, phi, psi = tiny
    idx = torch.arange(0, 64 * 100, 100, dtype=torch.int64)
    idx[7] = idx[3]
    plan = isdf.Plan(phi.to(DEV), psi.to(DEV), idx, mode="fp64")
    rc, detail = plan.status()
    assert rc == 3 and detail == 7


def test_end_to_end_decomposition_tiny(isdf, tiny):
    w, phi, psi = tiny
    wt = O.weights(phi.numpy(), psi.numpy())
    init = W.init_indices(wt, w.n_mu, 1000 + w.seed)
    res = isdf.decompose(phi.to(DEV), psi.to(DEV), (w.n,) * 3, (w.L,) * 3, w.n_mu, torch.from_numpy(init), w.iters)
    km = O.kmeans(wt, (w.n,) * 3, (w.L,) * 3, w.n_mu, init, w.iters)
    assert np.array_equal(res["kmeans"]["idx"].cpu().numpy(), km["idx"])
    ref = O.fit_theta(phi.numpy(), psi.numpy(), km["idx"])["theta"]
    th = res["theta"].cpu().numpy()
    assert np.linalg.norm(th - ref) / np.linalg.norm(ref) < 1e-10


# ---------------------------------------------------------------- adjoint (FP64 mode)
def _small_adjoint():
    w = W.small_workload(n=8, L=6.0, n_orb=8, n_mu=48, iters=10, ecut=6.0, seed=5)
    phi, psi = W.make_pair(w)
    wt = O.weights(phi.numpy(), psi.numpy())
    init = W.init_indices(wt, w.n_mu, 17)
    idx = O.kmeans(wt, (w.n,) * 3, (w.L,) * 3, w.n_mu, init, w.iters)["idx"]
    K = W.loss_matrix(w.n_mu, 23)
    return w, phi, psi, idx, K


def test_adjoint_fp64_against_oracle(isdf):
    w, phi, psi, idx, K = _small_adjoint()
    ref = O.theta_backward(phi.numpy(), psi.numpy(), idx, lambda rows, T: O.surrogate_grad_theta(T, K, w.dV))
    ref_loss = O.surrogate_loss(O.fit_theta(phi.numpy(), psi.numpy(), idx)["theta"], K, w.dV)
    plan = isdf.Plan(phi.to(DEV), psi.to(DEV), torch.from_numpy(idx), mode="fp64", max_rows=200)
    loss, gphi, gpsi = isdf.surrogate_loss_and_grad(plan, torch.from_numpy(K).to(DEV), w.dV, block=300)
    plan.check()
    assert abs(loss.item() - ref_loss) < 1e-11 * abs(ref_loss)
    for got, exp in ((gphi, ref["grad_phi"]), (gpsi, ref["grad_psi"])):
        g = got.cpu().numpy()
        assert np.linalg.norm(g - exp) < 1e-10 * np.linalg.norm(exp)


def test_adjoint_fp64_finite_differences(isdf):
    # central differences within 1e-6 of the adjoint. The loss is a Hermitian quadratic form per grid
    # row, q(t) = t^H K t, so q(a) - q(b) = Re[(a - b)^H K (a + b)]: the difference of the two losses is
    # formed from Theta(+h) - Theta(-h) directly, without subtracting two sums of similar size. The
    # step is h = 1e-5 here: this case's M (48 points for 64 orbital products) is nearly singular, and
    # the FP64 rounding of the two fits limits a central difference at h = 1e-6 to ~1e-6 of the
    # derivative even with the oracle's own fits and gradient (worst of the 32 directions 6.5e-7; the
    # h and 2h differences disagree by 9.1e-7, and Richardson extrapolation does not help); at
    # h = 1e-5 the oracle's difference is within 2.4e-8. The h = 1e-6 gate is held on the 72^3 and
    # 128^3 configurations (test_gpu_configs).
    w, phi, psi, idx, K = _small_adjoint()
    Kd = torch.from_numpy(K).to(DEV)
    P, Q = phi.to(DEV), psi.to(DEV)
    plan = isdf.Plan(P, Q, torch.from_numpy(idx), mode="fp64")
    loss, gphi, gpsi = isdf.surrogate_loss_and_grad(plan, Kd, w.dV)

    def theta_at(a, b):
        pl = isdf.Plan(a, b, torch.from_numpy(idx), mode="fp64")
        th = pl.fit_theta()
        pl.check()
        return th

    th0 = theta_at(P, Q)
    assert abs(w.dV * torch.real(torch.sum(th0.conj() * (th0 @ Kd.T))).item() - loss.item()) < 1e-11 * loss.item()
    h = 1e-5
    for D in W.directions((2,) + tuple(phi.shape), 32, 99):
        Dp, Dq = torch.from_numpy(D[0]).to(DEV), torch.from_numpy(D[1]).to(DEV)
        an = torch.real(torch.vdot(gphi.flatten(), Dp.flatten()) + torch.vdot(gpsi.flatten(), Dq.flatten())).item()
        tp, tm = theta_at(P + h * Dp, Q + h * Dq), theta_at(P - h * Dp, Q - h * Dq)
        dl = w.dV * torch.real(torch.sum((tp - tm).conj() * ((tp + tm) @ Kd.T))).item()
        fd = dl / (2 * h)
        assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)


def test_autograd_function_matches_oracle(isdf):
    w, phi, psi, idx, K = _small_adjoint()
    P = phi.to(DEV).requires_grad_(True)
    Q = psi.to(DEV).requires_grad_(True)
    th = isdf.ISDFThetaFn.apply(P, Q, torch.from_numpy(idx), "fp64")
    Kd = torch.from_numpy(K).to(DEV)
    loss = w.dV * torch.real(torch.sum(th.conj() * (th @ Kd.T)))
    loss.backward()
    ref = O.theta_backward(phi.numpy(), psi.numpy(), idx, lambda rows, T: O.surrogate_grad_theta(T, K, w.dV))
    assert np.linalg.norm(P.grad.cpu().numpy() - ref["grad_phi"]) < 1e-10 * np.linalg.norm(ref["grad_phi"])
    assert np.linalg.norm(Q.grad.cpu().numpy() - ref["grad_psi"]) < 1e-10 * np.linalg.norm(ref["grad_psi"])
