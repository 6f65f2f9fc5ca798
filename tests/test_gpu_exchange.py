"""GPU parity of the ISDF exchange application (Sec. 2.3; isdf_exchange_*)
against the oracle on the same seeded inputs.

Tolerances, from the arithmetic: the FP64 FFT carries ~log2(N_r) eps of
relative error per column, so V agrees to 1e-12 of max |V|; the FP32 FFT of the
mixed mode to 1e-5. The products of the application are FP64-grade (exact
integer slicing) in FP64 mode and for shapes the split kernels do not take, so
the applied exchange agrees to 1e-11 of its Frobenius norm on identical inputs;
the mixed mode's split-FP16 x3 products (2^-22 per product, FP32 sums) to 1e-5."""
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
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _maxrel(got, ref):
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


@pytest.mark.parametrize("kernel,omega,q", [("coulomb", 0.0, None), ("erfc", 0.106, None),
                                            ("coulomb", 0.0, (0.13, -0.07, 0.02))])
def test_potential_fp64_tiny(isdf, kernel, omega, q):
    shape, cell, n_mu = (24, 24, 24), (10.0, 10.0, 10.0), 128
    theta = _crandn(np.random.default_rng(1), 24 ** 3, n_mu)
    ref = O.poisson(theta, shape, cell, kernel, omega, q or (0.0, 0.0, 0.0))
    ex = isdf.Exchange(shape, cell, n_mu, 4, 4, kernel=kernel, omega=omega, q=q)
    got = ex.potential(torch.from_numpy(theta).to(DEV)).cpu().numpy()
    ex.check()
    assert _maxrel(got, ref) < 1e-12


def test_potential_ragged_columns_strided_radix5_in_place(isdf):
    # n_mu = 100 is not a multiple of the 16-column tile; rows have 4 padding columns;
    # the 20-point axis takes a radix-5 stage; the transform overwrites its input
    shape, cell, n_mu = (20, 18, 16), (7.5, 6.0, 5.5), 100
    rng = np.random.default_rng(2)
    buf = _crandn(rng, 20 * 18 * 16, n_mu + 4)
    ref = O.poisson(buf[:, :n_mu], shape, cell, "erfc", 0.3)
    ex = isdf.Exchange(shape, cell, n_mu, 3, 5, kernel="erfc", omega=0.3)
    d = torch.from_numpy(buf).to(DEV)
    view = d[:, :n_mu]
    ex.potential(view, out=view)
    got = d.cpu().numpy()
    assert _maxrel(got[:, :n_mu], ref) < 1e-12
    assert np.array_equal(got[:, n_mu:], buf[:, n_mu:])     # padding untouched


@pytest.mark.parametrize("ld", [102, 101])
def test_potential_ragged_tile_c64_padded_rows(isdf, ld):
    # 24^3 takes the compile-time FFT; n_mu = 100 leaves a 4-column last tile; rows padded to an
    # even (ld = 102) and an odd (ld = 101) number of complex64 entries
    shape, cell, n_mu = (24, 24, 24), (9.0, 9.0, 9.0), 100
    buf = _crandn(np.random.default_rng(21), 24 ** 3, ld).astype(np.complex64)
    ref = O.poisson(buf[:, :n_mu], shape, cell, "coulomb")
    ex = isdf.Exchange(shape, cell, n_mu, 4, 4, orb_dtype=torch.complex64, mode="mixed")
    d = torch.from_numpy(buf).to(DEV)
    out = torch.zeros((24 ** 3, ld), dtype=torch.complex64, device=DEV)
    ex.potential(d[:, :n_mu], out=out[:, :n_mu])
    ex.check()
    got = out.cpu().numpy()
    assert _maxrel(got[:, :n_mu], ref) < 1e-5
    assert not np.any(got[:, n_mu:])                          # padding columns untouched
    assert np.array_equal(d.cpu().numpy(), buf)               # out of place: the input is only read


def test_potential_mixed_fp32(isdf):
    shape, cell, n_mu = (24, 24, 24), (10.0, 10.0, 10.0), 96
    theta = _crandn(np.random.default_rng(3), 24 ** 3, n_mu).astype(np.complex64)
    ref = O.poisson(theta, shape, cell, "coulomb")
    ex = isdf.Exchange(shape, cell, n_mu, 4, 4, orb_dtype=torch.complex64, mode="mixed")
    got = ex.potential(torch.from_numpy(theta).to(DEV)).cpu().numpy()
    assert _maxrel(got, ref) < 1e-5


def test_potential_medium_grid_sampled_columns(isdf):
    # the benchmark's launch shape (48^3 grid, 1024 columns); the oracle checks 16 sampled columns
    w = W.WORKLOADS["medium"]
    shape, cell = (w.n,) * 3, (w.L,) * 3
    rng = np.random.default_rng(4)
    theta = _crandn(rng, w.n_r, w.n_mu)
    ex = isdf.Exchange(shape, cell, w.n_mu, w.n_orb, w.n_orb)
    got = ex.potential(torch.from_numpy(theta).to(DEV))
    cols = np.sort(rng.choice(w.n_mu, 16, replace=False))
    ref = O.poisson(theta[:, cols], shape, cell, "coulomb")
    assert _maxrel(got[:, torch.from_numpy(cols).to(DEV)].cpu().numpy(), ref) < 1e-12


def _apply_case(isdf, w, mode, max_rows, row_begin, row_count, seed):
    phi, psi = W.make_pair(w)
    phi, psi = W.storage(phi, w), W.storage(psi, w)
    wt = O.weights(phi.numpy(), psi.numpy())
    idx = W.init_indices(wt, w.n_mu, 100 + seed)
    rng = np.random.default_rng(seed)
    V = _crandn(rng, w.n_r, w.n_mu)
    if mode == "mixed":
        V = V.astype(np.complex64)
    ex = isdf.Exchange((w.n,) * 3, (w.L,) * 3, w.n_mu, w.n_orb, w.n_orb, orb_dtype=phi.dtype, mode=mode,
                       max_rows=max_rows)
    got = ex.apply(phi.to(DEV), psi.to(DEV), torch.from_numpy(idx), torch.from_numpy(V).to(DEV),
                   row_begin, row_count).cpu().numpy()
    ex.check()
    return got, phi.numpy(), psi.numpy(), idx, V


def test_apply_fp64_tiny_blocks(isdf):
    w = W.WORKLOADS["tiny"]
    got, phi, psi, idx, V = _apply_case(isdf, w, "fp64", 1000, 0, w.n_r, 5)   # 14 blocks, ragged tail
    ref = O.exchange_apply(phi, psi, idx, V)
    assert np.linalg.norm(got - ref) < 1e-11 * np.linalg.norm(ref)


def test_apply_fp64_row_range(isdf):
    w = W.WORKLOADS["tiny"]
    got, phi, psi, idx, V = _apply_case(isdf, w, "fp64", 65536, 333, 5000, 6)
    ref = O.exchange_apply(phi, psi, idx, V, rows=np.arange(333, 5333))
    assert np.linalg.norm(got - ref) < 1e-11 * np.linalg.norm(ref)


def test_apply_mixed_split_products_c64(isdf):
    # split-FP16 x3 tensor-core products (N % 32 == 0, N_mu % 64 == 0): ~2^-22 per product
    w = W.small_workload(n=24, L=10.0, n_orb=32, n_mu=256, iters=4, ecut=10.0, seed=7, dtype="c64")
    got, phi, psi, idx, V = _apply_case(isdf, w, "mixed", 4096, 0, w.n_r, 7)   # 4 blocks, ragged tail
    ref = O.exchange_apply(phi, psi, idx, V)
    assert np.linalg.norm(got - ref) < 1e-5 * np.linalg.norm(ref)


def test_apply_mixed_split_products_row_range_c128_orbitals(isdf):
    w = W.WORKLOADS["tiny"]
    w = W.Workload(w.name, w.n, w.L, 32, 128, "c128", w.iters, w.ecut, w.kfrac, w.centres, 11)
    got, phi, psi, idx, V = _apply_case(isdf, w, "mixed", 65536, 1000, 7777, 11)
    ref = O.exchange_apply(phi, psi, idx, V, rows=np.arange(1000, 8777))
    assert np.linalg.norm(got - ref) < 1e-5 * np.linalg.norm(ref)


def test_apply_mixed_sliced_products_for_other_sizes(isdf):
    # N = 20 is outside the split kernels' shapes: exact slicing, FP64-grade products
    w = W.small_workload(n=16, L=8.0, n_orb=20, n_mu=100, iters=4, ecut=8.0, seed=12, dtype="c64")
    got, phi, psi, idx, V = _apply_case(isdf, w, "mixed", 1500, 0, w.n_r, 12)
    ref = O.exchange_apply(phi, psi, idx, V)
    assert np.linalg.norm(got - ref) < 1e-11 * np.linalg.norm(ref)


def test_apply_medium_sampled_rows(isdf):
    w = W.WORKLOADS["medium"]
    got, phi, psi, idx, V = _apply_case(isdf, w, "fp64", 65536, 0, w.n_r, 8)
    rows = W.subsample_rows(w.n_r, 2048, 9)
    ref = O.exchange_apply(phi, psi, idx, V, rows=rows)
    assert np.linalg.norm(got[rows] - ref) < 1e-11 * np.linalg.norm(ref)


def test_isdf_exchange_chain_tiny(isdf):
    # Theta for phi_i* psi_j (a plan on the pair (Psi, Phi)), its potentials and the application,
    # all on the GPU, against the same chain in the oracle
    w = W.WORKLOADS["tiny"]
    phi, psi = W.make_pair(w)
    wt = O.weights(phi.numpy(), psi.numpy())
    idx = O.kmeans(wt, (w.n,) * 3, (w.L,) * 3, w.n_mu, W.init_indices(wt, w.n_mu, 1000 + w.seed), w.iters)["idx"]
    theta_ref = O.fit_theta(psi.numpy(), phi.numpy(), idx)["theta"]
    ref = O.exchange_apply(phi.numpy(), psi.numpy(), idx,
                           O.poisson(theta_ref, (w.n,) * 3, (w.L,) * 3, "erfc", 0.106))
    P, Q = phi.to(DEV), psi.to(DEV)
    plan = isdf.Plan(Q, P, torch.from_numpy(idx), "fp64")
    theta = plan.fit_theta()
    ex = isdf.Exchange((w.n,) * 3, (w.L,) * 3, w.n_mu, w.n_orb, w.n_orb, kernel="erfc", omega=0.106)
    v = ex.potential(theta, out=theta)
    got = ex.apply(P, Q, torch.from_numpy(idx), v).cpu().numpy()
    plan.check()
    ex.check()
    assert np.linalg.norm(got - ref) < 1e-9 * np.linalg.norm(ref)


def test_apply_reports_bad_index(isdf):
    w = W.small_workload(n=8, L=6.0, n_orb=4, n_mu=16, iters=1, ecut=6.0, seed=3)
    phi, psi = W.make_pair(w)
    idx = np.arange(16, dtype=np.int64) * 7
    idx[5] = w.n_r + 3                          # checked by the gather kernel, row left zero
    ex = isdf.Exchange((w.n,) * 3, (w.L,) * 3, 16, 4, 4)
    V = torch.zeros((w.n_r, 16), dtype=torch.complex128, device=DEV)
    ex.apply(phi.to(DEV), psi.to(DEV), torch.from_numpy(idx), V)
    with pytest.raises(isdf.ISDFError):
        ex.check()


def test_binding_rejects_mismatched_shapes(isdf):
    w = W.small_workload(n=8, L=6.0, n_orb=4, n_mu=16, iters=1, ecut=6.0, seed=3)
    phi, psi = (x.to(DEV) for x in W.make_pair(w))
    ex = isdf.Exchange((w.n,) * 3, (w.L,) * 3, 16, 4, 4)
    V = torch.zeros((w.n_r, 16), dtype=torch.complex128, device=DEV)
    idx = torch.arange(16, dtype=torch.int64) * 7
    wide = torch.zeros((w.n_r, 8), dtype=torch.complex128, device=DEV)
    with pytest.raises(ValueError):
        ex.apply(wide[:, :6], psi, idx, V)                  # n_phi 6 != 4
    with pytest.raises(ValueError):
        ex.apply(phi, psi, idx, V[:, :8])                   # fewer than n_mu potentials
    with pytest.raises(ValueError):
        ex.potential(V, out=torch.zeros((w.n_r, 15), dtype=torch.complex128, device=DEV))
    out = ex.apply(phi, psi, idx, V)                        # the valid call still works
    assert out.shape == (w.n_r, 4) and not torch.any(out)


@pytest.mark.parametrize("shape,n_mu", [((1, 12, 10), 1), ((9, 1, 15), 33)])
def test_potential_length_one_axis_and_single_column(isdf, shape, n_mu):
    cell = (3.0, 4.5, 5.0)
    theta = _crandn(np.random.default_rng(41), int(np.prod(shape)), n_mu)
    ref = O.poisson(theta, shape, cell, "erfc", 0.5)
    ex = isdf.Exchange(shape, cell, n_mu, 2, 2, kernel="erfc", omega=0.5)
    got = ex.potential(torch.from_numpy(theta).to(DEV)).cpu().numpy()
    assert _maxrel(got, ref) < 1e-12
