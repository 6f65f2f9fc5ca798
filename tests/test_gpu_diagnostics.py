"""GPU parity of the Appendix-A decomposition diagnostics (isdf_fit_error,
isdf_cluster_residual) against the oracle on the same seeded inputs.

Tolerances: both sides sum O(N_r) FP64 terms in different orders, so z2 and R
agree to ~1e-13 relative; the fit residual ||Z||^2 - Re tr(Theta^H Y) inherits
Theta's 1e-10 gate, scaled by ||Z||^2."""
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


def _problem(name):
    w = W.WORKLOADS[name]
    phi, psi = W.make_pair(w)
    phi, psi = W.storage(phi, w), W.storage(psi, w)
    wt = O.weights(phi.numpy(), psi.numpy())
    return w, phi, psi, wt


@pytest.fixture(scope="module")
def tiny():
    w, phi, psi, wt = _problem("tiny")
    km = O.kmeans(wt, (w.n,) * 3, (w.L,) * 3, w.n_mu, W.init_indices(wt, w.n_mu, 1000 + w.seed), w.iters)
    return w, phi, psi, km


@pytest.fixture(scope="module")
def medium():
    w, phi, psi, wt = _problem("medium")
    km = O.kmeans(wt, (w.n,) * 3, (w.L,) * 3, w.n_mu, W.init_indices(wt, w.n_mu, 1000 + w.seed), w.iters)
    return w, phi, psi, km


def _fit_error_compare(isdf, phi, psi, idx, r0, r1, max_rows):
    ref = O.isdf_error(phi.numpy(), psi.numpy(), idx, row_range=(r0, r1))
    plan = isdf.Plan(phi.to(DEV), psi.to(DEV), torch.from_numpy(idx), "fp64", max_rows=max_rows)
    got = plan.fit_error(r0, r1 - r0)
    plan.check()
    z2 = ref["z2"]
    assert abs(got["z2"] - z2) <= 1e-13 * z2
    assert abs(got["trace"] - ref["trace"]) <= 1e-10 * z2
    assert abs(got["residual2"] - ref["residual2"]) <= 1e-10 * z2
    return ref, got


def test_fit_error_tiny_blocks(isdf, tiny):
    w, phi, psi, km = tiny
    # several internal blocks with a ragged tail
    _fit_error_compare(isdf, phi, psi, km["idx"], 0, w.n_r, max_rows=3000)


def test_fit_error_tiny_row_range(isdf, tiny):
    w, phi, psi, km = tiny
    ref, got = _fit_error_compare(isdf, phi, psi, km["idx"], 517, 517 + 4099, max_rows=65536)
    assert 0 < got["error"] < 1


def test_fit_error_medium_sampled_range(isdf, medium):
    w, phi, psi, km = medium
    r0 = 40000
    _fit_error_compare(isdf, phi, psi, km["idx"], r0, r0 + 8192 + 77, max_rows=4096)


def test_fit_error_rejects_mixed_plan(isdf):
    w = W.small_workload(n=8, L=6.0, n_orb=32, n_mu=64, iters=4, ecut=8.0, seed=9)
    phi, psi = W.make_pair(w)
    a, b = phi.to(torch.complex64).to(DEV), psi.to(torch.complex64).to(DEV)
    idx = W.init_indices(O.weights(phi.numpy(), psi.numpy()), w.n_mu, 5)
    plan = isdf.Plan(a, b, torch.from_numpy(idx), "mixed")
    with pytest.raises(isdf.ISDFError):
        plan.fit_error()


def test_cluster_residual_tiny_kmeans_labels(isdf, tiny):
    w, phi, psi, km = tiny
    ref = O.cluster_residual(phi.numpy(), psi.numpy(), km["labels"], km["idx"])
    got = isdf.cluster_residual(phi.to(DEV), psi.to(DEV), torch.from_numpy(km["labels"]),
                                torch.from_numpy(km["idx"]))
    assert abs(got["z2"] - ref["z2"]) <= 1e-13 * ref["z2"]
    assert abs(got["R"] - ref["R"]) <= 1e-12 * ref["z2"]


def test_cluster_residual_medium_full_grid(isdf, medium):
    w, phi, psi, km = medium
    ref = O.cluster_residual(phi.numpy(), psi.numpy(), km["labels"], km["idx"])
    got = isdf.cluster_residual(phi.to(DEV), psi.to(DEV), torch.from_numpy(km["labels"]),
                                torch.from_numpy(km["idx"]))
    assert abs(got["z2"] - ref["z2"]) <= 1e-13 * ref["z2"]
    assert abs(got["R"] - ref["R"]) <= 1e-12 * ref["z2"]


def test_cluster_residual_c64_unequal_widths_random_labels(isdf):
    rng = np.random.default_rng(12)
    n_r, n_phi, n_psi, n_mu = 5000 + 13, 37, 21, 97
    a = (rng.standard_normal((n_r, n_phi + 3)) + 1j * rng.standard_normal((n_r, n_phi + 3))).astype(np.complex64)
    b = (rng.standard_normal((n_r, n_psi)) + 1j * rng.standard_normal((n_r, n_psi))).astype(np.complex64)
    labels = rng.integers(0, n_mu, n_r).astype(np.int32)
    idx = rng.choice(n_r, n_mu, replace=False).astype(np.int64)
    ref = O.cluster_residual(a[:, :n_phi], b, labels, idx)
    A = torch.from_numpy(a).to(DEV)[:, :n_phi]     # leading dimension n_phi + 3
    got = isdf.cluster_residual(A, torch.from_numpy(b).to(DEV), torch.from_numpy(labels), torch.from_numpy(idx))
    assert abs(got["z2"] - ref["z2"]) <= 1e-12 * ref["z2"]
    assert abs(got["R"] - ref["R"]) <= 1e-12 * ref["z2"]


def test_cluster_residual_out_of_range_label_reported(isdf, tiny):
    w, phi, psi, km = tiny
    lab = km["labels"].copy()
    lab[100] = w.n_mu                         # the kernel checks and skips this row
    with pytest.raises(ValueError):
        isdf.cluster_residual(phi.to(DEV), psi.to(DEV), torch.from_numpy(lab), torch.from_numpy(km["idx"]))


def test_cluster_residual_every_point_its_own_cluster_is_zero(isdf):
    # each row projected on itself (Eq. proj with r_mu = r): R = 0 up to rounding
    w = W.small_workload(n=8, L=6.0, n_orb=6, n_mu=512, iters=1, ecut=6.0, seed=13)
    phi, psi = (x.to(DEV) for x in W.make_pair(w))
    lab = torch.arange(w.n_r, dtype=torch.int32)
    got = isdf.cluster_residual(phi, psi, lab, torch.arange(w.n_r, dtype=torch.int64))
    assert abs(got["R"]) <= 1e-13 * got["z2"]
