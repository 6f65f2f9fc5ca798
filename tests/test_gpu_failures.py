"""Failure paths of the device-side checks, made on the host so that no GPU
faults, traps or hangs:

* a bounded wait that runs out: the plan's test hook makes the MMA issuer of
  the tensor-core kernels wait on a barrier that nothing signals; the launch
  must report ISDF_ERR_TIMEOUT through isdf_plan_status, leave the context
  usable, and the same plan (after an update) and a fresh plan must then fit
  Theta exactly as before (split-FP16 products and exact-slicing FP64
  products alike);
* a NaN or infinity written into one row of Phi that is not an
  interpolation point: the fit must report ISDF_ERR_NONFINITE in both modes
  instead of returning a silently wrong Theta;
* a K-means run whose duplicated start point leaves a cluster without
  members, and one with an init index outside the grid: isdf_kmeans_status
  must return ISDF_ERR_EMPTY_CLUSTER / ISDF_ERR_INVALID_ARG as a status
  code, not only in the stats array."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2208_07731_gb300 import workload as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
TIMEOUT, NONFINITE, EMPTY, INVALID = 6, 5, 4, 1


@pytest.fixture(scope="module")
def isdf():
    from paper_2208_07731_gb300 import build
    build.build()
    import paper_2208_07731_gb300 as m
    return m


@pytest.fixture(scope="module")
def case(isdf):
    # 16^3 grid, 32 complex128 orbitals, 256 points: the split kernels take it (N % 32, N_mu % 64) and
    # the FP64 mode's products run on the tensor cores by exact slicing
    w = W.small_workload(n=16, L=8.0, n_orb=32, n_mu=256, iters=10, ecut=12.0, seed=23)
    phi, psi = W.make_pair(w, device=DEV)
    wt = isdf.weights(phi, psi)
    init = torch.from_numpy(W.init_indices(wt.cpu().numpy(), w.n_mu, 77))
    idx = isdf.kmeans(wt, (w.n,) * 3, (w.L,) * 3, w.n_mu, init, w.iters)["idx"]
    return w, phi.contiguous(), psi.contiguous(), idx


@pytest.mark.parametrize("mode", ["mixed", "fp64"])
def test_wait_that_runs_out_reports_timeout_and_context_stays_usable(isdf, case, mode):
    w, phi, psi, idx = case
    plan = isdf.Plan(phi, psi, idx, mode=mode, max_rows=1024)
    ref = plan.fit_theta()
    plan.check()
    plan.set_wait_budget(-20000)      # the MMA issuer waits 20,000 cycles on a barrier nothing signals
    bad = plan.fit_theta()
    rc, detail = plan.status()
    assert rc == TIMEOUT, (rc, detail)
    del bad
    # the same plan after an update (which clears the status), and a fresh plan, fit exactly as before
    plan.set_wait_budget(0)
    plan.update(idx)
    again = plan.fit_theta()
    plan.check()
    assert torch.equal(again, ref)
    fresh = isdf.Plan(phi, psi, idx, mode=mode, max_rows=1024)
    assert torch.equal(fresh.fit_theta(), ref)
    fresh.check()
    # and the result is still the oracle's Theta (the FP64 gate / the split-precision gate)
    rows = W.subsample_rows(w.n_r, 512, 5)
    p_h, q_h = phi.cpu().numpy(), psi.cpu().numpy()
    pm, qm = O.gather(p_h, q_h, idx.cpu().numpy())
    T = O.theta_rows(p_h, q_h, pm, qm, O.cholesky(O.form_M(pm, qm)), rows)
    got = again[torch.from_numpy(rows).to(DEV)].cpu().numpy().astype(np.complex128)
    err = np.linalg.norm(got - T) / np.linalg.norm(T)
    assert err < (1e-10 if mode == "fp64" else 1e-5), err
    plan.close()
    fresh.close()


@pytest.mark.parametrize("mode", ["mixed", "fp64"])
@pytest.mark.parametrize("value", [float("nan"), float("inf")])
def test_non_finite_orbital_row_is_reported(isdf, case, mode, value):
    w, phi, psi, idx = case
    bad_row = int(np.setdiff1d(np.arange(w.n_r), idx.cpu().numpy())[w.n_r // 3])
    P = phi.clone()
    P[bad_row, 5] = complex(value, 0.0)
    plan = isdf.Plan(P, psi, idx, mode=mode, max_rows=1024)
    th = plan.fit_theta()
    rc, _ = plan.status()
    assert rc == NONFINITE, rc
    del th
    # the clean orbitals in the same process: no error left behind
    clean = isdf.Plan(phi, psi, idx, mode=mode, max_rows=1024)
    clean.fit_theta()
    clean.check()
    plan.close()
    clean.close()


def test_kmeans_status_codes(isdf):
    shape, cell = (8, 8, 8), (4.0, 4.0, 4.0)
    rng = np.random.default_rng(2)
    wt = torch.from_numpy(rng.random(512)).to(DEV)
    # a duplicated start point, no update: the copy's cluster has no member
    km = isdf.kmeans(wt, shape, cell, 5, torch.tensor([5, 5, 100, 300, 411]), 0)
    assert isdf.kmeans_status(km) == EMPTY
    assert km["idx"][1].item() == -1 and km["stats"][2].item() == 1
    with pytest.raises(isdf.ISDFError):
        isdf.kmeans_check(km)
    # an init index outside the grid
    km = isdf.kmeans(wt, shape, cell, 4, torch.tensor([0, 10, 20, 512]), 2)
    assert isdf.kmeans_status(km) == INVALID and km["stats"][2].item() == -2
    assert bool((km["idx"] == -1).all())
    # a negative weight
    w2 = wt.clone()
    w2[7] = -1.0
    km = isdf.kmeans(w2, shape, cell, 4, torch.tensor([0, 10, 20, 30]), 2)
    assert isdf.kmeans_status(km) == NONFINITE and km["stats"][2].item() == -1
    # a normal run
    km = isdf.kmeans(wt, shape, cell, 4, torch.tensor([0, 10, 20, 30]), 3)
    assert isdf.kmeans_status(km) == 0
    isdf.kmeans_check(km)
