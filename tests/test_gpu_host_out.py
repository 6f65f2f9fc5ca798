"""Theta fitted into page-locked host memory (isdf_fit_theta_host): bit-identical to the device fit in both modes
for a row window that spans more blocks than the plan has staging blocks (ragged last block), a host leading
dimension larger than n_mu (the padding stays untouched), and a second call with another window; pageable and
device outputs are refused before any work is enqueued."""
import ctypes

import pytest
import torch

from paper_2208_07731_gb300 import workload as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
INVALID = 1


@pytest.fixture(scope="module")
def isdf():
    from paper_2208_07731_gb300 import build
    build.build()
    import paper_2208_07731_gb300 as m
    return m


@pytest.fixture(scope="module")
def case(isdf):
    w = W.small_workload(n=16, L=8.0, n_orb=32, n_mu=256, iters=10, ecut=12.0, seed=29)
    phi, psi = W.make_pair(w, device=DEV)
    wt = isdf.weights(phi, psi)
    init = torch.from_numpy(W.init_indices(wt.cpu().numpy(), w.n_mu, 78))
    idx = isdf.kmeans(wt, (w.n,) * 3, (w.L,) * 3, w.n_mu, init, w.iters)["idx"]
    return w, phi.contiguous(), psi.contiguous(), idx


@pytest.mark.parametrize("mode", ["mixed", "fp64"])
def test_host_fit_equals_device_fit(isdf, case, mode):
    w, phi, psi, idx = case
    plan = isdf.Plan(phi, psi, idx, mode=mode, max_rows=512)
    r0, n = 37, w.n_r - 42                    # 4,054 rows: 7 blocks of 512 and one of 470
    ref = plan.fit_theta(r0, n).cpu()
    host = torch.zeros((n, w.n_mu + 3), dtype=ref.dtype).pin_memory()
    plan.fit_theta_host(host[:, :w.n_mu], r0, n)
    torch.cuda.current_stream().synchronize()
    assert torch.equal(host[:, :w.n_mu], ref)
    assert bool((host[:, w.n_mu:] == 0).all())
    host2 = torch.empty((1000, w.n_mu), dtype=ref.dtype).pin_memory()
    plan.fit_theta_host(host2, 1000, 1000)
    torch.cuda.current_stream().synchronize()
    assert torch.equal(host2, plan.fit_theta(1000, 1000).cpu())
    plan.check()
    plan.close()


def test_host_fit_refuses_pageable_and_device_memory(isdf, case):
    w, phi, psi, idx = case
    plan = isdf.Plan(phi, psi, idx, mode="mixed", max_rows=512)
    pageable = torch.empty((64, w.n_mu), dtype=torch.complex64)
    with pytest.raises(ValueError):
        plan.fit_theta_host(pageable, 0, 64)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    lib = isdf.lib()
    assert lib.isdf_fit_theta_host(plan._h, 0, 64, ctypes.c_void_p(pageable.data_ptr()), w.n_mu, st) == INVALID
    dev_out = torch.empty((64, w.n_mu), dtype=torch.complex64, device=DEV)
    assert lib.isdf_fit_theta_host(plan._h, 0, 64, ctypes.c_void_p(dev_out.data_ptr()), w.n_mu, st) == INVALID
    plan.check()
    plan.close()


def test_mixed_fit_reads_only_its_operand_copies(isdf, case):
    # in the split-precision mode the fit reads the FP16 copies made by the plan update, not the orbitals:
    # overwriting them after the update (as a pipeline loading the next decomposition does) changes nothing
    w, phi, psi, idx = case
    P, Q = phi.clone(), psi.clone()
    plan = isdf.Plan(P, Q, idx, mode="mixed", max_rows=512)
    ref = plan.fit_theta()
    P.zero_()
    Q.fill_(float("nan"))
    assert torch.equal(plan.fit_theta(), ref)
    host = torch.empty((w.n_r, w.n_mu), dtype=ref.dtype).pin_memory()
    plan.fit_theta_host(host)
    torch.cuda.current_stream().synchronize()
    assert torch.equal(host, ref.cpu())
    plan.check()
    plan.close()
