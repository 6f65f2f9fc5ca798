"""GPU tests of the batched decompositions (several orbital pairs on one grid;
isdf_weights with ISDF_W_ACCUMULATE, isdf_batch_*): the shared weight is
bit-exact against the oracle's left-to-right sum, every pair's Theta from the
concurrent batch is bit-identical to a plan run alone, and matches the oracle
(FP64 1e-10, mixed 1e-5); the batch follows new points and replays from a CUDA
graph."""
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


@pytest.fixture(scope="module")
def kp():
    w = W.small_workload(n=24, L=10.0, n_orb=32, n_mu=128, iters=20, ecut=10.0, seed=21)
    pairs = W.kpoint_pairs(w, 3)
    return w, pairs


def _shared_weight_gpu(isdf, pairs):
    wbuf = None
    for b, (p, q) in enumerate(pairs):
        if b == 0:
            wbuf = isdf.weights(p.to(DEV), q.to(DEV))
        else:
            isdf.weights(p.to(DEV), q.to(DEV), out=wbuf, accumulate=True)
    return wbuf


def test_shared_weight_bit_exact(isdf, kp):
    w, pairs = kp
    ref = O.shared_weights([(p.numpy(), q.numpy()) for p, q in pairs])
    assert np.array_equal(_shared_weight_gpu(isdf, pairs).cpu().numpy(), ref)


def test_shared_weight_psm_alpha_c64(isdf, kp):
    w, pairs = kp
    p64 = [(p.to(torch.complex64), q.to(torch.complex64)) for p, q in pairs]
    for kind, alpha in (("psm", 2.0), ("ssm", 3.0)):
        ref = O.shared_weights([(p.numpy(), q.numpy()) for p, q in p64], kind, alpha)
        g = isdf.weights(p64[0][0].to(DEV), p64[0][1].to(DEV), kind, alpha)
        for p, q in p64[1:]:
            isdf.weights(p.to(DEV), q.to(DEV), kind, alpha, out=g, accumulate=True)
        assert np.array_equal(g.cpu().numpy(), ref)


def _idx(w, pairs, seed):
    wt = O.shared_weights([(p.numpy(), q.numpy()) for p, q in pairs])
    return O.kmeans(wt, (w.n,) * 3, (w.L,) * 3, w.n_mu, W.init_indices(wt, w.n_mu, seed), w.iters)["idx"]


@pytest.mark.parametrize("mode,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_batch_equals_single_plans_and_oracle(isdf, kp, mode, tol):
    w, pairs = kp
    idx = torch.from_numpy(_idx(w, pairs, 7))
    dev_pairs = [(p.to(DEV), q.to(DEV)) for p, q in pairs]
    batch = isdf.Batch(dev_pairs, idx, mode=mode, max_rows=5000)
    got = batch.fit_theta()
    batch.check()
    for b, (p, q) in enumerate(dev_pairs):
        single = isdf.Plan(p, q, idx, mode, max_rows=5000)
        alone = single.fit_theta()
        single.check()
        assert torch.equal(got[b], alone)
    ref = O.fit_theta(pairs[1][0].numpy(), pairs[1][1].numpy(), idx.numpy())["theta"]
    g = got[1].cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(g - ref) < tol * np.linalg.norm(ref)


def test_batch_update_and_graph_replay(isdf, kp):
    w, pairs = kp
    idx0 = torch.from_numpy(_idx(w, pairs, 8)).to(DEV)
    idx1 = torch.from_numpy(_idx(w, pairs, 9)).to(DEV)
    dev_pairs = [(p.to(DEV), q.to(DEV)) for p, q in pairs]
    batch = isdf.Batch(dev_pairs, idx0, mode="mixed", max_rows=w.n_r)
    out = [torch.empty((w.n_r, w.n_mu), dtype=torch.complex64, device=DEV) for _ in pairs]
    idx_dev = idx0.clone()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):                     # warm-up outside the capture
        batch.update(idx_dev)
        batch.fit_theta(out=out)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batch.update(idx_dev)
        batch.fit_theta(out=out)
    idx_dev.copy_(idx1)                                # new points, same graph
    graph.replay()
    torch.cuda.synchronize()
    batch.check()
    for b, (p, q) in enumerate(dev_pairs):
        single = isdf.Plan(p, q, idx1, "mixed", max_rows=w.n_r)
        assert torch.equal(out[b], single.fit_theta())


def test_batch_of_one_is_a_plan(isdf, kp):
    w, pairs = kp
    idx = torch.from_numpy(_idx(w, pairs[:1], 10))
    p, q = pairs[0][0].to(DEV), pairs[0][1].to(DEV)
    batch = isdf.Batch([(p, q)], idx, mode="fp64")
    got = batch.fit_theta()[0]
    batch.check()
    assert torch.equal(got, isdf.Plan(p, q, idx, "fp64").fit_theta())
