"""Full-size workloads on the GPU, through the C ABI, against the CPU oracle.

waterbox (96^3 grid, 256 complex64 orbitals, 2048 points, T = 100): the whole
K-means bit-exact against the oracle, mixed Theta on sampled rows <= 1e-5.
adjoint (72^3, 192 orbitals, 1536 points fixed from a prior K-means): the
FP64 and tensor-core adjoints of the exchange-like surrogate against the
oracle gradient, and the FP64 adjoint against central finite differences on
32 seeded directions scaled to the orbital norms (h = 1e-6 within 1e-6, the
difference of the two losses formed without cancellation).
silica (128^3, 1024 orbitals, 4096 points): K-means checked step by step
against the oracle (lock-step: one exact update from the GPU's labels, the
brute-force assignment of a 131,072-point sample, the final snap) and through
properties that hold at any size (sampled labels are the nearest centroids
under the FP64 formula, every cluster is non-empty, snapped points are
distinct members nearest to their centroids), and
Theta fitted in blocks of 131,072 rows, never fully resident, <= 1e-5 against
the oracle on a 16,384-row sample."""
import math

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


def _gpu_pair(w):
    phi, psi = W.make_pair(w, device=DEV)
    return W.storage(phi, w).contiguous(), W.storage(psi, w).contiguous()


def test_waterbox_kmeans_bit_exact_and_mixed_theta(isdf):
    w = W.WORKLOADS["waterbox"]
    phi, psi = _gpu_pair(w)
    wt = isdf.weights(phi, psi)
    p_h, q_h = phi.cpu().numpy(), psi.cpu().numpy()
    wt_ref = O.weights(p_h, q_h)
    assert np.array_equal(wt.cpu().numpy(), wt_ref)
    init = W.init_indices(wt_ref, w.n_mu, 1000 + w.seed)
    shape, cell = (w.n,) * 3, (w.L,) * 3
    km = isdf.kmeans(wt, shape, cell, w.n_mu, torch.from_numpy(init), w.iters)
    ref = O.kmeans(wt_ref, shape, cell, w.n_mu, init, w.iters)
    assert np.array_equal(km["idx"].cpu().numpy(), ref["idx"])
    assert np.array_equal(km["labels"].cpu().numpy(), ref["labels"])
    assert np.array_equal(km["centroids"].cpu().numpy(), ref["centroids"])
    st = km["stats"].cpu().numpy()
    assert st[1] == ref["near_ties"] and st[2] == ref["empty"] == 0
    plan = isdf.Plan(phi, psi, km["idx"], mode="mixed", max_rows=131072)
    th = plan.fit_theta()
    plan.check()
    rows = W.subsample_rows(w.n_r, 8192, 2000 + w.seed)
    pm, qm = O.gather(p_h, q_h, ref["idx"])
    M = O.form_M(pm, qm)
    T = O.theta_rows(p_h, q_h, pm, qm, O.cholesky(M), rows)
    got = th[torch.from_numpy(rows).to(DEV)].cpu().numpy().astype(np.complex128)
    err = np.linalg.norm(got - T) / np.linalg.norm(T)
    dT = got - T
    zerr = np.sqrt(np.real(np.sum((dT @ M) * dT.conj())) / np.real(np.sum((T @ M) * T.conj())))
    assert err < 1e-5 and zerr < 1e-5, (err, zerr)


def _adjoint_setup(isdf):
    w = W.WORKLOADS["adjoint"]
    phi, psi = _gpu_pair(w)
    wt = isdf.weights(phi, psi)
    init = torch.from_numpy(W.init_indices(wt.cpu().numpy(), w.n_mu, 1000 + w.seed))
    idx = isdf.kmeans(wt, (w.n,) * 3, (w.L,) * 3, w.n_mu, init, w.iters)["idx"]
    K = W.loss_matrix(w.n_mu, 3000 + w.seed)
    return w, phi, psi, idx, K


def test_adjoint_config_against_oracle_gradient(isdf):
    w, phi, psi, idx, K = _adjoint_setup(isdf)
    plan = isdf.Plan(phi, psi, idx, mode="fp64", max_rows=65536)
    loss, gphi, gpsi = isdf.surrogate_loss_and_grad(plan, torch.from_numpy(K).to(DEV), w.dV, block=65536)
    plan.check()
    p_h, q_h = phi.cpu().numpy(), psi.cpu().numpy()
    ref = O.theta_backward(p_h, q_h, idx.cpu().numpy(), lambda rows, T: O.surrogate_grad_theta(T, K, w.dV),
                           block=32768)
    for got, exp in ((gphi, ref["grad_phi"]), (gpsi, ref["grad_psi"])):
        g = got.cpu().numpy()
        assert np.linalg.norm(g - exp) < 1e-9 * np.linalg.norm(exp)
    # the tensor-core adjoint against the same FP64 oracle gradient
    mplan = isdf.Plan(phi, psi, idx, mode="mixed", max_rows=65536)
    _, mphi, mpsi = isdf.surrogate_loss_and_grad(mplan, torch.from_numpy(K).to(DEV), w.dV, block=65536)
    mplan.check()
    for got, exp in ((mphi, ref["grad_phi"]), (mpsi, ref["grad_psi"])):
        assert np.linalg.norm(got.cpu().numpy() - exp) < 1e-4 * np.linalg.norm(exp)


def test_adjoint_config_finite_differences(isdf):
    w, phi, psi, idx, _ = _adjoint_setup(isdf)
    # a Hermitian positive-definite K = c I + U U^H with U of rank 32 (passed to the adjoint as a
    # dense matrix): per grid row the loss is q(t) = c |t|^2 + |U^H t|^2, and the central difference
    # q(t+) - q(t-) = c Re<t+ - t-, t+ + t-> + Re<U^H (t+ - t-), U^H (t+ + t-)> is formed block by block
    # from the two FP64 fits, without subtracting two large sums (whose rounding would be ~3e-6 of the
    # derivative at h = 1e-6 on 5.7e8 terms)
    rng = np.random.default_rng(3000 + w.seed)
    Qk, _ = np.linalg.qr(rng.standard_normal((w.n_mu, 32)) + 1j * rng.standard_normal((w.n_mu, 32)))
    U = Qk * np.sqrt(rng.uniform(1.0, 9.0, size=32))[None, :]
    c = 1.0
    K = c * np.eye(w.n_mu) + U @ U.conj().T
    K = 0.5 * (K + K.conj().T)
    Kd = torch.from_numpy(K).to(DEV)
    Ucd = torch.from_numpy(U.conj()).to(DEV)
    P = phi.to(torch.complex128)
    Q = psi.to(torch.complex128)
    B = 131072
    plan = isdf.Plan(P, Q, idx, mode="fp64", max_rows=B)
    loss, gphi, gpsi = isdf.surrogate_loss_and_grad(plan, Kd, w.dV, block=B)
    plan.check()
    plan.close()
    bufs = [torch.empty_like(P), torch.empty_like(Q), torch.empty_like(P), torch.empty_like(Q)]
    plus = isdf.Plan(bufs[0].copy_(P), bufs[1].copy_(Q), idx, mode="fp64", max_rows=B)
    minus = isdf.Plan(bufs[2].copy_(P), bufs[3].copy_(Q), idx, mode="fp64", max_rows=B)
    tp = torch.empty((B, w.n_mu), dtype=torch.complex128, device=DEV)
    tm = torch.empty_like(tp)

    # the loss at the plus plan's orbitals, from one fit
    def loss_plus():
        plus.update(idx)
        tot = 0.0
        for r0 in range(0, w.n_r, B):
            n = min(B, w.n_r - r0)
            plus.fit_theta(r0, n, out=tp[:n])
            tot += (c * torch.linalg.vector_norm(tp[:n]) ** 2 + torch.linalg.vector_norm(tp[:n] @ Ucd) ** 2).item()
        return w.dV * tot

    def loss_difference(Dp, Dq, h):
        bufs[0].copy_(P).add_(Dp, alpha=h)
        bufs[1].copy_(Q).add_(Dq, alpha=h)
        bufs[2].copy_(P).add_(Dp, alpha=-h)
        bufs[3].copy_(Q).add_(Dq, alpha=-h)
        plus.update(idx)
        minus.update(idx)
        tot = 0.0
        for r0 in range(0, w.n_r, B):
            n = min(B, w.n_r - r0)
            plus.fit_theta(r0, n, out=tp[:n])
            minus.fit_theta(r0, n, out=tm[:n])
            d, s = tp[:n] - tm[:n], tp[:n] + tm[:n]
            tot += (c * torch.real(torch.vdot(d.flatten(), s.flatten())) +
                    torch.real(torch.vdot((d @ Ucd).flatten(), (s @ Ucd).flatten()))).item()
        return w.dV * tot

    assert abs(loss_plus() - loss.item()) < 1e-10 * abs(loss.item())
    gen = torch.Generator(device=DEV).manual_seed(4242)
    h = 1e-6
    for d in range(32):
        Dp = torch.randn(P.shape, dtype=torch.complex128, device=DEV, generator=gen)
        Dq = torch.randn(Q.shape, dtype=torch.complex128, device=DEV, generator=gen)
        # scaled to the orbitals' norms, so that h is a relative step
        Dp *= torch.linalg.vector_norm(P) / torch.linalg.vector_norm(Dp)
        Dq *= torch.linalg.vector_norm(Q) / torch.linalg.vector_norm(Dq)
        an = torch.real(torch.vdot(gphi.flatten(), Dp.flatten()) + torch.vdot(gpsi.flatten(), Dq.flatten())).item()
        fd = loss_difference(Dp, Dq, h) / (2 * h)
        assert abs(fd - an) <= 1e-6 * abs(an), (d, fd, an)
    plus.check()
    minus.check()


def test_silica_kmeans_lock_step_against_oracle(isdf):
    """The 128^3 x 4096 K-means checked step by step against the oracle's single steps of
    Algorithm 1: for t in {0, 1, 50, T-1}, the GPU's centroids after t + 1 updates equal the
    oracle's update (exact 128-bit sums, Eq. r_k) applied to the GPU's labels and centroids after t
    updates, and those labels equal the oracle's brute-force assignment (Eq. opt) of a seeded
    131,072-point sample; the final snap equals the oracle's nearest members."""
    w = W.WORKLOADS["silica"]
    phi, psi = _gpu_pair(w)
    wt = isdf.weights(phi, psi)
    shape, cell = (w.n,) * 3, (w.L,) * 3
    wt_h = wt.cpu().numpy()
    # the weights on a row sample (the full grid is checked bit for bit on the waterbox workload)
    rs = torch.from_numpy(W.subsample_rows(w.n_r, 8192, 7)).to(DEV)
    assert np.array_equal(wt_h[rs.cpu().numpy()], O.weights(phi[rs].cpu().numpy(), psi[rs].cpu().numpy()))
    del phi, psi
    init = torch.from_numpy(W.init_indices(wt_h, w.n_mu, 1000 + w.seed))
    sample = W.subsample_rows(w.n_r, 131072, 2000 + w.seed)
    for t in (0, 1, 50, w.iters - 1):
        a = isdf.kmeans(wt, shape, cell, w.n_mu, init, t, objective=False)
        b = isdf.kmeans(wt, shape, cell, w.n_mu, init, t + 1, labels=False, objective=False)
        c_t = a["centroids"].cpu().numpy()
        lab_t = a["labels"].cpu().numpy()
        assert np.array_equal(b["centroids"].cpu().numpy(), O.kmeans_update(wt_h, shape, cell, lab_t, c_t)), t
        lab_s, _ = O.kmeans_assign(shape, cell, c_t, sample)
        assert np.array_equal(lab_t[sample], lab_s), t
    km = isdf.kmeans(wt, shape, cell, w.n_mu, init, w.iters, objective=False)
    idx_ref, empty = O.kmeans_snap(shape, cell, km["centroids"].cpu().numpy(), km["labels"].cpu().numpy())
    assert empty == 0 and np.array_equal(km["idx"].cpu().numpy(), idx_ref)
    assert isdf.kmeans_status(km) == 0


def test_silica_kmeans_properties_and_blocked_mixed_theta(isdf):
    w = W.WORKLOADS["silica"]
    phi, psi = _gpu_pair(w)
    wt = isdf.weights(phi, psi)
    shape, cell = (w.n,) * 3, (w.L,) * 3
    init = torch.from_numpy(W.init_indices(wt.cpu().numpy(), w.n_mu, 1000 + w.seed))
    km = isdf.kmeans(wt, shape, cell, w.n_mu, init, w.iters)
    st = km["stats"].cpu().numpy()
    assert st[2] == 0
    idx = km["idx"].cpu().numpy()
    lab = km["labels"].cpu().numpy()
    cen = km["centroids"].cpu().numpy()
    assert len(set(idx.tolist())) == w.n_mu
    x = O.grid_coords(shape, cell)
    # labels of sampled points are their nearest centroids under the FP64 formula (lowest index on ties)
    rs = W.subsample_rows(w.n_r, 4096, 99)
    d = ((x[rs][:, None, :] - cen[None, :, :]) ** 2).sum(-1)
    assert np.array_equal(lab[rs], np.argmin(d, axis=1))
    # snapped points belong to their clusters and are their nearest members (sampled clusters)
    assert np.array_equal(lab[idx], np.arange(w.n_mu))
    for m in range(0, w.n_mu, 257):
        mem = np.nonzero(lab == m)[0]
        dm = ((x[mem] - cen[m]) ** 2).sum(1)
        assert idx[m] == mem[np.argmin(dm)]
    # Theta in blocks of 131,072 rows, compared with the oracle on a 16,384-row sample
    plan = isdf.Plan(phi, psi, km["idx"], mode="mixed", max_rows=131072)
    rows = W.subsample_rows(w.n_r, 16384, 2000 + w.seed)
    p_h = phi.cpu().numpy()
    q_h = psi.cpu().numpy()
    pm, qm = O.gather(p_h, q_h, idx)
    M = O.form_M(pm, qm)
    T = O.theta_rows(p_h, q_h, pm, qm, O.cholesky(M), rows)
    blk = torch.empty((131072, w.n_mu), dtype=torch.complex64, device=DEV)
    got = np.empty_like(T)
    for b0 in range(0, w.n_r, 131072):
        plan.fit_theta(b0, 131072, out=blk)
        sel = (rows >= b0) & (rows < b0 + 131072)
        got[sel] = blk[torch.from_numpy(rows[sel] - b0).to(DEV)].cpu().numpy()
    plan.check()
    err = np.linalg.norm(got - T) / np.linalg.norm(T)
    dT = got - T
    zerr = np.sqrt(np.real(np.sum((dT @ M) * dT.conj())) / np.real(np.sum((T @ M) * T.conj())))
    assert err < 1e-5 and zerr < 1e-5, (err, zerr)


def test_silica_adjoint_mixed_vs_fp64_and_central_differences(isdf):
    """Config 4 (128^3, 1024 complex64 orbitals, 4096 points, blocks of 131,072 rows, Theta never
    stored): the tensor-core gradient of the exchange-like surrogate against the FP64 GPU gradient
    (itself pinned to the oracle gradient at 72^3), and the FP64 gradient against central differences
    at h = 1e-6 on four directions, each loss difference formed from the two fits' Theta difference
    (the per-row loss is a Hermitian quadratic form): three directions supported on a row range
    without interpolation points (only those Theta rows move; fitted through a plan on
    [Phi[idx]; Phi[range]]) and one on 64 interpolation points (M moves; two full FP64 fits)."""
    w = W.WORKLOADS["silica"]
    phi, psi = _gpu_pair(w)
    shape, cell = (w.n,) * 3, (w.L,) * 3
    wt = isdf.weights(phi, psi)
    init = torch.from_numpy(W.init_indices(wt.cpu().numpy(), w.n_mu, 1000 + w.seed))
    idx = isdf.kmeans(wt, shape, cell, w.n_mu, init, w.iters, labels=False, objective=False)["idx"]
    del wt
    rng = np.random.default_rng(3000 + w.seed)
    Qk, _ = np.linalg.qr(rng.standard_normal((w.n_mu, 32)) + 1j * rng.standard_normal((w.n_mu, 32)))
    U = Qk * np.sqrt(rng.uniform(1.0, 9.0, size=32))[None, :]
    c = 1.0
    K = c * np.eye(w.n_mu) + U @ U.conj().T
    Kd = torch.from_numpy(0.5 * (K + K.conj().T)).to(DEV)
    Ucd = torch.from_numpy(U.conj()).to(DEV)
    B = 131072

    def q_diff(tp, tm):
        # sum over rows of q(t+) - q(t-), q(t) = c |t|^2 + |U^H t|^2, without cancellation
        d, s = tp - tm, tp + tm
        return (c * torch.real(torch.vdot(d.flatten(), s.flatten())) +
                torch.real(torch.vdot((d @ Ucd).flatten(), (s @ Ucd).flatten()))).item()

    # the tensor-core gradient, kept in complex64 (its rounding is far below the 1e-4 comparison)
    mplan = isdf.Plan(phi, psi, idx, mode="mixed", max_rows=B)
    _, mphi, mpsi = isdf.surrogate_loss_and_grad(mplan, Kd, w.dV, block=B)
    mplan.check()
    mplan.close()
    mphi, mpsi = mphi.to(torch.complex64), mpsi.to(torch.complex64)
    torch.cuda.empty_cache()
    # the FP64 gradient on the same (complex64-valued) orbitals
    plan = isdf.Plan(phi, psi, idx, mode="fp64", max_rows=B)
    loss, gphi, gpsi = isdf.surrogate_loss_and_grad(plan, Kd, w.dV, block=B)
    plan.check()
    plan.close()
    num = den = 0.0
    for x, y in ((mphi, gphi), (mpsi, gpsi)):
        for r0 in range(0, w.n_r, B):
            yb = y[r0:r0 + B]
            num += (torch.linalg.vector_norm(x[r0:r0 + B].to(torch.complex128) - yb) ** 2).item()
            den += (torch.linalg.vector_norm(yb) ** 2).item()
    assert math.sqrt(num / den) < 1e-4, math.sqrt(num / den)
    del mphi, mpsi, x, y, yb   # the loop variables would keep two gradients alive
    torch.cuda.empty_cache()

    h = 1e-6
    gen = torch.Generator(device=DEV).manual_seed(777)
    idx_h = idx.cpu().numpy()
    is_point = np.zeros(w.n_r, bool)
    is_point[idx_h] = True
    # (1) three directions on row ranges of 8,192 rows (interpolation rows in the range left unperturbed)
    R = 8192
    for r0 in (123 * 512, w.n_r // 2 + 77, w.n_r - R):
        keep = torch.from_numpy(~is_point[r0:r0 + R]).to(DEV)[:, None]
        Dp = torch.randn((R, w.n_orb), dtype=torch.complex128, device=DEV, generator=gen) * keep
        Dq = torch.randn((R, w.n_orb), dtype=torch.complex128, device=DEV, generator=gen) * keep
        Pr, Qr = phi[r0:r0 + R].to(torch.complex128), psi[r0:r0 + R].to(torch.complex128)
        Dp *= torch.linalg.vector_norm(Pr) / torch.linalg.vector_norm(Dp)
        Dq *= torch.linalg.vector_norm(Qr) / torch.linalg.vector_norm(Dq)
        an = torch.real(torch.vdot(gphi[r0:r0 + R].flatten(), Dp.flatten()) +
                        torch.vdot(gpsi[r0:r0 + R].flatten(), Dq.flatten())).item()
        th = []
        for sgn in (1.0, -1.0):
            sp = torch.cat([phi[idx].to(torch.complex128), Pr + sgn * h * Dp]).contiguous()
            sq = torch.cat([psi[idx].to(torch.complex128), Qr + sgn * h * Dq]).contiguous()
            pl = isdf.Plan(sp, sq, torch.arange(w.n_mu, device=DEV), mode="fp64", max_rows=R)
            th.append(pl.fit_theta(w.n_mu, R))
            pl.check()
            pl.close()
        fd = w.dV * q_diff(th[0], th[1]) / (2 * h)
        assert abs(fd - an) <= 1e-6 * abs(an), (r0, fd, an)
        del th
    # (2) one direction on 64 interpolation points: M moves, so every Theta row moves
    S = torch.from_numpy(np.sort(rng.choice(idx_h, 64, replace=False))).to(DEV)
    Dp = torch.randn((64, w.n_orb), dtype=torch.complex128, device=DEV, generator=gen)
    Dq = torch.randn((64, w.n_orb), dtype=torch.complex128, device=DEV, generator=gen)
    an = torch.real(torch.vdot(gphi[S].flatten(), Dp.flatten()) + torch.vdot(gpsi[S].flatten(), Dq.flatten())).item()
    del gphi, gpsi
    torch.cuda.empty_cache()
    P = phi.to(torch.complex128)
    Q = psi.to(torch.complex128)
    del phi, psi
    torch.cuda.empty_cache()
    P0, Q0 = P[S].clone(), Q[S].clone()
    plans = []
    B = 32768      # smaller blocks here: two FP64 plans and the complex128 orbitals share the GPU
    for sgn in (1.0, -1.0):
        P[S] = P0 + sgn * h * Dp
        Q[S] = Q0 + sgn * h * Dq
        plans.append(isdf.Plan(P, Q, idx, mode="fp64", max_rows=B))   # gathers the perturbed points
    torch.cuda.synchronize()
    # the rows at S themselves, with their own perturbed values
    rows_s = []
    for pl, sgn in zip(plans, (1.0, -1.0)):
        P[S] = P0 + sgn * h * Dp
        Q[S] = Q0 + sgn * h * Dq
        rows_s.append(torch.stack([pl.fit_theta(int(r), 1)[0] for r in S.tolist()]))
        torch.cuda.synchronize()
    P[S], Q[S] = P0, Q0
    tot = q_diff(rows_s[0], rows_s[1])
    tp = torch.empty((B, w.n_mu), dtype=torch.complex128, device=DEV)
    tm = torch.empty_like(tp)
    s_h = S.cpu().numpy()
    for r0 in range(0, w.n_r, B):
        n = min(B, w.n_r - r0)
        plans[0].fit_theta(r0, n, out=tp[:n])
        plans[1].fit_theta(r0, n, out=tm[:n])
        # every row of the block but those at S (fitted above from their perturbed values)
        loc = torch.from_numpy(s_h[(s_h >= r0) & (s_h < r0 + n)] - r0).to(DEV)
        tot += q_diff(tp[:n], tm[:n]) - (q_diff(tp[loc], tm[loc]) if len(loc) else 0.0)
    for pl in plans:
        pl.check()
        pl.close()
    fd = w.dV * tot / (2 * h)
    assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)
