"""Oracle functions. TEST INFRASTRUCTURE ONLY (see the package docstring).

The weight function and the K-means live in isdf_oracle.c (plain C, FP64,
no FMA contraction); everything from the gathered rows on is numpy/scipy in
complex128. Each function names the part of the paper it restates.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import scipy.linalg as sla

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "isdf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C half of the oracle (gcc, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.oracle_weights.argtypes = [P, ctypes.c_int64, ctypes.c_int32, P, ctypes.c_int64, ctypes.c_int32,
                                       ctypes.c_int64, ctypes.c_int32, ctypes.c_double, P]
        lib.oracle_kmeans.argtypes = [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, ctypes.c_int32, P,
                                      ctypes.c_int32, ctypes.c_int32, P, P, P, P, P, P]
        lib.oracle_fixed_point_scale.argtypes = [ctypes.c_int64, ctypes.c_double, P]
        I32, I64 = ctypes.c_int32, ctypes.c_int64
        lib.oracle_kmeans_update.argtypes = [P, I32, I32, I32, P, I32, P, P, P]
        lib.oracle_kmeans_assign.argtypes = [I32, I32, I32, P, I32, P, P, I64, P, P]
        lib.oracle_kmeans_snap.argtypes = [I32, I32, I32, P, I32, P, P, P]
        _lib = lib
    return _lib


def _c128(x) -> np.ndarray:
    x = np.asarray(x)
    if x.dtype != np.complex128:
        x = x.astype(np.complex128)  # exact for complex64
    return np.ascontiguousarray(x)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------
# Weight function, Sec. 2.2, Eq. weight function 2 (SSM and its alpha family)
# and Eq. weight function (PSM).
# --------------------------------------------------------------------------
def weights(phi, psi, kind: str = "ssm", alpha: float = 2.0) -> np.ndarray:
    phi, psi = _c128(phi), _c128(psi)
    n_r = phi.shape[0]
    assert psi.shape[0] == n_r
    w = np.empty(n_r, dtype=np.float64)
    load().oracle_weights(_ptr(phi), phi.shape[1], phi.shape[1], _ptr(psi), psi.shape[1], psi.shape[1],
                          n_r, 1 if kind == "psm" else 0, float(alpha), _ptr(w))
    return w


def fixed_point_scale(n_r: int, wmax: float, cell) -> int:
    cell = np.ascontiguousarray(cell, dtype=np.float64)
    return int(load().oracle_fixed_point_scale(n_r, float(wmax), _ptr(cell)))


# --------------------------------------------------------------------------
# Weighted K-means, Algorithm 1 with Eq. opt (second form) and Eq. r_k.
# --------------------------------------------------------------------------
def kmeans(w, shape, cell, n_mu: int, init_idx, max_iter: int, early_stop: bool = False) -> dict:
    w = np.ascontiguousarray(w, dtype=np.float64)
    nx, ny, nz = (int(v) for v in shape)
    cell = np.ascontiguousarray(cell, dtype=np.float64)
    init = np.ascontiguousarray(init_idx, dtype=np.int64)
    assert init.shape == (n_mu,) and w.shape == (nx * ny * nz,)
    idx = np.empty(n_mu, np.int64)
    cen = np.empty((n_mu, 3), np.float64)
    obj = np.empty(max_iter + 1, np.float64)
    nit = np.zeros(1, np.int32)
    ties = np.zeros(1, np.int64)
    lab = np.empty(nx * ny * nz, np.int32)
    rc = load().oracle_kmeans(_ptr(w), nx, ny, nz, _ptr(cell), n_mu, _ptr(init), max_iter, int(early_stop),
                              _ptr(idx), _ptr(cen), _ptr(obj), _ptr(nit), _ptr(ties), _ptr(lab))
    if rc < 0:
        raise ValueError("oracle_kmeans: invalid arguments")
    return {"idx": idx, "centroids": cen, "objective": obj, "n_iter": int(nit[0]),
            "near_ties": int(ties[0]), "labels": lab, "empty": int(rc)}


def kmeans_update(w, shape, cell, labels, centroids) -> np.ndarray:
    """One centroid update of Algorithm 1 (Eq. r_k, exact 128-bit sums) from given
    labels; clusters without weight keep their centroid. Returns n_mu x 3."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    nx, ny, nz = (int(v) for v in shape)
    cell = np.ascontiguousarray(cell, dtype=np.float64)
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    c_in = np.ascontiguousarray(centroids, dtype=np.float64)
    n_mu = c_in.shape[0]
    out = np.empty_like(c_in)
    if load().oracle_kmeans_update(_ptr(w), nx, ny, nz, _ptr(cell), n_mu, _ptr(lab), _ptr(c_in), _ptr(out)) != 0:
        raise ValueError("oracle_kmeans_update: invalid arguments")
    return out


def kmeans_assign(shape, cell, centroids, points) -> tuple:
    """Assignment (Eq. opt, second form) of the listed grid points by brute force:
    (labels, squared distances), lowest mu on ties."""
    nx, ny, nz = (int(v) for v in shape)
    cell = np.ascontiguousarray(cell, dtype=np.float64)
    c = np.ascontiguousarray(centroids, dtype=np.float64)
    pts = np.ascontiguousarray(points, dtype=np.int64)
    lab = np.empty(pts.shape[0], np.int32)
    dist = np.empty(pts.shape[0], np.float64)
    if load().oracle_kmeans_assign(nx, ny, nz, _ptr(cell), c.shape[0], _ptr(c), _ptr(pts), pts.shape[0], _ptr(lab),
                                   _ptr(dist)) != 0:
        raise ValueError("oracle_kmeans_assign: invalid arguments")
    return lab, dist


def kmeans_snap(shape, cell, centroids, labels) -> tuple:
    """Snap (last step of Algorithm 1): each centroid's nearest member, lowest r on
    ties, -1 for an empty cluster. Returns (idx, empty count)."""
    nx, ny, nz = (int(v) for v in shape)
    cell = np.ascontiguousarray(cell, dtype=np.float64)
    c = np.ascontiguousarray(centroids, dtype=np.float64)
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    idx = np.empty(c.shape[0], np.int64)
    rc = load().oracle_kmeans_snap(nx, ny, nz, _ptr(cell), c.shape[0], _ptr(c), _ptr(lab), _ptr(idx))
    if rc < 0:
        raise ValueError("oracle_kmeans_snap: invalid labels")
    return idx, int(rc)


def grid_coords(shape, cell) -> np.ndarray:
    """x_r = h*(ix, iy, iz) for every grid point, in FP64 (N_r x 3)."""
    nx, ny, nz = shape
    h = [cell[0] / nx, cell[1] / ny, cell[2] / nz]
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    return np.stack([ix.ravel() * h[0], iy.ravel() * h[1], iz.ravel() * h[2]], axis=1)


# --------------------------------------------------------------------------
# Interpolation vectors, Sec. 2.1: Theta = Z C^H (C C^H)^-1 (Eq. theta, read
# with the Hermitian adjoint for complex orbitals) built through the separable
# structure Z C^H = (Phi Phi_mu^H) o conj(Psi Psi_mu^H) (Eqs. phipsi,
# muRownuCol, muRownuColden), with C C^H = M formed the same way from the
# selected rows (Eq. Cmu: C's rows are Z at the interpolation points).
# --------------------------------------------------------------------------
def gather(phi, psi, idx):
    """Phi_mu = Phi[idx, :], Psi_mu = Psi[idx, :] (Eq. Cmu)."""
    idx = np.asarray(idx, dtype=np.int64)
    return _c128(np.asarray(phi)[idx]), _c128(np.asarray(psi)[idx])


def gram_hadamard(phi_rows, psi_rows, phi_mu, psi_mu) -> np.ndarray:
    """Y = (Phi Phi_mu^H) o conj(Psi Psi_mu^H) for the given rows (Eq. muRownuCol)."""
    A = _c128(phi_rows) @ phi_mu.conj().T
    B = _c128(psi_rows) @ psi_mu.conj().T
    return A * B.conj()


def form_M(phi_mu, psi_mu) -> np.ndarray:
    """M = C C^H = (Phi_mu Phi_mu^H) o conj(Psi_mu Psi_mu^H)."""
    return gram_hadamard(phi_mu, psi_mu, phi_mu, psi_mu)


def cholesky(M) -> np.ndarray:
    """Lower Cholesky factor L, M = L L^H (the linear solver of Sec. 2.4)."""
    return sla.cholesky(M, lower=True, check_finite=True)


def theta_rows(phi, psi, phi_mu, psi_mu, L, rows) -> np.ndarray:
    """Theta rows for a set of grid rows: Theta^H = L^-H (L^-1 Y^H)."""
    rows = np.asarray(rows, dtype=np.int64)
    Y = gram_hadamard(np.asarray(phi)[rows], np.asarray(psi)[rows], phi_mu, psi_mu)
    X = sla.solve_triangular(L, Y.conj().T, lower=True)
    T = sla.solve_triangular(L.conj().T, X, lower=False)
    return T.conj().T


def fit_theta(phi, psi, idx, block: int = 65536) -> dict:
    """Full Theta (N_r x N_mu, complex128), computed in row blocks."""
    phi_mu, psi_mu = gather(phi, psi, idx)
    M = form_M(phi_mu, psi_mu)
    L = cholesky(M)
    n_r = np.asarray(phi).shape[0]
    theta = np.empty((n_r, len(idx)), np.complex128)
    for b in range(0, n_r, block):
        rows = np.arange(b, min(n_r, b + block))
        theta[rows] = theta_rows(phi, psi, phi_mu, psi_mu, L, rows)
    return {"theta": theta, "M": M, "L": L, "phi_mu": phi_mu, "psi_mu": psi_mu}


# --------------------------------------------------------------------------
# Exchange-like surrogate loss and the adjoint of the Theta fit at fixed
# interpolation points (derived from Eq. theta and Eq. muRownuCol):
#   L = dV sum_r sum_{mu,nu} Re[conj(Theta_r,mu) K_mu,nu Theta_r,nu]
#   grad convention: G = dL/dRe X + i dL/dIm X, so dL = Re tr(G^H dX).
# --------------------------------------------------------------------------
def surrogate_loss(theta, K, dV: float) -> float:
    theta = _c128(theta)
    return float(dV * np.real(np.sum(theta.conj() * (theta @ np.asarray(K).T))))


def surrogate_grad_theta(theta, K, dV: float) -> np.ndarray:
    """dL/dTheta = 2 dV Theta conj(K) for Hermitian K."""
    return 2.0 * dV * (_c128(theta) @ np.asarray(K).conj())


def theta_backward(phi, psi, idx, grad_theta_fn, block: int = 65536) -> dict:
    """Gradients of a real loss of Theta(Phi, Psi) at fixed idx.

    grad_theta_fn(rows, theta_rows) -> dL/dTheta on those rows. Steps:
      Ybar = Thetabar M^-1, Mbar = -Theta^H Ybar,
      Abar = Ybar o B, Bbar = conj(Ybar) o A,
      Phibar = Abar Phi_mu, Phibar_mu += Abar^H Phi   (Psi likewise with Bbar),
      Abar_mu = Mbar o B_mu, Bbar_mu = conj(Mbar) o A_mu,
      Phibar_mu += (Abar_mu + Abar_mu^H) Phi_mu, scattered into Phibar[idx].
    """
    phi, psi = _c128(phi), _c128(psi)
    idx = np.asarray(idx, dtype=np.int64)
    phi_mu, psi_mu = gather(phi, psi, idx)
    A_mu = phi_mu @ phi_mu.conj().T
    B_mu = psi_mu @ psi_mu.conj().T
    M = A_mu * B_mu.conj()
    L = cholesky(M)
    n_r, n_mu = phi.shape[0], len(idx)
    gphi = np.zeros_like(phi)
    gpsi = np.zeros_like(psi)
    gphi_mu = np.zeros_like(phi_mu)
    gpsi_mu = np.zeros_like(psi_mu)
    Mbar = np.zeros((n_mu, n_mu), np.complex128)
    loss = 0.0
    for b in range(0, n_r, block):
        rows = np.arange(b, min(n_r, b + block))
        A = phi[rows] @ phi_mu.conj().T
        B = psi[rows] @ psi_mu.conj().T
        Y = A * B.conj()
        T = sla.solve_triangular(L.conj().T, sla.solve_triangular(L, Y.conj().T, lower=True), lower=False).conj().T
        G = grad_theta_fn(rows, T)
        # Ybar = G M^-1 (M Hermitian): Ybar^H = M^-1 G^H
        Yb = sla.solve_triangular(L.conj().T, sla.solve_triangular(L, G.conj().T, lower=True), lower=False).conj().T
        Mbar -= T.conj().T @ Yb
        Ab = Yb * B
        Bb = Yb.conj() * A
        gphi[rows] += Ab @ phi_mu
        gpsi[rows] += Bb @ psi_mu
        gphi_mu += Ab.conj().T @ phi[rows]
        gpsi_mu += Bb.conj().T @ psi[rows]
    Ab_mu = Mbar * B_mu
    Bb_mu = Mbar.conj() * A_mu
    gphi_mu += (Ab_mu + Ab_mu.conj().T) @ phi_mu
    gpsi_mu += (Bb_mu + Bb_mu.conj().T) @ psi_mu
    np.add.at(gphi, idx, gphi_mu)
    np.add.at(gpsi, idx, gpsi_mu)
    return {"grad_phi": gphi, "grad_psi": gpsi, "Mbar": Mbar, "L": L}


def explicit_Z(phi, psi) -> np.ndarray:
    """Z(r) = [phi_i(r) conj(psi_j(r))]_{i,j}, N_r x (N_phi N_psi), column i*N_psi + j
    (the transposed Khatri-Rao product, Sec. 1). Small inputs only."""
    phi, psi = _c128(phi), _c128(psi)
    return (phi[:, :, None] * psi.conj()[:, None, :]).reshape(phi.shape[0], -1)


# --------------------------------------------------------------------------
# Diagnostics of the decomposition (Appendix A).
def isdf_error(phi, psi, idx, block: int = 65536, row_range=None) -> dict:
    """||Z - Theta C||_F^2 and ||Z||_F^2 without forming Z: Theta solves the least-squares
    problem min ||Z - Theta C|| (Eq. theta), so ||Z - Theta C||^2 = ||Z||^2 - Re tr(Theta^H Y)
    with Y = Z C^H (Eq. muRownuCol), and ||Z(r)||^2 = (sum_i |phi_i(r)|^2)(sum_j |psi_j(r)|^2)
    (Eq. Zmu). row_range = (begin, end) restricts both sums to those grid rows (C still
    comes from idx over the whole grid). Returns z2, trace, the squared residual and the
    relative error."""
    phi, psi = _c128(phi), _c128(psi)
    phi_mu, psi_mu = gather(phi, psi, idx)
    L = cholesky(form_M(phi_mu, psi_mu))
    r0, r1 = (0, phi.shape[0]) if row_range is None else (int(row_range[0]), int(row_range[1]))
    z2 = float(np.sum(np.sum(np.abs(phi[r0:r1]) ** 2, 1) * np.sum(np.abs(psi[r0:r1]) ** 2, 1)))
    tr = 0.0
    for b in range(r0, r1, block):
        rows = np.arange(b, min(r1, b + block))
        Y = gram_hadamard(phi[rows], psi[rows], phi_mu, psi_mu)
        T = theta_rows(phi, psi, phi_mu, psi_mu, L, rows)
        tr += float(np.real(np.sum(T.conj() * Y)))
    res2 = max(z2 - tr, 0.0)
    return {"z2": z2, "trace": tr, "residual2": res2, "error": float(np.sqrt(res2 / z2))}


def cluster_residual(phi, psi, labels, idx) -> dict:
    """R of Eq. errorISDF: every row Z(r) of cluster mu projected on the row Z(r_mu) of its
    selected point (Eq. proj), summed squared distances, written with Eq. Zmu:
    R = sum_r [p(r) q(r) - |a(r)|^2 |b(r)|^2 / (p(r_mu) q(r_mu))], p = sum_i |phi_i|^2,
    q = sum_j |psi_j|^2, a(r) = Phi(r) . Phi*(r_mu), b(r) = Psi(r) . Psi*(r_mu).
    Returns R and z2 = ||Z||_F^2."""
    phi, psi = _c128(phi), _c128(psi)
    labels = np.asarray(labels, dtype=np.int64)
    idx = np.asarray(idx, dtype=np.int64)
    p = np.sum(np.abs(phi) ** 2, 1)
    q = np.sum(np.abs(psi) ** 2, 1)
    s = idx[labels]
    a = np.sum(phi * phi[s].conj(), 1)
    b = np.sum(psi * psi[s].conj(), 1)
    R = float(np.sum(p * q - (np.abs(a) ** 2) * (np.abs(b) ** 2) / (p[s] * q[s])))
    return {"R": R, "z2": float(np.sum(p * q))}


# --------------------------------------------------------------------------
# ISDF exchange application, Sec. 2.3 (Eq. v, Eq. v2, Eq. V_mu).
# Periodic cell [0, L_x) x [0, L_y) x [0, L_z). A column f of grid samples is
# read as the band-limited periodic function sum_G c(G) exp(i G.r) with
# c = fftn(f) / N_r. A pair product that carries a Bloch phase exp(i q.r)
# (orbitals at different k) is passed as its periodic part: q then only
# enters the kernel as |G + q|, and the result is the periodic part of V.
# --------------------------------------------------------------------------
def kernel_hat(shape, cell, kind: str = "coulomb", omega: float = 0.0, q=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Fourier coefficients of the interaction on the FFT grid, as an (nx, ny, nz) array:
    4 pi / |G + q|^2 for the bare Coulomb kernel 1/|r - r'| of Eq. V_mu (the G + q = 0 term
    set to zero: the neutralising background), and 4 pi (1 - exp(-|G + q|^2 / (4 omega^2)))
    / |G + q|^2 for the short-range erfc(omega |r - r'|) / |r - r'| kernel of screened
    hybrid functionals (finite at zero: pi / omega^2). G = 2 pi m / L with m the signed
    FFT frequency of each index (numpy's fftfreq order)."""
    axes = []
    for n, L, qa in zip(shape, cell, q):
        m = np.fft.fftfreq(int(n), d=1.0 / int(n))          # 0, 1, ..., -1 (integers as floats)
        axes.append(2.0 * np.pi * m / float(L) + float(qa))
    gx, gy, gz = np.meshgrid(*axes, indexing="ij")
    g2 = gx * gx + gy * gy + gz * gz
    out = np.zeros_like(g2)
    nz_ = g2 > 0.0
    if kind == "coulomb":
        out[nz_] = 4.0 * np.pi / g2[nz_]
    elif kind == "erfc":
        if omega <= 0.0:
            raise ValueError("the erfc kernel needs omega > 0")
        out[nz_] = -4.0 * np.pi * np.expm1(-g2[nz_] / (4.0 * omega * omega)) / g2[nz_]
        out[~nz_] = np.pi / (omega * omega)
    else:
        raise ValueError(kind)
    return out


def poisson(zeta, shape, cell, kind: str = "coulomb", omega: float = 0.0, q=(0.0, 0.0, 0.0)) -> np.ndarray:
    """V_mu(r) = int zeta_mu(r') v(r - r') dr' for every column mu of zeta (N_r x N_mu, grid
    order r = (ix*ny + iy)*nz + iz), Eq. V_mu, solved in reciprocal space: V = ifftn(K^ fftn(zeta))."""
    z = _c128(zeta)
    nx, ny, nz = (int(v) for v in shape)
    n_mu = z.shape[1]
    cube = z.T.reshape(n_mu, nx, ny, nz)
    Vh = np.fft.fftn(cube, axes=(1, 2, 3)) * kernel_hat(shape, cell, kind, omega, q)[None]
    return np.ascontiguousarray(np.fft.ifftn(Vh, axes=(1, 2, 3)).reshape(n_mu, nx * ny * nz).T)


def exchange_apply(phi, psi, idx, V, rows=None) -> np.ndarray:
    """(V_X psi_j)(r) ~ -sum_mu V_mu(r) sum_i phi_i(r) phi_i*(r_mu) psi_j(r_mu), Eq. v2, for
    grid rows `rows` (all by default): -(V o (Phi Phi_mu^H)) Psi_mu, N_rows x N_psi."""
    phi, psi, V = _c128(phi), _c128(psi), _c128(V)
    idx = np.asarray(idx, dtype=np.int64)
    sel = slice(None) if rows is None else np.asarray(rows)
    A = phi[sel] @ phi[idx].conj().T                      # sum_i phi_i(r) phi_i*(r_mu)
    return -(V[sel] * A) @ psi[idx]


def exchange_direct(phi, psi, shape, cell, kind: str = "coulomb", omega: float = 0.0,
                    q=(0.0, 0.0, 0.0)) -> np.ndarray:
    """(V_X psi_j)(r) = -sum_i phi_i(r) int phi_i*(r') psi_j(r') v(r - r') dr', Eq. v, with one
    Poisson solve per pair (i, j): N_phi N_psi solves, for small cases only."""
    phi, psi = _c128(phi), _c128(psi)
    out = np.zeros((phi.shape[0], psi.shape[1]), dtype=np.complex128)
    for i in range(phi.shape[1]):
        pair = phi[:, i].conj()[:, None] * psi                  # phi_i*(r') psi_j(r'), all j
        out -= phi[:, i][:, None] * poisson(pair, shape, cell, kind, omega, q)
    return out


# --------------------------------------------------------------------------
# Interpolation points by QR with column pivoting (Sec. 2.1, Eq. QRCP), the
# accuracy comparator of the K-means selection, on a randomized sketch of Z^T.
# --------------------------------------------------------------------------
def qrcp_sketch(phi, psi, A, B) -> np.ndarray:
    """S = Z G for the random matrix G whose column k is a_k (x) conj(b_k) (A: N_phi x p, B: N_psi x p):
    S(r, k) = sum_ij phi_i(r) conj(psi_j(r)) A_ik conj(B_jk) = (Phi A)(r, k) conj((Psi B)(r, k))."""
    phi, psi, A, B = _c128(phi), _c128(psi), _c128(A), _c128(B)
    return (phi @ A) * np.conj(psi @ B)


def qrcp_points(S, n_mu: int) -> dict:
    """The first n_mu pivots of QR with column pivoting of S^T (Eq. QRCP: the columns of S^T are the grid
    points), by greedy pivoted Gram-Schmidt: at step k the column with the largest residual norm (the first
    one on ties) is the pivot r_k, |R_kk| its residual norm, and every residual column loses its component
    along the normalised pivot column. Residual norms are recomputed from the residuals at every step."""
    R = _c128(S).copy()
    norms = np.sum(np.abs(R) ** 2, axis=1)
    piv, rdiag = [], []
    for _ in range(int(n_mu)):
        j = int(np.argmax(norms))
        nrm = float(np.sqrt(norms[j]))
        q = R[j] / nrm
        piv.append(j)
        rdiag.append(nrm)
        coef = R @ q.conj()                     # q^H s_r for every column r of S^T
        R -= np.outer(coef, q)
        norms = np.sum(np.abs(R) ** 2, axis=1)
        norms[piv] = -1.0
    return {"idx": np.array(piv, dtype=np.int64), "rdiag": np.array(rdiag)}


# --------------------------------------------------------------------------
# Several orbital pairs on one grid (k-points or spin channels of complex
# Bloch orbitals, Sec. 2.1): one weight shared by all pairs.
# --------------------------------------------------------------------------
def shared_weights(pairs, kind: str = "ssm", alpha: float = 2.0) -> np.ndarray:
    """w(r) = sum_b w_b(r) over the pairs (phi_b, psi_b) in order b = 0, 1, ..., each w_b the weight
    function of Sec. 2.2, summed left to right in FP64."""
    w = None
    for phi, psi in pairs:
        wb = weights(phi, psi, kind, alpha)
        w = wb.copy() if w is None else w + wb
    return w
