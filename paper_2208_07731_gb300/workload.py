"""Seeded synthetic plane-wave workloads for the complex-valued K-means ISDF.

This module only manufactures inputs: complex Bloch orbitals on a cubic grid,
the seeded weighted-random K-means initialisation, the Hermitian matrix of the
exchange-like surrogate loss and row subsamples. It holds none of the ISDF
arithmetic (no weights, no K-means step, no fit), and both the CUDA path and
the CPU oracle consume exactly the arrays it returns.

The paper's workloads are DFT orbitals of liquid water, silicon, an Al-Si
alloy and silica (Sec. 3, Table 2). Those structures and pseudopotentials are
not available, so the orbitals here are random plane-wave expansions with the
paper's grids and cutoffs: coefficients c_iG = (a + i b)/sqrt(2), a, b ~ N(0, 1),
damped by exp(-|G|^2/4) over the sphere |G|^2/2 <= E_cut, optionally plus
Gaussian-localised density centres, times the Bloch phase exp(i k.r), then
orthonormalised (the Q of A = QR with a real positive R diagonal, by
Cholesky-QR applied twice) and scaled
so that sum_r conj(phi_i) phi_j dV = delta_ij.

Grid convention: n^3 points, linear index r = (ix*n + iy)*n + iz, coordinates
x_r = h*(ix, iy, iz) with h = L/n.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic ISDF decomposition problem (sizes follow Sec. 3)."""
    name: str
    n: int            # grid points per axis; N_r = n^3
    L: float          # cubic cell edge in bohr
    n_orb: int        # N_phi = N_psi
    n_mu: int         # number of interpolation points
    dtype: str        # "c128" or "c64": storage type of the orbitals
    iters: int        # Lloyd iterations T
    ecut: float       # plane-wave cutoff in Ha
    kfrac: tuple      # Bloch vector k in units of 2*pi/L
    centres: str      # "none", "random48" or "lattice6"
    seed: int

    @property
    def n_r(self) -> int:
        return self.n ** 3

    @property
    def h(self) -> float:
        return self.L / self.n

    @property
    def dV(self) -> float:
        return self.L ** 3 / self.n_r


WORKLOADS = {
    # plain FP64, tiny: 24^3 grid, 16 orbitals, 128 points, 50 iterations
    "tiny": Workload("tiny", 24, 10.0, 16, 128, "c128", 50, 10.0, (0.25, 0.0, 0.0), "none", 0),
    # plain FP64, medium: 48^3 grid, 128 orbitals, 1024 points, 100 iterations
    "medium": Workload("medium", 48, 18.0, 128, 1024, "c128", 100, 20.0, (0.25, 0.25, 0.0), "none", 1),
    # mixed precision, water-box-like: 96^3 grid, 256 complex64 orbitals, 2048 points
    "waterbox": Workload("waterbox", 96, 23.5, 256, 2048, "c64", 100, 20.0, (0.25, 0.25, 0.0), "random48", 2),
    # differentiation: 72^3 grid, 192 complex64 orbitals, 1536 points
    "adjoint": Workload("adjoint", 72, 17.625, 192, 1536, "c64", 100, 20.0, (0.25, 0.25, 0.0), "none", 3),
    # large: 128^3 grid, 1024 complex64 orbitals, 4096 points, silica-like lattice of centres
    "silica": Workload("silica", 128, 30.0, 1024, 4096, "c64", 100, 20.0, (0.25, 0.25, 0.0), "lattice6", 4),
    # 8 pairs (k-points) on one 48^3 grid with small N: the batched decompositions
    "kpoints": Workload("kpoints", 48, 18.0, 32, 256, "c128", 100, 20.0, (0.0, 0.0, 0.0), "none", 5),
}


def kpoint_pairs(w: Workload, count: int, device="cpu"):
    """`count` orbital pairs on one grid, like the k-points of one cell: pair b uses the Bloch vector
    k_b = (b % 4, b // 4, 0) / 8 (units of 2 pi / L) and seed w.seed + 100 b; (Phi_b, Psi_b) complex128."""
    out = []
    for b in range(count):
        wb = dataclasses.replace(w, kfrac=(0.125 * (b % 4), 0.125 * (b // 4), 0.0), seed=w.seed + 100 * b)
        out.append(make_pair(wb, device))
    return out


def small_workload(n=8, L=6.0, n_orb=4, n_mu=16, iters=10, ecut=6.0, seed=7,
                   dtype="c128", centres="none") -> Workload:
    """A user-sized workload for tests (same recipe, free sizes)."""
    return Workload(f"small{n}", n, L, n_orb, n_mu, dtype, iters, ecut,
                    (0.25, 0.125, 0.0), centres, seed)


def _gvectors(w: Workload):
    m_max = int(math.floor(math.sqrt(2.0 * w.ecut) * w.L / (2.0 * math.pi)))
    if 2 * m_max >= w.n:
        raise ValueError("cutoff sphere does not fit the FFT grid")
    r = np.arange(-m_max, m_max + 1)
    mx, my, mz = np.meshgrid(r, r, r, indexing="ij")
    m = np.stack([mx.ravel(), my.ravel(), mz.ravel()], axis=1)
    G = (2.0 * math.pi / w.L) * m
    keep = 0.5 * np.sum(G * G, axis=1) <= w.ecut
    return m[keep], G[keep]


def _centre_positions(w: Workload, rng: np.random.Generator):
    if w.centres == "none":
        return None
    if w.centres == "random48":
        return rng.uniform(0.0, w.L, size=(48, 3))
    if w.centres == "lattice6":
        a = w.L / 6.0
        g = (np.arange(6) + 0.5) * a
        X, Y, Zc = np.meshgrid(g, g, g, indexing="ij")
        return np.stack([X.ravel(), Y.ravel(), Zc.ravel()], axis=1)
    raise ValueError(w.centres)


def _coefficients(w: Workload, G: np.ndarray, seed: int) -> np.ndarray:
    """Plane-wave coefficients (n_orb x n_G, complex128) for one orbital set."""
    rng = np.random.default_rng(seed)
    nG = G.shape[0]
    g2 = np.sum(G * G, axis=1)
    c = (rng.standard_normal((w.n_orb, nG)) + 1j * rng.standard_normal((w.n_orb, nG))) / math.sqrt(2.0)
    c *= np.exp(-g2 / 4.0)[None, :]
    R = _centre_positions(w, rng)
    if R is not None:
        sigma = 1.0
        g = (rng.standard_normal((w.n_orb, R.shape[0])) + 1j * rng.standard_normal((w.n_orb, R.shape[0]))) / math.sqrt(2.0)
        E = np.exp(-1j * (R @ G.T))                         # centres x G
        loc = (g @ E) * np.exp(-0.5 * g2 * sigma * sigma)[None, :]
        beta = np.linalg.norm(c) / np.linalg.norm(loc)
        c = c + beta * loc
    return c


def make_orbitals(w: Workload, seed_offset: int, device="cpu") -> torch.Tensor:
    """Orthonormal complex128 orbitals, shape (N_r, n_orb), row-major.

    seed_offset 0 gives Phi, 1 gives Psi (independent draws, seeds 2s, 2s+1).
    """
    m, G = _gvectors(w)
    c = _coefficients(w, G, 2 * w.seed + seed_offset)
    n = w.n
    grid = torch.zeros((w.n_orb, n, n, n), dtype=torch.complex128, device=device)
    mi = torch.as_tensor(np.mod(m, n), device=device)
    grid[:, mi[:, 0], mi[:, 1], mi[:, 2]] = torch.as_tensor(c, device=device)
    psi = torch.fft.ifftn(grid, dim=(1, 2, 3)) * float(n ** 3)
    del grid
    # Bloch phase exp(i k.r) with k = kfrac * 2*pi/L and r = h*(ix, iy, iz)
    idx = torch.arange(n, device=device, dtype=torch.float64)
    ph = [torch.exp(1j * (2.0 * math.pi * kf / n) * idx) for kf in w.kfrac]
    phase = ph[0][:, None, None] * ph[1][None, :, None] * ph[2][None, None, :]
    psi = (psi * phase[None]).reshape(w.n_orb, w.n_r).transpose(0, 1).contiguous()
    Q = _orthonormalise(psi)
    del psi
    return (Q / math.sqrt(w.dV)).contiguous()


def _orthonormalise(A: torch.Tensor) -> torch.Tensor:
    """Q of the QR factorisation A = QR with a real positive R diagonal.

    Cholesky-QR applied twice: G = A^H A = R^H R (the small N x N Gram matrix is
    factored on the host), A <- A R^-1. Only matrix products run on the
    device, so no GPU linear-algebra library is needed.
    """
    for _ in range(2):
        G = (A.conj().transpose(0, 1) @ A).cpu().numpy()
        G = 0.5 * (G + G.conj().T)
        R = np.linalg.cholesky(G).conj().T
        Rinv = np.linalg.solve(R, np.eye(R.shape[0], dtype=R.dtype))
        A = A @ torch.from_numpy(np.triu(Rinv)).to(A.device)
    return A


def make_pair(w: Workload, device="cpu"):
    """(Phi, Psi) in complex128 on `device`."""
    return make_orbitals(w, 0, device), make_orbitals(w, 1, device)


def storage(x: torch.Tensor, w: Workload) -> torch.Tensor:
    """Round to the workload's storage dtype (complex64 for the mixed configs)."""
    return x.to(torch.complex64) if w.dtype == "c64" else x


def init_indices(weights: np.ndarray, n_mu: int, seed: int) -> np.ndarray:
    """Seeded weighted-random distinct grid indices, P(r) proportional to w(r).

    Efraimidis-Spirakis sampling without replacement: key_r = -ln(u_r)/w_r with
    u_r uniform in (0, 1], keep the n_mu smallest keys (ties broken by r), and
    return them in ascending grid order. The paper leaves the initialisation
    open (Algorithm 1, first step); points with w = 0 are never drawn unless
    fewer than n_mu points carry weight.
    """
    w = np.asarray(weights, dtype=np.float64)
    rng = np.random.default_rng(seed)
    u = 1.0 - rng.random(w.shape[0])
    with np.errstate(divide="ignore"):
        key = np.where(w > 0, -np.log(u) / np.where(w > 0, w, 1.0), np.inf)
    order = np.argsort(key, kind="stable")[:n_mu]
    return np.sort(order).astype(np.int64)


def loss_matrix(n_mu: int, seed: int) -> np.ndarray:
    """Seeded Hermitian positive-definite K = Q diag(lambda) Q^H, lambda in [1, 10]."""
    rng = np.random.default_rng(seed)
    A = (rng.standard_normal((n_mu, n_mu)) + 1j * rng.standard_normal((n_mu, n_mu))) / math.sqrt(2.0)
    Q, _ = np.linalg.qr(A)
    lam = rng.uniform(1.0, 10.0, size=n_mu)
    K = (Q * lam[None, :]) @ Q.conj().T
    return 0.5 * (K + K.conj().T)


def subsample_rows(n_r: int, count: int, seed: int) -> np.ndarray:
    """Seeded row sample without replacement, ascending."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n_r, size=min(count, n_r), replace=False)).astype(np.int64)


def directions(shape, count: int, seed: int):
    """Seeded complex directions of unit Frobenius norm (for finite differences)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        d = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        out.append(d / np.linalg.norm(d))
    return out
