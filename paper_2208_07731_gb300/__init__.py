"""GB300-native complex-valued K-means ISDF (arXiv 2208.07731).

Thin Python binding over the C ABI of libisdf.so (include/isdf.h). Every
function below only marshals torch CUDA tensors into pointers, sizes and the
current stream; every step of the method runs in the library's CUDA kernels.
There is no CPU fallback: a missing or unloadable library raises.

    import paper_2208_07731_gb300 as isdf
    w = isdf.weights(phi, psi)                                   # Sec. 2.2, Eq. weight function 2
    km = isdf.kmeans(w, (n, n, n), (L, L, L), n_mu, init, iters)  # Algorithm 1
    plan = isdf.Plan(phi, psi, km["idx"], mode="fp64")            # Eq. theta
    theta = plan.fit_theta()
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libisdf.so")
_lib = None

C128, C64 = 0, 1
SSM, PSM = 0, 1
W_ACCUMULATE = 0x100
FP64, MIXED = 0, 1
PLAN_FP64_SIMT = 0x100   # mode flag: plan-update products on the FP64 pipe only
EARLY_STOP = 1
TIMER_KINDS = {"gram": 0, "apply": 1, "gather_M": 2, "cholesky": 3, "tri_inverse": 4, "minv": 5, "mixed_prep": 6}
STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA runtime error", 3: "C C^H is not Hermitian positive definite",
          4: "empty K-means cluster", 5: "non-finite value", 6: "bounded device wait timed out",
          7: "workspace missing or too small", 8: "unsupported size"}


class ISDFError(RuntimeError):
    def __init__(self, code: int, what: str, detail: int | None = None):
        self.code = code
        self.detail = detail
        msg = f"{what}: {STATUS.get(code, code)}"
        if detail is not None:
            msg += f" (detail {detail})"
        super().__init__(msg)


def lib():
    """Load libisdf.so (built by paper_2208_07731_gb300.build). Raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"libisdf.so is not built ({_LIB_PATH}); run paper_2208_07731_gb300.build.build()")
        L = ctypes.CDLL(_LIB_PATH)
        P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.isdf_weights.argtypes = [P, I64, I32, P, I64, I32, I64, I32, I32, D, P, P]
        L.isdf_kmeans_workspace.argtypes = [I32, I32, I32, I32, P]
        L.isdf_kmeans.argtypes = [P, I32, I32, I32, P, I32, P, I32, I32, P, P, P, P, P, P, ctypes.c_size_t, P]
        L.isdf_plan_create.argtypes = [P, P, I64, P, I64, I64, I32, I32, I32, P, I32, I32, I64, P]
        L.isdf_fit_theta.argtypes = [P, I64, I64, P, I64, P]
        L.isdf_fit_theta_host.argtypes = [P, I64, I64, P, I64, P]
        L.isdf_fit_theta_backward.argtypes = [P, I64, I64, P, I64, P, D, P, I64, P, I64, P, P]
        L.isdf_fit_theta_backward_finalize.argtypes = [P, P, I64, P, I64, P]
        L.isdf_plan_status.argtypes = [P, P]
        L.isdf_plan_copy_matrix.argtypes = [P, I32, P, P]
        L.isdf_plan_update.argtypes = [P, P, P]
        L.isdf_plan_set_wait_budget.argtypes = [P, I64]
        L.isdf_kmeans_status.argtypes = [P, P]
        L.isdf_fit_error.argtypes = [P, I64, I64, P, P]
        L.isdf_cluster_residual.argtypes = [P, I64, I32, P, I64, I32, I64, I32, P, P, I32, P, P, P]
        L.isdf_batch_create.argtypes = [P, I32, P, P, P, P, I64, I32, I32, I32, P, I32, I32, I64, P]
        L.isdf_batch_update.argtypes = [P, P, P]
        L.isdf_batch_fit_theta.argtypes = [P, I64, I64, P, I64, P]
        L.isdf_batch_plan.argtypes = [P, I32]
        L.isdf_batch_plan.restype = ctypes.c_void_p
        L.isdf_batch_status.argtypes = [P, P, P]
        L.isdf_batch_destroy.argtypes = [P]
        L.isdf_batch_destroy.restype = None
        for f in ("isdf_batch_create", "isdf_batch_update", "isdf_batch_fit_theta", "isdf_batch_status"):
            getattr(L, f).restype = ctypes.c_int32
        L.isdf_qrcp_points.argtypes = [P, I64, I32, P, I64, I32, I64, I32, P, P, I32, I32, P, P, P]
        L.isdf_qrcp_points.restype = ctypes.c_int32
        L.isdf_exchange_create.argtypes = [P, I32, I32, I32, P, I32, I32, I32, I32, I32, I32, D, P, I64, P]
        L.isdf_exchange_potential.argtypes = [P, P, I64, P, I64, P]
        L.isdf_exchange_apply.argtypes = [P, P, I64, P, I64, P, P, I64, I64, I64, P, I64, P]
        L.isdf_exchange_status.argtypes = [P]
        L.isdf_exchange_destroy.argtypes = [P]
        L.isdf_exchange_destroy.restype = None
        L.isdf_plan_enable_timing.argtypes = [P, I32]
        L.isdf_plan_kernel_time.argtypes = [P, I32, P, P, P]
        L.isdf_kernel_launches.argtypes = []
        L.isdf_kernel_launches.restype = ctypes.c_ulonglong
        L.isdf_plan_destroy.argtypes = [P]
        L.isdf_status_string.argtypes = [I32]
        L.isdf_status_string.restype = ctypes.c_char_p
        for f in ("isdf_weights", "isdf_kmeans_workspace", "isdf_kmeans", "isdf_plan_create", "isdf_fit_theta",
                  "isdf_fit_theta_host", "isdf_fit_theta_backward", "isdf_fit_theta_backward_finalize", "isdf_plan_status",
                  "isdf_plan_copy_matrix", "isdf_plan_update", "isdf_plan_enable_timing", "isdf_plan_kernel_time",
                  "isdf_fit_error", "isdf_cluster_residual", "isdf_exchange_create", "isdf_exchange_potential",
                  "isdf_exchange_apply", "isdf_exchange_status", "isdf_plan_set_wait_budget",
                  "isdf_kmeans_status"):
            getattr(L, f).restype = ctypes.c_int32
        _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != 0:
        raise ISDFError(rc, what)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _orbitals(x: torch.Tensor):
    """(pointer tensor, ld, n, dtype code) of an N_r x N complex CUDA matrix with unit column stride."""
    if not x.is_cuda or x.dim() != 2 or x.stride(1) != 1:
        raise ValueError("orbitals must be 2-D CUDA tensors with contiguous rows")
    if x.dtype == torch.complex128:
        code = C128
    elif x.dtype == torch.complex64:
        code = C64
    else:
        raise TypeError("orbitals must be complex128 or complex64")
    return x, x.stride(0), x.shape[1], code


def weights(phi: torch.Tensor, psi: torch.Tensor, kind: str = "ssm", alpha: float = 2.0, out=None, stream=None,
            accumulate: bool = False):
    """w(r) = sum_i |phi_i|^alpha + sum_j |psi_j|^alpha (kind "ssm") or the PSM product (kind "psm");
    accumulate=True adds the pair's weight into out (a weight shared by several pairs)."""
    a, lda, na, ca = _orbitals(phi)
    b, ldb, nb, cb = _orbitals(psi)
    if ca != cb or a.shape[0] != b.shape[0]:
        raise ValueError("phi and psi must share dtype and row count")
    n_r = a.shape[0]
    if accumulate and out is None:
        raise ValueError("accumulate needs the running weight as out")
    w = out if out is not None else torch.empty(n_r, dtype=torch.float64, device=a.device)
    code = (PSM if kind == "psm" else SSM) | (W_ACCUMULATE if accumulate else 0)
    _check(lib().isdf_weights(_ptr(a), lda, na, _ptr(b), ldb, nb, n_r, ca, code, float(alpha), _ptr(w),
                              _stream(stream)), "isdf_weights")
    return w


def kmeans_workspace_bytes(shape, n_mu: int) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().isdf_kmeans_workspace(int(shape[0]), int(shape[1]), int(shape[2]), int(n_mu), ctypes.byref(n)),
           "isdf_kmeans_workspace")
    return int(n.value)


def kmeans(w: torch.Tensor, shape, cell, n_mu: int, init_idx: torch.Tensor, max_iter: int,
           early_stop: bool = False, workspace: torch.Tensor | None = None, labels: bool = True,
           objective: bool = True, stream=None) -> dict:
    """Weighted Lloyd K-means on the grid; returns device tensors idx, centroids,
    objective, labels and stats = (updates, near ties, empty clusters, FP64-decided points)."""
    nx, ny, nz = (int(v) for v in shape)
    dev = w.device
    if w.dtype != torch.float64 or not w.is_cuda or not w.is_contiguous() or w.numel() != nx * ny * nz:
        raise ValueError("w must be a contiguous float64 CUDA tensor of nx*ny*nz entries")
    init = init_idx.to(device=dev, dtype=torch.int64).contiguous()
    if init.numel() != n_mu:
        raise ValueError("init_idx must hold n_mu indices")
    nbytes = kmeans_workspace_bytes(shape, n_mu)
    ws = workspace if workspace is not None else torch.empty(nbytes, dtype=torch.uint8, device=dev)
    if ws.numel() < nbytes:
        raise ValueError("workspace too small")
    idx = torch.empty(n_mu, dtype=torch.int64, device=dev)
    cen = torch.empty((n_mu, 3), dtype=torch.float64, device=dev)
    obj = torch.empty(max_iter + 1, dtype=torch.float64, device=dev) if objective else None
    lab = torch.empty(nx * ny * nz, dtype=torch.int32, device=dev) if labels else None
    stats = torch.zeros(4, dtype=torch.int64, device=dev)
    cellh = (ctypes.c_double * 3)(*[float(c) for c in cell])
    _check(lib().isdf_kmeans(_ptr(w), nx, ny, nz, cellh, int(n_mu), _ptr(init), int(max_iter),
                             EARLY_STOP if early_stop else 0, _ptr(idx), _ptr(cen), _ptr(obj), _ptr(lab),
                             _ptr(stats), _ptr(ws), ws.numel(), _stream(stream)), "isdf_kmeans")
    return {"idx": idx, "centroids": cen, "objective": obj, "labels": lab, "stats": stats}


def kmeans_status(km: dict, stream=None) -> int:
    """Status code of a finished kmeans() call (isdf_kmeans_status; synchronises the stream):
    0, or ISDF_ERR_EMPTY_CLUSTER / ISDF_ERR_NONFINITE / ISDF_ERR_INVALID_ARG."""
    return int(lib().isdf_kmeans_status(_ptr(km["stats"]), _stream(stream)))


def kmeans_check(km: dict, stream=None):
    """Raise ISDFError unless the kmeans() call ended without an empty cluster or bad input."""
    _check(kmeans_status(km, stream), "isdf_kmeans")


class Plan:
    """Theta fit at fixed interpolation points (isdf_plan_*): gathers Phi_mu,
    Psi_mu, forms M = C C^H in FP64, factors it and forms M^-1 on creation.
    fp64_products="tensor" runs the large FP64 products of that update on the
    tensor cores by exact integer slicing (FP64-level error); "simt" keeps
    them on the FP64 pipe."""

    def __init__(self, phi: torch.Tensor, psi: torch.Tensor, idx: torch.Tensor, mode: str = "fp64",
                 max_rows: int = 65536, stream=None, fp64_products: str = "tensor"):
        a, lda, na, ca = _orbitals(phi)
        b, ldb, nb, cb = _orbitals(psi)
        if ca != cb or a.shape[0] != b.shape[0]:
            raise ValueError("phi and psi must share dtype and row count")
        self.phi, self.psi = a, b
        self.idx = idx.to(device=a.device, dtype=torch.int64).contiguous()
        self.n_r, self.n_phi, self.n_psi, self.n_mu = a.shape[0], na, nb, self.idx.numel()
        self.mode = MIXED if mode == "mixed" else FP64
        self.theta_dtype = torch.complex64 if self.mode == MIXED else torch.complex128
        self._h = ctypes.c_void_p(0)
        if fp64_products not in ("tensor", "simt"):
            raise ValueError("fp64_products is 'tensor' (exact-slicing tensor-core products) or 'simt'")
        flags = PLAN_FP64_SIMT if fp64_products == "simt" else 0
        _check(lib().isdf_plan_create(ctypes.byref(self._h), _ptr(a), lda, _ptr(b), ldb, self.n_r, na, nb, ca,
                                      _ptr(self.idx), self.n_mu, self.mode | flags, int(max_rows), _stream(stream)),
               "isdf_plan_create")

    def close(self):
        if self._h and self._h.value:
            lib().isdf_plan_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def status(self):
        d = ctypes.c_int32(0)
        rc = lib().isdf_plan_status(self._h, ctypes.byref(d))
        return int(rc), int(d.value)

    def check(self):
        rc, d = self.status()
        if rc != 0:
            raise ISDFError(rc, "isdf_plan_status", d)

    def matrix(self, which: str, stream=None) -> torch.Tensor:
        """Copy of a plan-owned matrix: "M", "L", "Minv", "Phi_mu", "Psi_mu"."""
        code = {"M": 0, "L": 1, "Minv": 2, "Phi_mu": 3, "Psi_mu": 4}[which]
        cols = self.n_mu if code < 3 else (self.n_phi if code == 3 else self.n_psi)
        out = torch.empty((self.n_mu, cols), dtype=torch.complex128, device=self.phi.device)
        _check(lib().isdf_plan_copy_matrix(self._h, code, _ptr(out), _stream(stream)), "isdf_plan_copy_matrix")
        return out

    def update(self, idx: torch.Tensor, stream=None):
        """Recompute the plan for new interpolation points (and the current orbitals) without reallocating."""
        self.idx = idx.to(device=self.phi.device, dtype=torch.int64).contiguous()
        if self.idx.numel() != self.n_mu:
            raise ValueError("update needs the plan's n_mu points")
        _check(lib().isdf_plan_update(self._h, _ptr(self.idx), _stream(stream)), "isdf_plan_update")

    def set_wait_budget(self, cycles: int):
        """Cycle budget of the tensor-core kernels' pipeline waits for later launches (<= 0: default)."""
        _check(lib().isdf_plan_set_wait_budget(self._h, int(cycles)), "isdf_plan_set_wait_budget")

    def enable_timing(self, capacity: int = 4096):
        _check(lib().isdf_plan_enable_timing(self._h, int(capacity)), "isdf_plan_enable_timing")

    def kernel_time(self, kind: str):
        """(total ms, launches, rows) of a timed kind since the last query: 'gram', 'apply' (the two
        GEMM kernels) or a plan stage 'gather_M', 'cholesky', 'tri_inverse', 'minv', 'mixed_prep'."""
        ms, n, rows = ctypes.c_double(0), ctypes.c_int64(0), ctypes.c_int64(0)
        _check(lib().isdf_plan_kernel_time(self._h, TIMER_KINDS[kind], ctypes.byref(ms), ctypes.byref(n),
                                           ctypes.byref(rows)), "isdf_plan_kernel_time")
        return ms.value, n.value, rows.value

    def fit_theta(self, row_begin: int = 0, row_count: int | None = None, out=None, stream=None):
        if row_count is None:
            row_count = self.n_r - row_begin
        th = out if out is not None else torch.empty((row_count, self.n_mu), dtype=self.theta_dtype,
                                                     device=self.phi.device)
        if th.dtype != self.theta_dtype or th.stride(1) != 1:
            raise ValueError("theta output has the wrong dtype or layout")
        _check(lib().isdf_fit_theta(self._h, int(row_begin), int(row_count), _ptr(th), th.stride(0),
                                    _stream(stream)), "isdf_fit_theta")
        return th

    def fit_theta_host(self, out, row_begin: int = 0, row_count: int | None = None, stream=None):
        """Theta rows into `out`, a pinned CPU tensor (row_count x n_mu, unit column stride): each row block is
        fitted into a device staging block and copied to `out` while the next block is fitted. Ordered on
        `stream`; synchronise it before reading `out`."""
        if row_count is None:
            row_count = self.n_r - row_begin
        if out.device.type != "cpu" or not out.is_pinned():
            raise ValueError("out must be a pinned (page-locked) CPU tensor")
        if (out.dtype != self.theta_dtype or out.dim() != 2 or out.stride(1) != 1 or out.shape[0] < row_count
                or out.shape[1] < self.n_mu):
            raise ValueError("theta output has the wrong dtype, shape or layout")
        _check(lib().isdf_fit_theta_host(self._h, int(row_begin), int(row_count), _ptr(out), out.stride(0),
                                         _stream(stream)), "isdf_fit_theta_host")
        return out

    def fit_error(self, row_begin: int = 0, row_count: int | None = None, stream=None) -> dict:
        """Least-squares residual of the fit (Appendix A): device scalars z2 = ||Z||_F^2,
        trace = Re tr(Theta^H Y), and the relative error sqrt(1 - trace / z2) as a float."""
        if row_count is None:
            row_count = self.n_r - row_begin
        sums = torch.zeros(2, dtype=torch.float64, device=self.phi.device)
        _check(lib().isdf_fit_error(self._h, int(row_begin), int(row_count), _ptr(sums), _stream(stream)),
               "isdf_fit_error")
        z2, tr = (float(v) for v in sums.cpu())
        return {"z2": z2, "trace": tr, "residual2": z2 - tr,
                "error": max(0.0, 1.0 - tr / z2) ** 0.5 if z2 > 0 else 0.0}

    def backward(self, row_begin: int, row_count: int, grad_phi: torch.Tensor, grad_psi: torch.Tensor,
                 grad_theta: torch.Tensor | None = None, K: torch.Tensor | None = None, dV: float = 1.0,
                 loss: torch.Tensor | None = None, stream=None):
        if grad_theta is not None and (grad_theta.dtype != self.theta_dtype or grad_theta.stride(1) != 1):
            raise ValueError("grad_theta has the wrong dtype or layout")
        if K is not None and (K.dtype != torch.complex128 or not K.is_contiguous()):
            raise ValueError("K must be a contiguous complex128 matrix")
        for g in (grad_phi, grad_psi):
            if g.dtype != torch.complex128 or g.stride(1) != 1:
                raise ValueError("gradients are complex128 with contiguous rows")
        _check(lib().isdf_fit_theta_backward(self._h, int(row_begin), int(row_count), _ptr(grad_theta),
                                             grad_theta.stride(0) if grad_theta is not None else 0, _ptr(K),
                                             float(dV), _ptr(grad_phi), grad_phi.stride(0), _ptr(grad_psi),
                                             grad_psi.stride(0), _ptr(loss), _stream(stream)),
               "isdf_fit_theta_backward")

    def backward_finalize(self, grad_phi: torch.Tensor, grad_psi: torch.Tensor, stream=None):
        _check(lib().isdf_fit_theta_backward_finalize(self._h, _ptr(grad_phi), grad_phi.stride(0), _ptr(grad_psi),
                                                      grad_psi.stride(0), _stream(stream)),
               "isdf_fit_theta_backward_finalize")


def cluster_residual(phi: torch.Tensor, psi: torch.Tensor, labels: torch.Tensor, idx: torch.Tensor,
                     stream=None) -> dict:
    """R of Eq. errorISDF: every row Z(r) projected on the row of its cluster's point
    idx[labels[r]] (Appendix A); returns {"R", "z2"} as floats."""
    a, lda, na, ca = _orbitals(phi)
    b, ldb, nb, cb = _orbitals(psi)
    if ca != cb or a.shape[0] != b.shape[0]:
        raise ValueError("phi and psi must share dtype and row count")
    lab = labels.to(device=a.device, dtype=torch.int32).contiguous()
    ix = idx.to(device=a.device, dtype=torch.int64).contiguous()
    if lab.numel() != a.shape[0]:
        raise ValueError("labels must hold one entry per grid point")
    sums = torch.zeros(2, dtype=torch.float64, device=a.device)
    bad = torch.zeros(1, dtype=torch.int32, device=a.device)
    _check(lib().isdf_cluster_residual(_ptr(a), lda, na, _ptr(b), ldb, nb, a.shape[0], ca, _ptr(lab), _ptr(ix),
                                       ix.numel(), _ptr(sums), _ptr(bad), _stream(stream)), "isdf_cluster_residual")
    if int(bad.item()):
        raise ValueError("labels or idx out of range")
    z2, R = (float(v) for v in sums.cpu())
    return {"R": R, "z2": z2}


def qrcp_points(phi: torch.Tensor, psi: torch.Tensor, A: torch.Tensor, B: torch.Tensor, n_mu: int,
                stream=None) -> dict:
    """Interpolation points by column-pivoted QR of the randomized sketch S^T, S = (Phi A) o conj(Psi B)
    (Sec. 2.1, Eq. QRCP): device tensors idx (n_mu) and rdiag = |R_kk|. A: N_phi x p, B: N_psi x p."""
    a, lda, na, ca = _orbitals(phi)
    b, ldb, nb, cb = _orbitals(psi)
    if ca != cb or a.shape[0] != b.shape[0]:
        raise ValueError("phi and psi must share dtype and row count")
    Ad = A.to(device=a.device, dtype=torch.complex128).contiguous()
    Bd = B.to(device=a.device, dtype=torch.complex128).contiguous()
    p = Ad.shape[1]
    if Ad.shape[0] != na or tuple(Bd.shape) != (nb, p):
        raise ValueError("A must be N_phi x p and B N_psi x p")
    idx = torch.empty(int(n_mu), dtype=torch.int64, device=a.device)
    rdiag = torch.empty(int(n_mu), dtype=torch.float64, device=a.device)
    _check(lib().isdf_qrcp_points(_ptr(a), lda, na, _ptr(b), ldb, nb, a.shape[0], ca, _ptr(Ad), _ptr(Bd), int(p),
                                  int(n_mu), _ptr(idx), _ptr(rdiag), _stream(stream)), "isdf_qrcp_points")
    return {"idx": idx, "rdiag": rdiag}


class Batch:
    """Batched decompositions (isdf_batch_*): one plan per orbital pair on a shared grid and shared
    interpolation points; update() and fit_theta() run the pairs on concurrent streams."""

    def __init__(self, pairs, idx: torch.Tensor, mode: str = "fp64", max_rows: int = 65536, stream=None):
        if len(pairs) == 0:
            raise ValueError("a batch needs at least one orbital pair")
        ops = [(_orbitals(p), _orbitals(q)) for p, q in pairs]
        if len({a.device for (a, _, _, _), _ in ops} | {b.device for _, (b, _, _, _) in ops}) != 1:
            raise ValueError("every pair must live on the same device")
        (a0, _, na, ca), (_, _, nb, cb) = ops[0]
        for (a, _, n1, c1), (b, _, n2, c2) in ops:
            if (n1, n2, c1, c2) != (na, nb, ca, cb) or a.shape[0] != a0.shape[0] or b.shape[0] != a0.shape[0]:
                raise ValueError("every pair must share sizes and dtype")
        self.pairs = [(a, b) for (a, _, _, _), (b, _, _, _) in ops]
        self.count, self.n_r, self.n_mu = len(ops), a0.shape[0], idx.numel()
        self.idx = idx.to(device=a0.device, dtype=torch.int64).contiguous()
        self.mode = MIXED if mode == "mixed" else FP64
        self.theta_dtype = torch.complex64 if self.mode == MIXED else torch.complex128
        n = self.count
        P = ctypes.c_void_p
        self._phi = (P * n)(*[a.data_ptr() for (a, _, _, _), _ in ops])
        self._psi = (P * n)(*[b.data_ptr() for _, (b, _, _, _) in ops])
        self._ldp = (ctypes.c_int64 * n)(*[lda for (_, lda, _, _), _ in ops])
        self._ldq = (ctypes.c_int64 * n)(*[ldb for _, (_, ldb, _, _) in ops])
        self._h = P(0)
        _check(lib().isdf_batch_create(ctypes.byref(self._h), n, self._phi, self._ldp, self._psi, self._ldq,
                                       self.n_r, na, nb, ca, _ptr(self.idx), self.n_mu, self.mode, int(max_rows),
                                       _stream(stream)), "isdf_batch_create")

    def close(self):
        if self._h and self._h.value:
            lib().isdf_batch_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self):
        which, d = ctypes.c_int32(-1), ctypes.c_int32(0)
        rc = lib().isdf_batch_status(self._h, ctypes.byref(which), ctypes.byref(d))
        if rc != 0:
            raise ISDFError(rc, f"isdf_batch_status (pair {which.value})", d.value)

    def update(self, idx: torch.Tensor, stream=None):
        self.idx = idx.to(device=self.idx.device, dtype=torch.int64).contiguous()
        _check(lib().isdf_batch_update(self._h, _ptr(self.idx), _stream(stream)), "isdf_batch_update")

    def fit_theta(self, row_begin: int = 0, row_count: int | None = None, out=None, stream=None):
        """Theta of every pair (a list of row_count x n_mu tensors)."""
        if row_count is None:
            row_count = self.n_r - row_begin
        th = out if out is not None else [torch.empty((row_count, self.n_mu), dtype=self.theta_dtype,
                                                      device=self.idx.device) for _ in range(self.count)]
        ld = th[0].stride(0)
        for t in th:
            if t.dtype != self.theta_dtype or t.stride(1) != 1 or t.stride(0) != ld:
                raise ValueError("theta outputs need the mode's dtype and one common layout")
        ptrs = (ctypes.c_void_p * self.count)(*[t.data_ptr() for t in th])
        _check(lib().isdf_batch_fit_theta(self._h, int(row_begin), int(row_count), ptrs, ld, _stream(stream)),
               "isdf_batch_fit_theta")
        return th


class Exchange:
    """ISDF exchange application (Sec. 2.3, isdf_exchange_*): potential() solves the periodic
    Poisson problems V_mu = v * zeta_mu (Eq. V_mu) for all columns of Theta by FFT, apply()
    forms (V_X psi_j)(r) = -[(V o (Phi Phi_mu^H)) Psi_mu](r, j) (Eq. v2). kernel is "coulomb"
    (1/r) or "erfc" (erfc(omega r)/r). Theta must interpolate phi_i* psi_j, i.e. come from a
    Plan built on the pair (Psi, Phi)."""

    KERNELS = {"coulomb": 0, "erfc": 1}

    def __init__(self, shape, cell, n_mu: int, n_phi: int, n_psi: int, orb_dtype=torch.complex128,
                 mode: str = "fp64", kernel: str = "coulomb", omega: float = 0.0, q=None,
                 max_rows: int = 65536, device=None, stream=None):
        nx, ny, nz = (int(v) for v in shape)
        self.shape, self.n_r = (nx, ny, nz), nx * ny * nz
        self.n_mu, self.n_phi, self.n_psi = int(n_mu), int(n_phi), int(n_psi)
        self.mode = MIXED if mode == "mixed" else FP64
        self.v_dtype = torch.complex64 if self.mode == MIXED else torch.complex128
        self.orb_dtype = orb_dtype
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        cellh = (ctypes.c_double * 3)(*[float(c) for c in cell])
        qh = (ctypes.c_double * 3)(*[float(c) for c in q]) if q is not None else None
        self._h = ctypes.c_void_p(0)
        with torch.cuda.device(self.device):
            _check(lib().isdf_exchange_create(ctypes.byref(self._h), nx, ny, nz, cellh, self.n_mu, self.n_phi,
                                              self.n_psi, C64 if orb_dtype == torch.complex64 else C128, self.mode,
                                              self.KERNELS[kernel], float(omega), qh, int(max_rows),
                                              _stream(stream)), "isdf_exchange_create")

    def close(self):
        if self._h and self._h.value:
            lib().isdf_exchange_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self):
        rc = lib().isdf_exchange_status(self._h)
        if rc != 0:
            raise ISDFError(rc, "isdf_exchange_status")

    def potential(self, theta: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """V (n_r x n_mu, the dtype of the mode); out may be theta itself (in place)."""
        if theta.dtype != self.v_dtype or theta.stride(1) != 1 or tuple(theta.shape) != (self.n_r, self.n_mu):
            raise ValueError("theta must be n_r x n_mu with contiguous rows in the mode's dtype")
        v = out if out is not None else torch.empty_like(theta)
        if v.dtype != self.v_dtype or v.stride(1) != 1 or tuple(v.shape) != (self.n_r, self.n_mu):
            raise ValueError("output has the wrong dtype, shape or layout")
        _check(lib().isdf_exchange_potential(self._h, _ptr(theta), theta.stride(0), _ptr(v), v.stride(0),
                                             _stream(stream)), "isdf_exchange_potential")
        return v

    def apply(self, phi: torch.Tensor, psi: torch.Tensor, idx: torch.Tensor, v: torch.Tensor,
              row_begin: int = 0, row_count: int | None = None, out=None, stream=None) -> torch.Tensor:
        """(V_X psi_j)(r) for rows [row_begin, row_begin + row_count), complex128."""
        a, lda, na, ca = _orbitals(phi)
        b, ldb, nb, cb = _orbitals(psi)
        if (a.shape[0], na, b.shape[0], nb) != (self.n_r, self.n_phi, self.n_r, self.n_psi):
            raise ValueError("phi and psi must be n_r x n_phi and n_r x n_psi as created")
        if v.dim() != 2 or v.shape[0] != self.n_r or v.shape[1] < self.n_mu:
            raise ValueError("v must hold n_r rows of n_mu potentials")
        if row_count is None:
            row_count = self.n_r - row_begin
        if a.dtype != self.orb_dtype or b.dtype != self.orb_dtype:
            raise ValueError("orbitals must have the dtype the exchange was created for")
        ix = idx.to(device=a.device, dtype=torch.int64).contiguous()
        o = out if out is not None else torch.empty((row_count, self.n_psi), dtype=torch.complex128, device=a.device)
        if v.dtype != self.v_dtype or v.stride(1) != 1 or o.dtype != torch.complex128 or o.stride(1) != 1:
            raise ValueError("v or out has the wrong dtype or layout")
        if o.dim() != 2 or o.shape[0] < row_count or o.shape[1] < self.n_psi:
            raise ValueError("out must hold row_count rows of n_psi entries")
        _check(lib().isdf_exchange_apply(self._h, _ptr(a), lda, _ptr(b), ldb, _ptr(ix), _ptr(v), v.stride(0),
                                         int(row_begin), int(row_count), _ptr(o), o.stride(0), _stream(stream)),
               "isdf_exchange_apply")
        return o


def kernel_launches() -> int:
    """Kernels launched by libisdf in this process so far."""
    return int(lib().isdf_kernel_launches())


def decompose(phi, psi, shape, cell, n_mu, init_idx, iters, mode="fp64", kind="ssm", alpha=2.0,
              early_stop=False, max_rows=65536, theta_out=None):
    """One ISDF decomposition: weights -> K-means -> Theta fit (all on the GPU)."""
    w = weights(phi, psi, kind, alpha)
    km = kmeans(w, shape, cell, n_mu, init_idx, iters, early_stop=early_stop)
    plan = Plan(phi, psi, km["idx"], mode=mode, max_rows=max_rows)
    theta = plan.fit_theta(out=theta_out)
    return {"w": w, "kmeans": km, "plan": plan, "theta": theta}


class ISDFThetaFn(torch.autograd.Function):
    """Theta(Phi, Psi) at fixed idx with the hand-written adjoint kernels.

    Forward computes Theta through the plan; backward replays the fit block by
    block (Theta is recomputed, never saved) and returns dL/dPhi, dL/dPsi in
    complex128 (torch's convention dL/dRe + i dL/dIm), cast to the input dtype.
    """

    @staticmethod
    def forward(ctx, phi, psi, idx, mode="fp64", max_rows=65536):
        plan = Plan(phi.detach(), psi.detach(), idx, mode=mode, max_rows=max_rows)
        theta = plan.fit_theta()
        ctx.plan = plan
        ctx.dtypes = (phi.dtype, psi.dtype)
        return theta

    @staticmethod
    def backward(ctx, grad_theta):
        plan = ctx.plan
        gphi = torch.zeros((plan.n_r, plan.n_phi), dtype=torch.complex128, device=grad_theta.device)
        gpsi = torch.zeros((plan.n_r, plan.n_psi), dtype=torch.complex128, device=grad_theta.device)
        g = grad_theta.to(plan.theta_dtype).contiguous()
        for r0 in range(0, plan.n_r, 1 << 20):
            n = min(1 << 20, plan.n_r - r0)
            plan.backward(r0, n, gphi, gpsi, grad_theta=g[r0:r0 + n])
        plan.backward_finalize(gphi, gpsi)
        return gphi.to(ctx.dtypes[0]), gpsi.to(ctx.dtypes[1]), None, None, None


def surrogate_loss_and_grad(plan: Plan, K: torch.Tensor, dV: float, block: int = 1 << 20):
    """Fused exchange-like surrogate L = dV sum_r Re[conj(Theta_r) K Theta_r] and
    its gradients dL/dPhi, dL/dPsi, with Theta recomputed per block (never stored)."""
    dev = plan.phi.device
    gphi = torch.zeros((plan.n_r, plan.n_phi), dtype=torch.complex128, device=dev)
    gpsi = torch.zeros((plan.n_r, plan.n_psi), dtype=torch.complex128, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    for r0 in range(0, plan.n_r, block):
        n = min(block, plan.n_r - r0)
        plan.backward(r0, n, gphi, gpsi, K=K, dV=dV, loss=loss)
    plan.backward_finalize(gphi, gpsi)
    return loss, gphi, gpsi
