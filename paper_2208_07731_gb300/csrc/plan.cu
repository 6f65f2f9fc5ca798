// Step 3 (Sec. 2.1, Eq. theta; Eqs. phipsi, muRownuCol, muRownuColden;
// Sec. 2.4): the interpolation-vector fit and its adjoint at fixed
// interpolation points. Host orchestration of the kernels in zgemm.cu,
// chol.cu and mixed.cu.
#include <stdlib.h>
#include <string.h>

#include "chol.cuh"
#include "mixed.cuh"
#include "plan.cuh"
#include "zgemm.cuh"

namespace {

__global__ void gather_rows(const void *src, int64_t ld, int type, int n, const int64_t *idx, int n_mu,
                            int64_t n_r, double2 *dst, DeviceStatus *st)
{
    const int64_t total = (int64_t)n_mu * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(e / n), i = (int)(e % n);
        int64_t r = idx[m];
        if (r < 0 || r >= n_r) {
            set_status(st, ISDF_ERR_INVALID_ARG, m);
            r = 0;
        }
        double2 v = type == ISDF_C128 ? cload(static_cast<const double2 *>(src), r * ld + i)
                                      : cload(static_cast<const float2 *>(src), r * ld + i);
        if (!isfinite(v.x) || !isfinite(v.y)) set_status(st, ISDF_ERR_NONFINITE, m);
        dst[e] = v;
    }
}

// Abar = Ybar o B (into A's place), Bbar = conj(Ybar) o A (into B's place)
__global__ void hadamard_adjoint(const double2 *Yb, double2 *A, double2 *B, int64_t total)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const double2 y = Yb[e], a = A[e], b = B[e];
        A[e] = cmul(y, b);
        B[e] = cmul(cconj(y), a);
    }
}

// X = Mbar o Bmu + (Mbar o Bmu)^H   and   Xp = conj(Mbar) o Amu + (conj(Mbar) o Amu)^H
__global__ void hermitian_parts(const double2 *Mbar, const double2 *Amu, const double2 *Bmu, double2 *X,
                                double2 *Xp, int n)
{
    const int64_t total = (int64_t)n * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        const int64_t t = (int64_t)j * n + i;
        const double2 a = cmul(Mbar[e], Bmu[e]), at = cmul(Mbar[t], Bmu[t]);
        X[e] = make_double2(a.x + at.x, a.y - at.y);
        const double2 b = cmul(cconj(Mbar[e]), Amu[e]), bt = cmul(cconj(Mbar[t]), Amu[t]);
        Xp[e] = make_double2(b.x + bt.x, b.y - bt.y);
    }
}

__global__ void scatter_add_rows(const double2 *src, int n, const int64_t *idx, int n_mu, double2 *dst, int64_t ld)
{
    const int64_t total = (int64_t)n_mu * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(e / n), i = (int)(e % n);
        double2 *d = dst + idx[m] * ld + i;
        const double2 v = src[e];
        d->x += v.x;
        d->y += v.y;
    }
}

// loss += 1/2 Re sum conj(Theta) o G   (G = 2 dV Theta conj(K))
template <typename T>
__global__ void surrogate_loss_kernel(const T *theta, int64_t ldt, const double2 *G, int64_t ldg, int rows, int n,
                                      double *loss)
{
    __shared__ double red[8];
    double s = 0.0;
    const int64_t total = (int64_t)rows * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / n), c = (int)(e % n);
        const double2 t = cload(theta, (int64_t)r * ldt + c), g = G[(int64_t)r * ldg + c];
        s += t.x * g.x + t.y * g.y;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) b += red[i];
        atomicAdd(loss, 0.5 * b);
    }
}

unsigned grid_for(int64_t total, unsigned cap = 8192)
{
    const int64_t g = (total + 255) / 256;
    return (unsigned)(g < 1 ? 1 : (g < cap ? g : cap));
}

ZOperand opnd(const void *p, int64_t s0, int64_t s1, int conj, int type)
{
    ZOperand o;
    o.p = p;
    o.s0 = s0;
    o.s1 = s1;
    o.conj = conj;
    o.type = type;
    return o;
}

ZGemm gemm1(int M, int N, int K, ZOperand A, ZOperand B, void *C, int64_t ldc, int ctype, double alpha, int beta)
{
    ZGemm g{};
    g.M = M;
    g.N = N;
    g.K = K;
    g.A1 = A;
    g.B1 = B;
    g.C = C;
    g.scm = ldc;
    g.scn = 1;
    g.ctype = ctype;
    g.alpha = alpha;
    g.beta = beta;
    g.splits = 1;
    return g;
}

// split-K factor for an M x N product over K grid rows that fits `cap` partial elements
int split_count(int M, int N, int K, size_t cap)
{
    const int tiles = ((M + 63) / 64) * ((N + 63) / 64);
    int s = 1;
    while (s < 64 && tiles * s < 2 * 152 && K / (s * 2) >= 256 && (size_t)(s * 2) * M * N <= cap) s *= 2;
    return s;
}

template <typename T>
isdf_status alloc(T **p, size_t count)
{
    ISDF_CUDA_TRY(cudaMalloc((void **)p, sizeof(T) * (count ? count : 1)));
    return ISDF_OK;
}

// Decomposition error of a row block (Appendix A diagnostics): per row, ||Z(r)||^2 =
// (sum_i |phi_i|^2)(sum_j |psi_j|^2) and Re sum_mu conj(Theta_r,mu) Y_r,mu; one warp per row,
// accumulated into sums[0], sums[1]
template <typename T>
__global__ void fit_error_kernel(const T *phi, int64_t ldp, int n_phi, const T *psi, int64_t ldq, int n_psi,
                                 const double2 *Y, const double2 *Th, int rows, int nm, double *sums)
{
    __shared__ double red[2][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double zs = 0.0, ts = 0.0;
    for (int r = blockIdx.x * (blockDim.x >> 5) + warp; r < rows; r += gridDim.x * (blockDim.x >> 5)) {
        double pp = 0.0, qq = 0.0, tt = 0.0;
        for (int i = lane; i < n_phi; i += 32) {
            const double2 a = cload(phi, (int64_t)r * ldp + i);
            pp += a.x * a.x + a.y * a.y;
        }
        for (int j = lane; j < n_psi; j += 32) {
            const double2 b = cload(psi, (int64_t)r * ldq + j);
            qq += b.x * b.x + b.y * b.y;
        }
        for (int m = lane; m < nm; m += 32) {
            const double2 t = Th[(int64_t)r * nm + m], y = Y[(int64_t)r * nm + m];
            tt += t.x * y.x + t.y * y.y;
        }
        for (int o = 16; o > 0; o >>= 1) {
            pp += __shfl_xor_sync(0xffffffffu, pp, o);
            qq += __shfl_xor_sync(0xffffffffu, qq, o);
            tt += __shfl_xor_sync(0xffffffffu, tt, o);
        }
        zs += pp * qq;
        ts += tt;
    }
    if (lane == 0) {
        red[0][warp] = zs;
        red[1][warp] = ts;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            a += red[0][i];
            b += red[1][i];
        }
        atomicAdd(sums, a);
        atomicAdd(sums + 1, b);
    }
}

// Y = A o conj(B) elementwise (rows x n_mu, leading dimension n_mu)
__global__ void hadamard_full(const double2 *A, const double2 *B, double2 *Y, int64_t total)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const double2 a = A[e], b = B[e];
        Y[e] = make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
    }
}

// M = A_mu o conj(B_mu) on the lower triangle (rows i, columns j <= i)
__global__ void hadamard_lower(const double2 *A, const double2 *B, double2 *M, int n)
{
    const int64_t total = (int64_t)n * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        if (j > i) continue;
        const double2 a = A[e], b = B[e];
        M[e] = make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
    }
}

// Y rows (and optionally the separate factors A, B) for rows [r0, r0 + rows)
isdf_status gram_hadamard_fp64(isdf_plan *p, int64_t r0, int rows, double2 *Y, double2 *A, double2 *B,
                               cudaStream_t st)
{
    const int t = p->dtype == ISDF_C128 ? ZG_C128 : ZG_C64;
    const size_t es = p->dtype == ISDF_C128 ? 16 : 8;
    ZGemm g{};
    g.M = rows;
    g.N = p->n_mu;
    g.K = p->n_phi;
    g.dual = 1;
    g.A1 = opnd(static_cast<const char *>(p->phi) + r0 * p->ld_phi * es, p->ld_phi, 1, 0, t);
    g.B1 = opnd(p->phi_mu, 1, p->n_phi, 1, ZG_C128);
    g.A2 = opnd(static_cast<const char *>(p->psi) + r0 * p->ld_psi * es, p->ld_psi, 1, 0, t);
    g.B2 = opnd(p->psi_mu, 1, p->n_psi, 1, ZG_C128);
    g.C = Y;
    g.scm = p->n_mu;
    g.scn = 1;
    g.ctype = ZG_C128;
    g.C1 = A;
    g.C2 = B;
    g.splits = 1;
    if (p->n_phi != p->n_psi) {
        // different K for the two products: run them as two single GEMMs + Hadamard
        return ISDF_ERR_UNSUPPORTED;
    }
    if (p->use_oz && p->blkA && p->blkB) {
        // the two products on the tensor cores (exact slicing), then the Hadamard product in FP64
        double2 *pa = A ? A : p->blkA, *pb = B ? B : p->blkB;
        ZGemm ga = gemm1(rows, p->n_mu, p->n_phi, g.A1, g.B1, pa, p->n_mu, ZG_C128, 1.0, 0);
        ZGemm gb = gemm1(rows, p->n_mu, p->n_psi, g.A2, g.B2, pb, p->n_mu, ZG_C128, 1.0, 0);
        if (oz_fits(ga, p->oz) && oz_fits(gb, p->oz)) {
            ISDF_TRY(oz_zgemm(ga, p->oz, p->oz_err, st));
            ISDF_TRY(oz_zgemm(gb, p->oz, p->oz_err, st));
            const int64_t tot = (int64_t)rows * p->n_mu;
            hadamard_full<<<grid_for(tot), 256, 0, st>>>(pa, pb, Y, tot); isdf_note_launch();
            ISDF_LAUNCH_CHECK();
            return ISDF_OK;
        }
    }
    return zgemm(g, st);
}

// an FP64 product of the fit or the adjoint: on the tensor cores by exact slicing when the
// plan enables it and the scratch holds the slices, else on the FP64 pipe
isdf_status fp64_product(isdf_plan *p, const ZGemm &g, cudaStream_t st)
{
    if (p->use_oz && oz_fits(g, p->oz)) return oz_zgemm(g, p->oz, p->oz_err, st);
    return zgemm(g, st);
}

// grow the slice scratch to hold the adjoint's products over a block of grid rows
// (K = max_rows for M-bar and Phi-bar_mu); a no-op once large enough
isdf_status oz_reserve_adjoint(isdf_plan *p)
{
    const int nm = p->n_mu, n = p->n_phi > p->n_psi ? p->n_phi : p->n_psi;
    const int64_t R = p->max_rows;
    size_t need_a = 0, need_b = 0, need_ma = 0, need_mb = 0;
    const int64_t shapes[4][3] = {{R, nm, nm}, {R, n, nm}, {nm, nm, R}, {nm, n, R}};
    for (const auto &sh : shapes) {
        size_t ha, hb, ra, rb;
        oz_sizes((int)sh[0], (int)sh[1], (int)sh[2], 1, &ha, &hb, &ra, &rb);
        need_a = ha > need_a ? ha : need_a;
        need_b = hb > need_b ? hb : need_b;
        need_ma = ra > need_ma ? ra : need_ma;
        need_mb = rb > need_mb ? rb : need_mb;
    }
    auto grow = [](auto **buf, size_t &cap, size_t need) -> isdf_status {
        if (cap >= need) return ISDF_OK;
        if (*buf) cudaFree(*buf);
        *buf = nullptr;
        cap = 0;
        ISDF_CUDA_TRY(cudaMalloc((void **)buf, sizeof(**buf) * need));
        cap = need;
        return ISDF_OK;
    };
    ISDF_TRY(grow(&p->oz.sa, p->oz.cap_a, need_a));
    ISDF_TRY(grow(&p->oz.sb, p->oz.cap_b, need_b));
    ISDF_TRY(grow(&p->oz.ma, p->oz.cap_ma, need_ma));
    ISDF_TRY(grow(&p->oz.mb, p->oz.cap_mb, need_mb));
    return ISDF_OK;
}

// a7-a9 for the current orbitals and interpolation points (no allocation)
isdf_status plan_compute(isdf_plan *p, const int64_t *idx, cudaStream_t st)
{
    const int n_mu = p->n_mu, n_phi = p->n_phi, n_psi = p->n_psi;
    const size_t nn = (size_t)n_mu * n_mu;
    ISDF_CUDA_TRY(cudaMemsetAsync(p->status, 0, sizeof(DeviceStatus), st));
    if (p->oz_err) ISDF_CUDA_TRY(cudaMemsetAsync(p->oz_err, 0, sizeof(int), st));
    ISDF_CUDA_TRY(cudaMemcpyAsync(p->idx, idx, sizeof(int64_t) * n_mu, cudaMemcpyDeviceToDevice, st));
    ISDF_CUDA_TRY(cudaMemsetAsync(p->Mbar, 0, sizeof(double2) * nn, st));
    ISDF_CUDA_TRY(cudaMemsetAsync(p->gphi_mu, 0, sizeof(double2) * n_mu * n_phi, st));
    ISDF_CUDA_TRY(cudaMemsetAsync(p->gpsi_mu, 0, sizeof(double2) * n_mu * n_psi, st));
    // the orbitals' FP16 operands (mixed mode) do not depend on the points: prepared on a
    // third stream while this one runs the FP64 update
    const bool fork_aux = p->mode == ISDF_MIXED && p->aux;
    StreamJoin aux_join;   // joins the aux stream back on any early return below
    if (fork_aux) {
        ISDF_CUDA_TRY(cudaEventRecord(p->ev_aux_fork, st));
        ISDF_CUDA_TRY(cudaStreamWaitEvent(p->aux, p->ev_aux_fork, 0));
        aux_join.arm(st, p->aux, p->ev_aux_join);
        ISDF_TRY(mixed_prepare_orbitals(p, p->aux));
    }
    // a7: Phi_mu = Phi[idx], Psi_mu = Psi[idx]  (Eq. Cmu)
    timer_start(p, 2, st);
    gather_rows<<<grid_for((int64_t)n_mu * n_phi), 256, 0, st>>>(p->phi, p->ld_phi, p->dtype, n_phi, p->idx, n_mu,
                                                                 p->n_r, p->phi_mu, p->status); isdf_note_launch();
    gather_rows<<<grid_for((int64_t)n_mu * n_psi), 256, 0, st>>>(p->psi, p->ld_psi, p->dtype, n_psi, p->idx, n_mu,
                                                                 p->n_r, p->psi_mu, p->status); isdf_note_launch();
    ISDF_LAUNCH_CHECK();
    // a8: M = (Phi_mu Phi_mu^H) o conj(Psi_mu Psi_mu^H), FP64, lower tiles then mirrored
    ZGemm g{};
    g.M = n_mu;
    g.N = n_mu;
    g.K = n_phi;
    g.dual = 1;
    g.A1 = opnd(p->phi_mu, n_phi, 1, 0, ZG_C128);
    g.B1 = opnd(p->phi_mu, 1, n_phi, 1, ZG_C128);
    g.A2 = opnd(p->psi_mu, n_psi, 1, 0, ZG_C128);
    g.B2 = opnd(p->psi_mu, 1, n_psi, 1, ZG_C128);
    g.C = p->M;
    g.scm = n_mu;
    g.scn = 1;
    g.ctype = ZG_C128;
    g.C1 = p->Amu;
    g.C2 = p->Bmu;
    g.lower_only = 1;
    g.splits = 1;
    ZGemm ga = gemm1(n_mu, n_mu, n_phi, g.A1, g.B1, p->Amu, n_mu, ZG_C128, 1.0, 0);
    ZGemm gb = gemm1(n_mu, n_mu, n_psi, g.A2, g.B2, p->Bmu, n_mu, ZG_C128, 1.0, 0);
    ga.lower_only = gb.lower_only = 1;
    if (p->use_oz && (int64_t)n_mu * n_mu >= (int64_t)256 * 256 && oz_fits(ga, p->oz) && oz_fits(gb, p->oz)) {
        // the two Gram products on the tensor cores (exact slicing), then the Hadamard product
        ISDF_TRY(oz_zgemm(ga, p->oz, p->oz_err, st));
        ISDF_TRY(oz_zgemm(gb, p->oz, p->oz_err, st));
        hadamard_lower<<<grid_for(nn), 256, 0, st>>>(p->Amu, p->Bmu, p->M, n_mu); isdf_note_launch();
        ISDF_LAUNCH_CHECK();
    } else {
        ISDF_TRY(zgemm_auto(g, nullptr, 0, st));
    }
    for (double2 *m : {p->M, p->Amu, p->Bmu}) ISDF_TRY(hermitian_mirror(m, n_mu, n_mu, st));
    timer_stop(p, 2, st, n_mu);
    // a9: M = L L^H, L^-1, M^-1 (FP64)
    ISDF_CUDA_TRY(cudaMemcpyAsync(p->L, p->M, sizeof(double2) * nn, cudaMemcpyDeviceToDevice, st));
    ISDF_TRY(cholesky_inverse(p->M, p->L, p->Linv, p->W, p->tmp, n_mu, p->partial, p->partial_elems, p->status, st,
                              p));
    if (p->mode == ISDF_MIXED) {
        if (fork_aux)
            ISDF_CUDA_TRY(aux_join.join());
        else
            ISDF_TRY(mixed_prepare_orbitals(p, st));
        timer_start(p, 6, st);
        ISDF_TRY(mixed_prepare(p, st));
        timer_stop(p, 6, st, p->n_r);
    }
    return ISDF_OK;
}

}  // namespace

extern "C" isdf_status isdf_plan_create(isdf_plan **plan, const void *phi, int64_t ld_phi, const void *psi,
                                        int64_t ld_psi, int64_t n_r, int32_t n_phi, int32_t n_psi, int32_t dtype,
                                        const int64_t *idx, int32_t n_mu, int32_t mode, int64_t max_rows,
                                        void *stream)
{
    if (!plan) return ISDF_ERR_INVALID_ARG;
    *plan = nullptr;
    if (!phi || !psi || !idx || n_r < 1 || n_phi < 1 || n_psi < 1 || ld_phi < n_phi || ld_psi < n_psi)
        return ISDF_ERR_INVALID_ARG;
    if (dtype != ISDF_C128 && dtype != ISDF_C64) return ISDF_ERR_INVALID_ARG;
    const int32_t mflags = mode & ~0xFF;
    mode &= 0xFF;
    if (mode != ISDF_FP64 && mode != ISDF_MIXED) return ISDF_ERR_INVALID_ARG;
    if (mflags & ~ISDF_PLAN_FP64_SIMT) return ISDF_ERR_INVALID_ARG;
    if (n_mu < 1 || n_mu > n_r || max_rows < 1) return ISDF_ERR_INVALID_ARG;
    if (n_mu > 8192 || n_phi > 4096 || n_psi > 4096) return ISDF_ERR_UNSUPPORTED;
    if (n_phi != n_psi) return ISDF_ERR_UNSUPPORTED;
    const size_t el = dtype == ISDF_C128 ? 16 : 8;
    if (!aligned(phi, el) || !aligned(psi, el)) return ISDF_ERR_INVALID_ARG;
    if (mode == ISDF_MIXED && !mixed_supported(n_phi, n_mu, ld_phi, ld_psi, dtype)) return ISDF_ERR_UNSUPPORTED;
    if (max_rows > n_r) max_rows = n_r;
    if (max_rows > 4 * 1024 * 1024) max_rows = 4 * 1024 * 1024;

    isdf_plan *p = static_cast<isdf_plan *>(calloc(1, sizeof(isdf_plan)));
    if (!p) return ISDF_ERR_CUDA;
    p->phi = phi;
    p->psi = psi;
    p->ld_phi = ld_phi;
    p->ld_psi = ld_psi;
    p->n_r = n_r;
    p->n_phi = n_phi;
    p->n_psi = n_psi;
    p->dtype = dtype;
    p->n_mu = n_mu;
    p->mode = mode;
    p->max_rows = max_rows;
    cudaStream_t st = as_stream(stream);
    p->last_stream = st;
    const size_t nn = (size_t)n_mu * n_mu;
    const size_t blk = (size_t)max_rows * n_mu;
    isdf_status s = ISDF_OK;
#define PLAN_ALLOC(ptr, cnt)                       \
    do {                                           \
        if ((s = alloc(&(ptr), (cnt))) != ISDF_OK) { \
            isdf_plan_destroy(p);                  \
            return s;                              \
        }                                          \
    } while (0)
    PLAN_ALLOC(p->status, 1);
    PLAN_ALLOC(p->idx, (size_t)n_mu);
    PLAN_ALLOC(p->phi_mu, (size_t)n_mu * n_phi);
    PLAN_ALLOC(p->psi_mu, (size_t)n_mu * n_psi);
    PLAN_ALLOC(p->M, nn);
    PLAN_ALLOC(p->Amu, nn);
    PLAN_ALLOC(p->Bmu, nn);
    PLAN_ALLOC(p->L, nn);
    PLAN_ALLOC(p->Linv, nn);
    PLAN_ALLOC(p->W, nn);
    PLAN_ALLOC(p->tmp, nn);
    PLAN_ALLOC(p->tmp2, nn);
    PLAN_ALLOC(p->Mbar, nn);
    PLAN_ALLOC(p->gphi_mu, (size_t)n_mu * n_phi);
    PLAN_ALLOC(p->gpsi_mu, (size_t)n_mu * n_psi);
    PLAN_ALLOC(p->blkY, blk);
    if (mode == ISDF_FP64) {
        PLAN_ALLOC(p->blkT, blk);
    }
    // split-K is used only while tiles * splits < 2 * 304, so 608 tiles of 64 x 64 bound the partials
    p->partial_elems = (size_t)4 * 608 * 64 * 64;
    PLAN_ALLOC(p->partial, p->partial_elems);
    p->use_oz = (mflags & ISDF_PLAN_FP64_SIMT) ? 0 : 1;
    if (p->use_oz) {
        // slice scratch for the largest product: n_mu x n_mu x max(n_mu, n) in the plan update, and
        // in FP64 mode a row block max_rows x n_mu x max(n_mu, n) of the fit (with its two Gram products)
        const int kmax = n_mu > n_phi ? n_mu : n_phi;
        const int64_t mrows = (mode == ISDF_FP64 && max_rows > n_mu) ? max_rows : n_mu;
        size_t ha, hb, ra, rb;
        oz_sizes((int)mrows, n_mu, kmax, 1, &ha, &hb, &ra, &rb);
        if (mode == ISDF_FP64) {
            PLAN_ALLOC(p->blkA, blk);
            PLAN_ALLOC(p->blkB, blk);
        }
        p->oz.cap_a = ha;
        p->oz.cap_b = hb;
        p->oz.cap_ma = ra;
        p->oz.cap_mb = rb;
        PLAN_ALLOC(p->oz.sa, ha);
        PLAN_ALLOC(p->oz.sb, hb);
        PLAN_ALLOC(p->oz.ma, ra);
        PLAN_ALLOC(p->oz.mb, rb);
        // exact group sums of the plan-update products (n_mu x n_mu outputs), up to 1 GB
        const size_t gints = (size_t)7 * n_mu * 2 * (size_t)n_mu;
        if (gints * sizeof(int) <= ((size_t)1 << 30)) {
            PLAN_ALLOC(p->oz.gsum, gints);
            p->oz.cap_g = gints;
        }
        PLAN_ALLOC(p->oz_err, 1);
        if (cudaMemsetAsync(p->oz_err, 0, sizeof(int), st) != cudaSuccess) {
            isdf_plan_destroy(p);
            return ISDF_ERR_CUDA;
        }
    }
#undef PLAN_ALLOC
    if (cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p->aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_aux_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_aux_join, cudaEventDisableTiming) != cudaSuccess) {
        isdf_plan_destroy(p);
        return ISDF_ERR_CUDA;
    }
    if ((s = plan_compute(p, idx, st)) != ISDF_OK) {
        isdf_plan_destroy(p);
        return s;
    }
    *plan = p;
    return ISDF_OK;
}

extern "C" isdf_status isdf_fit_theta(isdf_plan *p, int64_t row_begin, int64_t row_count, void *theta,
                                      int64_t ld_theta, void *stream)
{
    if (!p || row_begin < 0 || row_count < 0 || row_begin + row_count > p->n_r || ld_theta < p->n_mu)
        return ISDF_ERR_INVALID_ARG;
    if (row_count == 0) return ISDF_OK;
    if (!theta || !aligned(theta, p->mode == ISDF_FP64 ? 16 : 8)) return ISDF_ERR_INVALID_ARG;
    cudaStream_t st = as_stream(stream);
    p->last_stream = st;
    if (p->mode == ISDF_MIXED) return mixed_fit(p, row_begin, row_count, theta, ld_theta, st);
    for (int64_t r0 = row_begin; r0 < row_begin + row_count; r0 += p->max_rows) {
        const int rows = (int)((row_begin + row_count - r0) < p->max_rows ? (row_begin + row_count - r0) : p->max_rows);
        // a10: Y_b = (Phi_b Phi_mu^H) o conj(Psi_b Psi_mu^H)
        timer_start(p, 0, st);
        ISDF_TRY(gram_hadamard_fp64(p, r0, rows, p->blkY, nullptr, nullptr, st));
        timer_stop(p, 0, st, rows);
        // a11: Theta_b = Y_b M^-1
        double2 *out = static_cast<double2 *>(theta) + (r0 - row_begin) * ld_theta;
        ZGemm g = gemm1(rows, p->n_mu, p->n_mu, opnd(p->blkY, p->n_mu, 1, 0, ZG_C128),
                        opnd(p->W, p->n_mu, 1, 0, ZG_C128), out, ld_theta, ZG_C128, 1.0, 0);
        timer_start(p, 1, st);
        ISDF_TRY(fp64_product(p, g, st));
        timer_stop(p, 1, st, rows);
    }
    return ISDF_OK;
}

// Staging blocks, copy stream and events of isdf_fit_theta_host, made on its first call.
static isdf_status host_stage_init(isdf_plan *p, size_t es)
{
    if (!p->ev_hjoin) {
        if (!p->hcopy) ISDF_CUDA_TRY(cudaStreamCreateWithFlags(&p->hcopy, cudaStreamNonBlocking));
        if (!p->hcopy2) ISDF_CUDA_TRY(cudaStreamCreateWithFlags(&p->hcopy2, cudaStreamNonBlocking));
        for (int s = 0; s < ISDF_HOST_STAGES; ++s) {
            if (!p->ev_hfit[s]) ISDF_CUDA_TRY(cudaEventCreateWithFlags(&p->ev_hfit[s], cudaEventDisableTiming));
            if (!p->ev_hcopied[s]) ISDF_CUDA_TRY(cudaEventCreateWithFlags(&p->ev_hcopied[s], cudaEventDisableTiming));
            if (!p->ev_hhalf[s]) ISDF_CUDA_TRY(cudaEventCreateWithFlags(&p->ev_hhalf[s], cudaEventDisableTiming));
        }
        if (!p->ev_hjoin2) ISDF_CUDA_TRY(cudaEventCreateWithFlags(&p->ev_hjoin2, cudaEventDisableTiming));
        ISDF_CUDA_TRY(cudaEventCreateWithFlags(&p->ev_hjoin, cudaEventDisableTiming));   // last: marks all made
    }
    for (int s = 0; s < ISDF_HOST_STAGES; ++s)
        if (!p->hstage[s]) ISDF_CUDA_TRY(cudaMalloc(&p->hstage[s], (size_t)p->max_rows * p->n_mu * es));
    return ISDF_OK;
}

// true when [q, q + bytes) starts and ends in page-locked host memory
static bool page_locked(const void *q, size_t bytes)
{
    const char *ends[2] = {static_cast<const char *>(q), static_cast<const char *>(q) + bytes - 1};
    for (const char *e : ends) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, e) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if (a.type != cudaMemoryTypeHost) return false;
    }
    return true;
}

extern "C" isdf_status isdf_fit_theta_host(isdf_plan *p, int64_t row_begin, int64_t row_count, void *theta_host,
                                           int64_t ld_theta_host, void *stream)
{
    if (!p || row_begin < 0 || row_count < 0 || row_begin + row_count > p->n_r || ld_theta_host < p->n_mu)
        return ISDF_ERR_INVALID_ARG;
    if (row_count == 0) return ISDF_OK;
    const size_t es = p->mode == ISDF_FP64 ? 16 : 8;
    const size_t row_bytes = (size_t)p->n_mu * es, pitch = (size_t)ld_theta_host * es;
    if (!theta_host || !aligned(theta_host, es) ||
        !page_locked(theta_host, (size_t)(row_count - 1) * pitch + row_bytes))
        return ISDF_ERR_INVALID_ARG;
    ISDF_TRY(host_stage_init(p, es));
    cudaStream_t st = as_stream(stream);
    p->last_stream = st;
    // every return below leaves the caller's stream waiting for the copies issued so far
    StreamJoin join, join2;
    join.arm(st, p->hcopy, p->ev_hjoin);
    join2.arm(st, p->hcopy2, p->ev_hjoin2);
    char *dst = static_cast<char *>(theta_host);
    for (int64_t i = 0, r0 = row_begin; r0 < row_begin + row_count; ++i, r0 += p->max_rows) {
        const int s = (int)(i % ISDF_HOST_STAGES);
        const int64_t rows = (row_begin + row_count - r0) < p->max_rows ? (row_begin + row_count - r0) : p->max_rows;
        // the copy out of this staging block (block i - ISDF_HOST_STAGES) has finished; earlier calls ended joined
        if (i >= ISDF_HOST_STAGES) ISDF_CUDA_TRY(cudaStreamWaitEvent(st, p->ev_hcopied[s], 0));
        ISDF_TRY(isdf_fit_theta(p, r0, rows, p->hstage[s], p->n_mu, stream));
        ISDF_CUDA_TRY(cudaEventRecord(p->ev_hfit[s], st));
        // the block leaves in two halves on two copy streams (two copy engines when the device has them);
        // the first stream records the block's event once both halves have landed
        const int64_t h0 = (rows + 1) / 2;
        const char *src = static_cast<const char *>(p->hstage[s]);
        char *d = dst + (size_t)(r0 - row_begin) * pitch;
        cudaStream_t cs[2] = {p->hcopy, p->hcopy2};
        for (int k = 0; k < 2; ++k) {
            const int64_t a = k ? h0 : 0, n = k ? rows - h0 : h0;
            ISDF_CUDA_TRY(cudaStreamWaitEvent(cs[k], p->ev_hfit[s], 0));
            if (n == 0) continue;
            if (pitch == row_bytes)
                ISDF_CUDA_TRY(cudaMemcpyAsync(d + (size_t)a * pitch, src + (size_t)a * row_bytes, (size_t)n * row_bytes,
                                              cudaMemcpyDeviceToHost, cs[k]));
            else
                ISDF_CUDA_TRY(cudaMemcpy2DAsync(d + (size_t)a * pitch, pitch, src + (size_t)a * row_bytes, row_bytes,
                                                row_bytes, (size_t)n, cudaMemcpyDeviceToHost, cs[k]));
        }
        ISDF_CUDA_TRY(cudaEventRecord(p->ev_hhalf[s], p->hcopy2));
        ISDF_CUDA_TRY(cudaStreamWaitEvent(p->hcopy, p->ev_hhalf[s], 0));
        ISDF_CUDA_TRY(cudaEventRecord(p->ev_hcopied[s], p->hcopy));
    }
    ISDF_CUDA_TRY(join2.join());
    ISDF_CUDA_TRY(join.join());
    return ISDF_OK;
}

extern "C" isdf_status isdf_fit_error(isdf_plan *p, int64_t row_begin, int64_t row_count, double *sums,
                                      void *stream)
{
    if (!p || !sums || row_begin < 0 || row_count < 0 || row_begin + row_count > p->n_r) return ISDF_ERR_INVALID_ARG;
    if (p->mode != ISDF_FP64) return ISDF_ERR_UNSUPPORTED;
    if (!aligned(sums, 8)) return ISDF_ERR_INVALID_ARG;
    if (row_count == 0) return ISDF_OK;
    cudaStream_t st = as_stream(stream);
    p->last_stream = st;
    const int nm = p->n_mu;
    const size_t es = p->dtype == ISDF_C128 ? 16 : 8;
    if (!p->blkT) ISDF_TRY(alloc(&p->blkT, (size_t)p->max_rows * nm));
    for (int64_t r0 = row_begin; r0 < row_begin + row_count; r0 += p->max_rows) {
        const int rows = (int)((row_begin + row_count - r0) < p->max_rows ? (row_begin + row_count - r0) : p->max_rows);
        ISDF_TRY(gram_hadamard_fp64(p, r0, rows, p->blkY, nullptr, nullptr, st));
        ISDF_TRY(fp64_product(p, gemm1(rows, nm, nm, opnd(p->blkY, nm, 1, 0, ZG_C128), opnd(p->W, nm, 1, 0, ZG_C128),
                                       p->blkT, nm, ZG_C128, 1.0, 0), st));
        const unsigned g = (unsigned)((rows + 7) / 8 < 4096 ? (rows + 7) / 8 : 4096);
        const char *pr = static_cast<const char *>(p->phi) + r0 * p->ld_phi * es;
        const char *qr = static_cast<const char *>(p->psi) + r0 * p->ld_psi * es;
        if (p->dtype == ISDF_C128)
            fit_error_kernel<double2><<<g, 256, 0, st>>>(reinterpret_cast<const double2 *>(pr), p->ld_phi, p->n_phi,
                                                         reinterpret_cast<const double2 *>(qr), p->ld_psi, p->n_psi,
                                                         p->blkY, p->blkT, rows, nm, sums);
        else
            fit_error_kernel<float2><<<g, 256, 0, st>>>(reinterpret_cast<const float2 *>(pr), p->ld_phi, p->n_phi,
                                                        reinterpret_cast<const float2 *>(qr), p->ld_psi, p->n_psi,
                                                        p->blkY, p->blkT, rows, nm, sums);
        isdf_note_launch();
        ISDF_LAUNCH_CHECK();
    }
    return ISDF_OK;
}

extern "C" isdf_status isdf_fit_theta_backward(isdf_plan *p, int64_t row_begin, int64_t row_count,
                                               const void *grad_theta, int64_t ld_grad, const void *K, double dV,
                                               void *grad_phi, int64_t ld_gphi, void *grad_psi, int64_t ld_gpsi,
                                               double *loss, void *stream)
{
    if (!p || row_begin < 0 || row_count < 0 || row_begin + row_count > p->n_r) return ISDF_ERR_INVALID_ARG;
    if (!grad_phi || !grad_psi || ld_gphi < p->n_phi || ld_gpsi < p->n_psi) return ISDF_ERR_INVALID_ARG;
    if (!grad_theta && !K) return ISDF_ERR_INVALID_ARG;
    if (grad_theta && ld_grad < p->n_mu) return ISDF_ERR_INVALID_ARG;
    if (!aligned(grad_phi, 16) || !aligned(grad_psi, 16)) return ISDF_ERR_INVALID_ARG;
    if (row_count == 0) return ISDF_OK;
    cudaStream_t st = as_stream(stream);
    p->last_stream = st;
    if (p->mode == ISDF_MIXED)
        return mixed_backward(p, row_begin, row_count, grad_theta, ld_grad, K, dV, grad_phi, ld_gphi, grad_psi,
                              ld_gpsi, loss, st);
    const int nm = p->n_mu;
    const int t = p->dtype == ISDF_C128 ? ZG_C128 : ZG_C64;
    const size_t es = p->dtype == ISDF_C128 ? 16 : 8;
    if (!p->blkT) ISDF_TRY(alloc(&p->blkT, (size_t)p->max_rows * nm));
    if (!p->blkA) {
        ISDF_TRY(alloc(&p->blkA, (size_t)p->max_rows * nm));
        ISDF_TRY(alloc(&p->blkB, (size_t)p->max_rows * nm));
    }
    if (!p->blkG) ISDF_TRY(alloc(&p->blkG, (size_t)p->max_rows * nm));
    if (p->use_oz) {
        // the slice scratch may be reallocated: nothing queued may still read it
        ISDF_CUDA_TRY(cudaStreamSynchronize(st));
        ISDF_TRY(oz_reserve_adjoint(p));
    }
    for (int64_t r0 = row_begin; r0 < row_begin + row_count; r0 += p->max_rows) {
        const int rows = (int)((row_begin + row_count - r0) < p->max_rows ? (row_begin + row_count - r0) : p->max_rows);
        // recompute A_b, B_b and Y_b = A_b o conj(B_b)
        ISDF_TRY(gram_hadamard_fp64(p, r0, rows, p->blkY, p->blkA, p->blkB, st));
        // Theta_b = Y_b M^-1
        ISDF_TRY(fp64_product(p, gemm1(rows, nm, nm, opnd(p->blkY, nm, 1, 0, ZG_C128),
                                       opnd(p->W, nm, 1, 0, ZG_C128), p->blkT, nm, ZG_C128, 1.0, 0), st));
        // G_b
        const void *G;
        int gtype;
        int64_t ldg;
        if (grad_theta) {
            const size_t ges = p->mode == ISDF_MIXED ? 8 : 16;
            G = static_cast<const char *>(grad_theta) + (r0 - row_begin) * ld_grad * ges;
            gtype = p->mode == ISDF_MIXED ? ZG_C64 : ZG_C128;
            ldg = ld_grad;
        } else {
            // G = 2 dV Theta conj(K)
            ISDF_TRY(fp64_product(p, gemm1(rows, nm, nm, opnd(p->blkT, nm, 1, 0, ZG_C128),
                                           opnd(K, nm, 1, 1, ZG_C128), p->blkG, nm, ZG_C128, 2.0 * dV, 0), st));
            G = p->blkG;
            gtype = ZG_C128;
            ldg = nm;
            if (loss) {
                surrogate_loss_kernel<double2><<<grid_for((int64_t)rows * nm, 2048), 256, 0, st>>>(
                    p->blkT, nm, p->blkG, nm, rows, nm, loss); isdf_note_launch();
                ISDF_LAUNCH_CHECK();
            }
        }
        // Ybar = G M^-1 (into blkY)
        ISDF_TRY(fp64_product(p, gemm1(rows, nm, nm, opnd(G, ldg, 1, 0, gtype), opnd(p->W, nm, 1, 0, ZG_C128),
                                       p->blkY, nm, ZG_C128, 1.0, 0), st));
        // Mbar -= Theta_b^H Ybar
        {
            ZGemm g = gemm1(nm, nm, rows, opnd(p->blkT, 1, nm, 1, ZG_C128), opnd(p->blkY, nm, 1, 0, ZG_C128), p->Mbar,
                            nm, ZG_C128, -1.0, 1);
            g.splits = split_count(nm, nm, rows, p->partial_elems);
            g.partial = p->partial;
            if (p->use_oz && oz_fits(g, p->oz)) {
                g.splits = 1;
                ISDF_TRY(oz_zgemm(g, p->oz, p->oz_err, st));
            } else {
                ISDF_TRY(zgemm(g, st));
            }
        }
        // Abar = Ybar o B, Bbar = conj(Ybar) o A
        hadamard_adjoint<<<grid_for((int64_t)rows * nm), 256, 0, st>>>(p->blkY, p->blkA, p->blkB, (int64_t)rows * nm); isdf_note_launch();
        ISDF_LAUNCH_CHECK();
        // grad_phi[rows] += Abar Phi_mu, grad_psi[rows] += Bbar Psi_mu
        double2 *gp = static_cast<double2 *>(grad_phi) + r0 * ld_gphi;
        double2 *gq = static_cast<double2 *>(grad_psi) + r0 * ld_gpsi;
        ISDF_TRY(fp64_product(p, gemm1(rows, p->n_phi, nm, opnd(p->blkA, nm, 1, 0, ZG_C128),
                                       opnd(p->phi_mu, p->n_phi, 1, 0, ZG_C128), gp, ld_gphi, ZG_C128, 1.0, 1), st));
        ISDF_TRY(fp64_product(p, gemm1(rows, p->n_psi, nm, opnd(p->blkB, nm, 1, 0, ZG_C128),
                                       opnd(p->psi_mu, p->n_psi, 1, 0, ZG_C128), gq, ld_gpsi, ZG_C128, 1.0, 1), st));
        // Phibar_mu += Abar^H Phi_b, Psibar_mu += Bbar^H Psi_b
        {
            ZGemm g = gemm1(nm, p->n_phi, rows, opnd(p->blkA, 1, nm, 1, ZG_C128),
                            opnd(static_cast<const char *>(p->phi) + r0 * p->ld_phi * es, p->ld_phi, 1, 0, t),
                            p->gphi_mu, p->n_phi, ZG_C128, 1.0, 1);
            g.splits = split_count(nm, p->n_phi, rows, p->partial_elems);
            g.partial = p->partial;
            ZGemm h = gemm1(nm, p->n_psi, rows, opnd(p->blkB, 1, nm, 1, ZG_C128),
                            opnd(static_cast<const char *>(p->psi) + r0 * p->ld_psi * es, p->ld_psi, 1, 0, t),
                            p->gpsi_mu, p->n_psi, ZG_C128, 1.0, 1);
            h.splits = split_count(nm, p->n_psi, rows, p->partial_elems);
            h.partial = p->partial;
            for (ZGemm *q : {&g, &h}) {
                if (p->use_oz && oz_fits(*q, p->oz)) {
                    q->splits = 1;
                    ISDF_TRY(oz_zgemm(*q, p->oz, p->oz_err, st));
                } else {
                    ISDF_TRY(zgemm(*q, st));
                }
            }
        }
    }
    return ISDF_OK;
}

isdf_status backward_finalize_common(isdf_plan *p, void *grad_phi, int64_t ld_gphi, void *grad_psi, int64_t ld_gpsi,
                                     cudaStream_t st)
{
    const int nm = p->n_mu;
    const size_t nn = (size_t)nm * nm;
    // X = Abar_mu + Abar_mu^H with Abar_mu = Mbar o B_mu; X2 likewise with Bbar_mu = conj(Mbar) o A_mu
    double2 *X = p->tmp, *X2 = p->tmp2;
    hermitian_parts<<<grid_for((int64_t)nn), 256, 0, st>>>(p->Mbar, p->Amu, p->Bmu, X, X2, nm); isdf_note_launch();
    ISDF_LAUNCH_CHECK();
    ISDF_TRY(zgemm(gemm1(nm, p->n_phi, nm, opnd(X, nm, 1, 0, ZG_C128), opnd(p->phi_mu, p->n_phi, 1, 0, ZG_C128),
                         p->gphi_mu, p->n_phi, ZG_C128, 1.0, 1), st));
    ISDF_TRY(zgemm(gemm1(nm, p->n_psi, nm, opnd(X2, nm, 1, 0, ZG_C128), opnd(p->psi_mu, p->n_psi, 1, 0, ZG_C128),
                         p->gpsi_mu, p->n_psi, ZG_C128, 1.0, 1), st));
    scatter_add_rows<<<grid_for((int64_t)nm * p->n_phi), 256, 0, st>>>(p->gphi_mu, p->n_phi, p->idx, nm,
                                                                       static_cast<double2 *>(grad_phi), ld_gphi); isdf_note_launch();
    scatter_add_rows<<<grid_for((int64_t)nm * p->n_psi), 256, 0, st>>>(p->gpsi_mu, p->n_psi, p->idx, nm,
                                                                       static_cast<double2 *>(grad_psi), ld_gpsi); isdf_note_launch();
    ISDF_LAUNCH_CHECK();
    ISDF_CUDA_TRY(cudaMemsetAsync(p->Mbar, 0, sizeof(double2) * nn, st));
    ISDF_CUDA_TRY(cudaMemsetAsync(p->gphi_mu, 0, sizeof(double2) * nm * p->n_phi, st));
    ISDF_CUDA_TRY(cudaMemsetAsync(p->gpsi_mu, 0, sizeof(double2) * nm * p->n_psi, st));
    return ISDF_OK;
}

extern "C" isdf_status isdf_fit_theta_backward_finalize(isdf_plan *p, void *grad_phi, int64_t ld_gphi, void *grad_psi,
                                                        int64_t ld_gpsi, void *stream)
{
    if (!p || !grad_phi || !grad_psi || ld_gphi < p->n_phi || ld_gpsi < p->n_psi) return ISDF_ERR_INVALID_ARG;
    cudaStream_t st = as_stream(stream);
    p->last_stream = st;
    return backward_finalize_common(p, grad_phi, ld_gphi, grad_psi, ld_gpsi, st);
}

extern "C" isdf_status isdf_plan_update(isdf_plan *p, const int64_t *idx, void *stream)
{
    if (!p || !idx) return ISDF_ERR_INVALID_ARG;
    cudaStream_t st = as_stream(stream);
    p->last_stream = st;
    return plan_compute(p, idx, st);
}

// Under stream capture a plain record only orders work inside the graph; an external
// record node is needed for the event to be timed after each replay.
static void timer_record(cudaEvent_t ev, cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
    else
        cudaEventRecord(ev, st);
}

void timer_start(isdf_plan *p, int kind, cudaStream_t st)
{
    if (!p->timing || p->tused[kind] >= p->tcap) return;
    timer_record(p->tev[kind][2 * p->tused[kind]], st);
}

void timer_stop(isdf_plan *p, int kind, cudaStream_t st, int64_t rows)
{
    if (!p->timing || p->tused[kind] >= p->tcap) return;
    timer_record(p->tev[kind][2 * p->tused[kind] + 1], st);
    p->trows[kind][p->tused[kind]] = rows;
    p->tused[kind] += 1;
}

static void timing_free(isdf_plan *p)
{
    for (int k = 0; k < ISDF_TIMER_KINDS; ++k) {
        if (p->tev[k]) {
            for (int i = 0; i < 2 * p->tcap; ++i) cudaEventDestroy(p->tev[k][i]);
            free(p->tev[k]);
            p->tev[k] = nullptr;
        }
        free(p->trows[k]);
        p->trows[k] = nullptr;
        p->tused[k] = 0;
    }
    p->tcap = 0;
    p->timing = 0;
}

extern "C" isdf_status isdf_plan_enable_timing(isdf_plan *p, int32_t capacity)
{
    if (!p || capacity < 0) return ISDF_ERR_INVALID_ARG;
    if (p->last_stream) cudaStreamSynchronize(p->last_stream);
    timing_free(p);
    if (capacity == 0) return ISDF_OK;
    p->tcap = capacity;
    for (int k = 0; k < ISDF_TIMER_KINDS; ++k) {
        p->tev[k] = static_cast<cudaEvent_t *>(calloc(2 * (size_t)capacity, sizeof(cudaEvent_t)));
        p->trows[k] = static_cast<int64_t *>(calloc((size_t)capacity, sizeof(int64_t)));
        if (!p->tev[k] || !p->trows[k]) return ISDF_ERR_CUDA;
        for (int i = 0; i < 2 * capacity; ++i) ISDF_CUDA_TRY(cudaEventCreate(&p->tev[k][i]));
    }
    p->timing = 1;
    return ISDF_OK;
}

extern "C" isdf_status isdf_plan_kernel_time(isdf_plan *p, int32_t kind, double *total_ms, int64_t *launches,
                                             int64_t *rows)
{
    if (!p || kind < 0 || kind >= ISDF_TIMER_KINDS || !total_ms || !launches || !rows) return ISDF_ERR_INVALID_ARG;
    *total_ms = 0.0;
    *launches = 0;
    *rows = 0;
    if (!p->timing) return ISDF_OK;
    for (int i = 0; i < p->tused[kind]; ++i) {
        float ms = 0.f;
        ISDF_CUDA_TRY(cudaEventSynchronize(p->tev[kind][2 * i + 1]));
        ISDF_CUDA_TRY(cudaEventElapsedTime(&ms, p->tev[kind][2 * i], p->tev[kind][2 * i + 1]));
        *total_ms += ms;
        *rows += p->trows[kind][i];
    }
    *launches = p->tused[kind];
    p->tused[kind] = 0;
    return ISDF_OK;
}

extern "C" isdf_status isdf_plan_status(isdf_plan *p, int32_t *detail)
{
    if (!p) return ISDF_ERR_INVALID_ARG;
    ISDF_CUDA_TRY(cudaStreamSynchronize(p->last_stream));
    DeviceStatus h{0, 0};
    ISDF_CUDA_TRY(cudaMemcpy(&h, p->status, sizeof(h), cudaMemcpyDeviceToHost));
    if (detail) *detail = h.detail;
    if (h.code == 0) {
        int32_t m = 0;
        ISDF_TRY(mixed_status(p, &m));
        if (!m && p->oz_err) {
            int e = 0;
            ISDF_CUDA_TRY(cudaMemcpy(&e, p->oz_err, sizeof(int), cudaMemcpyDeviceToHost));
            if (e) m = e == 2 ? ISDF_ERR_NONFINITE : ISDF_ERR_TIMEOUT;
        }
        if (m && detail) *detail = -1;
        return (isdf_status)m;
    }
    return (isdf_status)h.code;
}

extern "C" isdf_status isdf_plan_set_wait_budget(isdf_plan *p, int64_t cycles)
{
    if (!p) return ISDF_ERR_INVALID_ARG;
    p->wait_budget = (long long)cycles;
    p->oz.wait_budget = p->wait_budget;
    return ISDF_OK;
}

extern "C" isdf_status isdf_plan_copy_matrix(const isdf_plan *p, int32_t which, void *dst, void *stream)
{
    if (!p || !dst) return ISDF_ERR_INVALID_ARG;
    const void *src = nullptr;
    size_t count = (size_t)p->n_mu * p->n_mu;
    switch (which) {
    case 0: src = p->M; break;
    case 1: src = p->L; break;
    case 2: src = p->W; break;
    case 3: src = p->phi_mu; count = (size_t)p->n_mu * p->n_phi; break;
    case 4: src = p->psi_mu; count = (size_t)p->n_mu * p->n_psi; break;
    default: return ISDF_ERR_INVALID_ARG;
    }
    ISDF_CUDA_TRY(cudaMemcpyAsync(dst, src, sizeof(double2) * count, cudaMemcpyDeviceToDevice, as_stream(stream)));
    return ISDF_OK;
}

extern "C" void isdf_plan_destroy(isdf_plan *p)
{
    if (!p) return;
    if (p->last_stream) cudaStreamSynchronize(p->last_stream);
    void *bufs[] = {p->status, p->idx, p->phi_mu, p->psi_mu, p->M, p->Amu, p->Bmu, p->L, p->Linv, p->W, p->tmp, p->tmp2,
                    p->Mbar, p->gphi_mu, p->gpsi_mu, p->blkY, p->blkT, p->blkA, p->blkB, p->blkG, p->partial,
                    p->oz.sa, p->oz.sb, p->oz.ma, p->oz.mb, p->oz.gsum, p->oz_err};
    for (void *b : bufs)
        if (b) cudaFree(b);
    mixed_release(p);
    timing_free(p);
    if (p->side) {
        cudaStreamSynchronize(p->side);
        cudaStreamDestroy(p->side);
    }
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_join) cudaEventDestroy(p->ev_join);
    if (p->aux) {
        cudaStreamSynchronize(p->aux);
        cudaStreamDestroy(p->aux);
    }
    if (p->ev_aux_fork) cudaEventDestroy(p->ev_aux_fork);
    if (p->ev_aux_join) cudaEventDestroy(p->ev_aux_join);
    for (cudaStream_t c : {p->hcopy, p->hcopy2})
        if (c) {
            cudaStreamSynchronize(c);
            cudaStreamDestroy(c);
        }
    for (int s = 0; s < ISDF_HOST_STAGES; ++s) {
        if (p->hstage[s]) cudaFree(p->hstage[s]);
        if (p->ev_hfit[s]) cudaEventDestroy(p->ev_hfit[s]);
        if (p->ev_hcopied[s]) cudaEventDestroy(p->ev_hcopied[s]);
        if (p->ev_hhalf[s]) cudaEventDestroy(p->ev_hhalf[s]);
    }
    if (p->ev_hjoin) cudaEventDestroy(p->ev_hjoin);
    if (p->ev_hjoin2) cudaEventDestroy(p->ev_hjoin2);
    free(p);
}
