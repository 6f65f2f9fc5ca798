// FP64 blocked Cholesky of M = C C^H (the paper solves its least-squares
// normal equations with a linear solver, Sec. 2.4), the inverse of the
// Cholesky factor and M^-1 = L^-H L^-1.
//
// Right-looking Cholesky with 32-wide panels: one CTA factors the diagonal
// block in shared memory and also inverts it; the panel below is L21 =
// A21 L11^-H (a GEMM with the inverted diagonal block); the trailing lower
// triangle is updated by A22 -= L21 L21^H. L^-1 is built recursively from the
// inverted diagonal blocks: inv([[A, 0], [B, C]]) = [[A^-1, 0], [-C^-1 B A^-1, C^-1]].
#include "chol.cuh"
#include "plan.cuh"
#include "zgemm.cuh"

namespace {

constexpr int NB = 32;    // diagonal block edge
constexpr int DT = 128;   // threads of the diagonal-block kernel

// Factor the nb x nb diagonal block at (k, k) of A (lower triangle used),
// write L_kk back (upper part zeroed) and L_kk^-1 into Linv at (k, k).
// A pivot not above 1e-13 of M's original diagonal entry (M0) is reported.
//
// Latency matters more than throughput here (one block per launch, on the
// critical path of the factorisation), so each elimination step costs one
// barrier: step j subtracts T[i][j] conj(T[c][j]) / d_j from the trailing
// triangle with the unscaled column j, and the columns are scaled by
// 1/sqrt(d_j) once at the end. The inverse is computed column by column; the
// 4 threads of a column sit in one warp, so it needs no block barrier.
__global__ void __launch_bounds__(DT) potrf_diag(double2 *A, int64_t lda, const double2 *M0, double2 *Linv,
                                                int64_t ldi, int k, int nb, DeviceStatus *st)
{
    __shared__ double2 T[NB][NB + 1];
    __shared__ double2 I[NB][NB + 1];
    __shared__ double d0s[NB];     // original diagonal entries of M
    __shared__ double rdiag[NB];   // 1 / L_jj
    if (st->code != 0) return;
    const int tid = threadIdx.x;
    for (int e = tid; e < NB * NB; e += DT) {
        const int i = e / NB, j = e % NB;
        T[i][j] = (i < nb && j <= i) ? A[(int64_t)(k + i) * lda + (k + j)] : make_double2(0.0, 0.0);
    }
    if (tid < nb) d0s[tid] = M0[(int64_t)(k + tid) * lda + (k + tid)].x;
    __syncthreads();
    // thread t updates row i = t % NB, columns c = j + 1 + slice, step 4
    const int my_row = tid % NB, slice = tid / NB;
    for (int j = 0; j < nb; ++j) {
        const double d = T[j][j].x;
        if (!(d > 1e-13 * d0s[j]) || isinf(d)) {
            if (tid == 0) set_status(st, isnan(d) ? ISDF_ERR_NONFINITE : ISDF_ERR_NOT_HPD, k + j);
            return;   // uniform: every thread read the same pivot
        }
        if (my_row > j && my_row < nb) {
            const double r = 1.0 / d;
            const double2 a = T[my_row][j];
            const double2 ar = make_double2(a.x * r, a.y * r);
            for (int c = j + 1 + slice; c <= my_row; c += DT / NB) {
                const double2 b = T[c][j];
                T[my_row][c].x -= ar.x * b.x + ar.y * b.y;
                T[my_row][c].y -= ar.y * b.x - ar.x * b.y;
            }
        }
        __syncthreads();
    }
    // L_jj = sqrt(d_j), L_ij = T_ij / sqrt(d_j)
    if (tid < nb) {
        const double l = sqrt(T[tid][tid].x);
        rdiag[tid] = 1.0 / l;
        T[tid][tid] = make_double2(l, 0.0);
    }
    __syncthreads();
    for (int e = tid; e < NB * NB; e += DT) {
        const int i = e / NB, j = e % NB;
        if (i < nb && j < i) {
            const double r = rdiag[j];
            T[i][j] = make_double2(T[i][j].x * r, T[i][j].y * r);
        }
    }
    __syncthreads();
    // inverse by forward substitution down each column c:
    // I[i][c] = (delta_ic - sum_{c <= l < i} T[i][l] I[l][c]) / T[i][i]
    {
        const int c = tid >> 2, part = tid & 3;
        for (int i = 0; i < NB; ++i) {
            double2 s = make_double2(0.0, 0.0);
            if (i < nb && c < i)
                for (int l = c + part; l < i; l += 4) {
                    const double2 a = T[i][l], b = I[l][c];
                    s.x += a.x * b.x - a.y * b.y;
                    s.y += a.x * b.y + a.y * b.x;
                }
            s.x += __shfl_xor_sync(0xffffffffu, s.x, 1);
            s.y += __shfl_xor_sync(0xffffffffu, s.y, 1);
            s.x += __shfl_xor_sync(0xffffffffu, s.x, 2);
            s.y += __shfl_xor_sync(0xffffffffu, s.y, 2);
            if (part == 0) {
                double2 v = make_double2(0.0, 0.0);
                if (i < nb && c <= i) {
                    const double r = rdiag[i];
                    v = make_double2(((i == c ? 1.0 : 0.0) - s.x) * r, -s.y * r);
                }
                I[i][c] = v;
            }
            __syncwarp();
        }
    }
    __syncthreads();
    for (int e = tid; e < nb * nb; e += DT) {
        const int i = e / nb, j = e % nb;
        A[(int64_t)(k + i) * lda + (k + j)] = j <= i ? T[i][j] : make_double2(0.0, 0.0);
        Linv[(int64_t)(k + i) * ldi + (k + j)] = j <= i ? I[i][j] : make_double2(0.0, 0.0);
    }
}

__global__ void zero_strict_upper(double2 *A, int n, int64_t lda)
{
    const int64_t total = (int64_t)n * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        if (j > i) A[(int64_t)i * lda + j] = make_double2(0.0, 0.0);
    }
}

ZOperand op(const double2 *p, int64_t s0, int64_t s1, int conj)
{
    ZOperand o;
    o.p = p;
    o.s0 = s0;
    o.s1 = s1;
    o.conj = conj;
    o.type = ZG_C128;
    return o;
}

ZGemm single(int M, int N, int K, ZOperand A, ZOperand B, double2 *C, int64_t ldc, double alpha, int beta)
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
    g.ctype = ZG_C128;
    g.alpha = alpha;
    g.beta = beta;
    g.splits = 1;
    return g;
}

// Linv[o:o+n, o:o+n] = inverse of the lower-triangular L block (its 64-wide
// diagonal blocks are already inverted in Linv).
isdf_status tri_inv(const double2 *L, double2 *Linv, double2 *tmp, int64_t ld, int o, int n, double2 *part,
                    size_t part_n, cudaStream_t st)
{
    if (n <= NB) return ISDF_OK;
    const int h = ((n / 2 + NB - 1) / NB) * NB;
    ISDF_TRY(tri_inv(L, Linv, tmp, ld, o, h, part, part_n, st));
    ISDF_TRY(tri_inv(L, Linv, tmp, ld, o + h, n - h, part, part_n, st));
    // tmp = L[o+h:o+n, o:o+h] * Linv[o:o+h, o:o+h]   (Linv lower: k >= n)
    ZGemm g1 = single(n - h, h, h, op(L + (int64_t)(o + h) * ld + o, ld, 1, 0),
                      op(Linv + (int64_t)o * ld + o, ld, 1, 0), tmp, h, 1.0, 0);
    g1.kmode = ZG_K_FROM_N0;
    ISDF_TRY(zgemm_auto(g1, part, part_n, st));
    // Linv[o+h:o+n, o:o+h] = -Linv[o+h:o+n, o+h:o+n] * tmp   (A lower: k <= m)
    ZGemm g2 = single(n - h, h, n - h, op(Linv + (int64_t)(o + h) * ld + (o + h), ld, 1, 0),
                      op(tmp, h, 1, 0), Linv + (int64_t)(o + h) * ld + o, ld, -1.0, 0);
    g2.k_to_m_end = 1;
    return zgemm_auto(g2, part, part_n, st);
}

}  // namespace

isdf_status cholesky_inverse(const double2 *M0, double2 *L, double2 *Linv, double2 *W, double2 *tmp, int n,
                             double2 *part, size_t part_n, DeviceStatus *st, cudaStream_t stream,
                             isdf_plan *tp)
{
    const int64_t ld = n;
    if (tp) timer_start(tp, 3, stream);
    ISDF_CUDA_TRY(cudaMemsetAsync(Linv, 0, sizeof(double2) * (size_t)n * n, stream));
    for (int k = 0; k < n; k += NB) {
        const int nb = n - k < NB ? n - k : NB;
        potrf_diag<<<1, DT, 0, stream>>>(L, ld, M0, Linv, ld, k, nb, st); isdf_note_launch();
        ISDF_LAUNCH_CHECK();
        const int rest = n - k - nb;
        if (rest <= 0) break;
        // L21 = A21 * Lkk^-H  (in place: one 64-wide CTA column per row block, no split-K)
        ZGemm p = single(rest, nb, nb, op(L + (int64_t)(k + nb) * ld + k, ld, 1, 0),
                         op(Linv + (int64_t)k * ld + k, 1, ld, 1), L + (int64_t)(k + nb) * ld + k, ld, 1.0, 0);
        p.tile = 32;  // N = nb fits one tile column, so the in-place update is race-free
        ISDF_TRY(zgemm(p, stream));
        // A22 -= L21 L21^H (lower tiles)
        ZGemm u = single(rest, rest, nb, op(L + (int64_t)(k + nb) * ld + k, ld, 1, 0),
                         op(L + (int64_t)(k + nb) * ld + k, 1, ld, 1), L + (int64_t)(k + nb) * ld + (k + nb), ld,
                         -1.0, 1);
        u.lower_only = 1;
        ISDF_TRY(zgemm_auto(u, part, part_n, stream));
    }
    {
        const int64_t total = (int64_t)n * n;
        const unsigned gr = (unsigned)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
        zero_strict_upper<<<gr, 256, 0, stream>>>(L, n, ld); isdf_note_launch();
        ISDF_LAUNCH_CHECK();
    }
    if (tp) {
        timer_stop(tp, 3, stream, n);
        timer_start(tp, 4, stream);
    }
    ISDF_TRY(tri_inv(L, Linv, tmp, ld, 0, n, part, part_n, stream));
    if (tp) {
        timer_stop(tp, 4, stream, n);
        timer_start(tp, 5, stream);
    }
    // W = Linv^H Linv: W_ij = sum_{k >= max(i, j)} conj(Linv_ki) Linv_kj (lower tiles, then mirrored)
    ZGemm w = single(n, n, n, op(Linv, 1, ld, 1), op(Linv, ld, 1, 0), W, ld, 1.0, 0);
    w.kmode = ZG_K_FROM_MAX_MN;
    w.lower_only = 1;
    ISDF_TRY(zgemm_auto(w, part, part_n, stream));
    ISDF_TRY(hermitian_mirror(W, n, ld, stream));
    if (tp) timer_stop(tp, 5, stream, n);
    return ISDF_OK;
}
