// FP64 blocked Cholesky of M = C C^H (the paper solves its least-squares
// normal equations with a linear solver, Sec. 2.4), the inverse of the
// Cholesky factor and M^-1 = L^-H L^-1.
//
// Right-looking Cholesky with 16-wide panels: one CTA factors the diagonal
// block in shared memory; the panel below, L21 = A21 L11^-H, is a forward
// substitution with L11 (one warp per row); the trailing lower triangle is
// updated by A22 -= L21 L21^H. The diagonal blocks are then inverted together,
// and L^-1 is assembled bottom-up from them, one batched launch per level:
// inv([[A, 0], [B, C]]) = [[A^-1, 0], [-C^-1 B A^-1, C^-1]].
// Above 512 rows (with the tensor-core FP64 products enabled) the matrix is
// split in halves recursively: the factor and the inverse of the leading half
// give L21 = A21 L11^-H as one product, the Schur complement A22 - L21 L21^H is
// one more, and the inverse's off-diagonal block two more, so that most flops
// run as large exact-slicing products instead of 16-wide FP64 steps.
#include "chol.cuh"
#include "plan.cuh"
#include "zgemm.cuh"
#include "ozaki.cuh"

namespace {

constexpr int NB = 16;    // diagonal block edge (short per-block FP64 chains on the critical path)
constexpr int EW = 256;   // element threads of the diagonal-block kernel (2 warps per SMSP hide FP64 latency)
constexpr int DT = EW + 32;   // plus one pivot warp
constexpr int MAXE = (NB * (NB + 1) / 2 + EW - 1) / EW;   // elements per thread and step

// 1/d for a positive normal d: a float seed (integer conversion, rcp.approx) refined by
// two Newton-Raphson steps r <- r + r (1 - d r), each doubling the correct bits
// (22 -> 44 -> 88), i.e. a result within about one ulp in four dependent FMAs.
__device__ __forceinline__ double recip_pos(double d)
{
    const int e = (int)((__double_as_longlong(d) >> 52) & 0x7FF) - 1023;
    if (e < -120 || e > 120) return 1.0 / d;
    float f;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(f) : "f"(d2f_int(d)));
    double r = f2d_int(f);
    double t = fma(-d, r, 1.0);
    r = fma(r, t, r);
    t = fma(-d, r, 1.0);
    return fma(r, t, r);
}

// Factor the nb x nb diagonal block at (k, k) of A (lower triangle used) and
// write L_kk back (upper part zeroed). A pivot not above 1e-13 of M's original
// diagonal entry (M0) is reported.
//
// GB300 issues FP64 at a low rate per SM, so on this one-CTA critical path
// the FP64 instruction count and its dependency chains set the time. The
// block is factored as L^ D L^H by elimination, one barrier per pivot: step j
// subtracts m_i conj(A_cj) from A_ic (j < c <= i), m_i = A_ij / d_j. The
// active entries of a step are numbered contiguously and dealt to 256
// threads, each loading all of its (up to 2) entries before computing them, so
// that their FP64 chains overlap and warps run full. A ninth warp meanwhile
// updates the next pivot and forms 1/d_{j+1}. Afterwards L = (eliminated
// columns) D^-1/2. The inverse of L_kk is not on this critical path: the
// panel is a forward substitution with L_kk (panel_solve) and the inverses of
// all diagonal blocks are formed together after the factorisation (inv_diag).
// The elimination of an nb x nb block held in shared memory (lower triangle of T; d0s its original diagonal
// entries of M), by every thread of a DT-thread CTA. Afterwards T's columns hold the eliminated values with
// d_j on the diagonal. Returns false (status set) at a pivot not above 1e-13 of d0 or not finite.
__device__ bool factor_block(double2 (*T)[NB + 1], const double *d0s, double *rpiv, int *bad, int k, int nb,
                             DeviceStatus *st)
{
    const int tid = threadIdx.x;
    if (tid == 0) {
        const double d = T[0][0].x;
        bad[0] = (!(d > 1e-13 * d0s[0]) || isinf(d)) ? 1 : 0;
        rpiv[0] = recip_pos(d);
    }
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        const int b = bad[j & 1];   // uniform: written before the last barrier, not rewritten until the next
        if (b) {
            if (tid == 0) set_status(st, isnan(T[b - 1][b - 1].x) ? ISDF_ERR_NONFINITE : ISDF_ERR_NOT_HPD, k + b - 1);
            return false;
        }
        const double r = rpiv[j];
        const int rows = nb - 1 - j;               // i = j+1 .. nb-1
        const int nT = rows * (rows + 1) / 2;      // j < c <= i; entry 0 is the next pivot (j+1, j+1)
        if (tid < EW) {
            int ii[MAXE], cc[MAXE];
            bool on[MAXE];
            double2 av[MAXE], bv[MAXE], tv[MAXE];
#pragma unroll
            for (int q = 0; q < MAXE; ++q) {
                const int e = 1 + tid + q * EW;
                on[q] = e < nT;
                int i = 0, c = 0;
                if (on[q]) {
                    // counted from the last column backwards: column nb-1-p holds p+1 entries
                    const int qq = nT - 1 - e;
                    int p = (int)((sqrtf(8.f * (float)qq + 1.f) - 1.f) * 0.5f);
                    if ((p + 1) * (p + 2) / 2 <= qq) ++p;
                    if (p * (p + 1) / 2 > qq) --p;
                    c = nb - 1 - p;
                    i = nb - 1 - (qq - p * (p + 1) / 2);
                    const double2 bb = T[c][j];
                    bv[q] = make_double2(bb.x, -bb.y);
                    tv[q] = T[i][c];
                    av[q] = T[i][j];
                }
                ii[q] = i;
                cc[q] = c;
            }
#pragma unroll
            for (int q = 0; q < MAXE; ++q) {
                if (on[q]) {   // t -= m conj(b), m = a / d_j
                    const double mx = av[q].x * r, my = av[q].y * r;
                    tv[q].x = fma(-mx, bv[q].x, fma(my, bv[q].y, tv[q].x));
                    tv[q].y = fma(-mx, bv[q].y, fma(-my, bv[q].x, tv[q].y));
                }
            }
#pragma unroll
            for (int q = 0; q < MAXE; ++q)
                if (on[q]) T[ii[q]][cc[q]] = tv[q];
        } else if (tid == EW && nT > 0) {   // the next pivot: A_{j+1,j+1} -= |A_{j+1,j}|^2 / d_j
            const double2 a = T[j + 1][j];
            const double d = fma(-fma(a.x, a.x, a.y * a.y), r, T[j + 1][j + 1].x);
            T[j + 1][j + 1] = make_double2(d, 0.0);
            bad[(j + 1) & 1] = (!(d > 1e-13 * d0s[j + 1]) || isinf(d)) ? j + 2 : 0;
            rpiv[j + 1] = recip_pos(d);
        }
        __syncthreads();
    }
    return true;
}

__global__ void __launch_bounds__(DT) potrf_diag(double2 *A, int64_t lda, const double2 *M0, int k, int nb,
                                                DeviceStatus *st)
{
    __shared__ double2 T[NB][NB + 1];
    __shared__ double d0s[NB];     // original diagonal entries of M
    __shared__ double rpiv[NB];    // 1 / d_j
    __shared__ double rs[NB];      // 1 / sqrt(d_j)
    __shared__ int bad[2];         // failing pivot + 1, or 0: written in step j - 1 into slot j & 1,
                                   // read at the top of step j (two slots keep the read race-free)
    if (st->code != 0) return;
    const int tid = threadIdx.x;
    for (int e = tid; e < NB * NB; e += DT) {
        const int i = e / NB, j = e % NB;
        T[i][j] = (i < nb && j <= i) ? A[(int64_t)(k + i) * lda + (k + j)] : make_double2(0.0, 0.0);
    }
    if (tid < nb) d0s[tid] = M0[(int64_t)(k + tid) * lda + (k + tid)].x;
    __syncthreads();
    if (!factor_block(T, d0s, rpiv, bad, k, nb, st)) return;
    if (tid < nb) rs[tid] = 1.0 / sqrt(T[tid][tid].x);
    __syncthreads();
    for (int e = tid; e < nb * nb; e += DT) {
        const int i = e / nb, j = e % nb;
        double2 l = make_double2(0.0, 0.0);
        if (j < i) l = make_double2(T[i][j].x * rs[j], T[i][j].y * rs[j]);
        else if (j == i) l = make_double2(T[i][i].x * rs[i], 0.0);   // sqrt(d_i)
        A[(int64_t)(k + i) * lda + (k + j)] = l;
    }
}

// Panel below block k in place: row x of L21 solves x L_kk^H = a (the row of A21),
// x_c = (a_c - sum_{l<c} x_l conj(L_cl)) / L_cc, one warp per row, lane c holding column c.
constexpr int PW = 8;   // rows (warps) per CTA
__global__ void __launch_bounds__(32 * PW) panel_solve(double2 *L, int64_t ld, int k, int nb, int rows,
                                                       const DeviceStatus *st)
{
    __shared__ double2 Lk[NB][NB + 1];
    __shared__ double rd[NB];
    if (st->code != 0) return;
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int i = e / NB, j = e % NB;
        Lk[i][j] = (i < nb && j <= i) ? L[(int64_t)(k + i) * ld + (k + j)] : make_double2(0.0, 0.0);
    }
    if (threadIdx.x < nb) rd[threadIdx.x] = 1.0 / L[(int64_t)(k + threadIdx.x) * ld + (k + threadIdx.x)].x;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = blockIdx.x * PW + warp; r < rows; r += gridDim.x * PW) {
        double2 *row = L + (int64_t)(k + nb + r) * ld + k;
        double2 acc = lane < nb ? row[lane] : make_double2(0.0, 0.0);
        double2 x = make_double2(0.0, 0.0);
        for (int s = 0; s < nb; ++s) {
            double2 xs = make_double2(acc.x * rd[s], acc.y * rd[s]);
            xs.x = __shfl_sync(0xffffffffu, xs.x, s);
            xs.y = __shfl_sync(0xffffffffu, xs.y, s);
            if (lane == s) x = xs;
            if (lane > s && lane < nb) {   // acc -= x_s conj(L_cs)
                const double2 b = Lk[lane][s];
                acc.x = fma(-xs.x, b.x, fma(-xs.y, b.y, acc.x));
                acc.y = fma(-xs.y, b.x, fma(xs.x, b.y, acc.y));
            }
        }
        if (lane < nb) row[lane] = x;
    }
}

// One look-ahead step in a single launch. With block column k final and the next block column at
// k1 = k + NB (nb1 wide, `rows` rows below its diagonal block):
//   D   = A[k1:k1+nb1, k1:k1+nb1] - P P^H,  P = L[k1:k1+nb1, k:k+NB]   every CTA, in shared memory
//   L11 = chol(D)                                                      every CTA, the same elimination
//   x_r L11^H = A[r, k1:k1+nb1] - L[r, k:k+NB] P^H                      this CTA's rows r, one warp each
// Every CTA reads the old diagonal block before anyone may overwrite it: the CTA that arrives last on the
// status word's counter (after its reads) writes L11 back and resets the counter; no CTA waits for another.
// This replaces the column update, its split-K reduction, potrf_diag and panel_solve on the critical path.
constexpr int kStepCtas = 152;   // at most one CTA per SM: each repeats the diagonal block's FP64 work
__global__ void __launch_bounds__(DT) chol_step(double2 *A, int64_t lda, const double2 *M0, int k, int k1, int nb1,
                                               int rows, DeviceStatus *st)
{
    __shared__ double2 T[NB][NB + 1];
    __shared__ double2 P[NB][NB + 1];
    __shared__ double d0s[NB], rpiv[NB], rs[NB], rd[NB];
    __shared__ int bad[2];
    __shared__ int last;
    if (st->code != 0) return;
    const int tid = threadIdx.x;
    const double2 zero = make_double2(0.0, 0.0);
    for (int e = tid; e < NB * NB; e += DT) {
        const int i = e / NB, l = e % NB;
        P[i][l] = i < nb1 ? A[(int64_t)(k1 + i) * lda + (k + l)] : zero;
    }
    if (tid < nb1) d0s[tid] = M0[(int64_t)(k1 + tid) * lda + (k1 + tid)].x;
    __syncthreads();
    for (int e = tid; e < NB * NB; e += DT) {   // D = A - P P^H, lower triangle
        const int i = e / NB, j = e % NB;
        double2 t = zero;
        if (i < nb1 && j <= i) {
            t = A[(int64_t)(k1 + i) * lda + (k1 + j)];
#pragma unroll 4
            for (int l = 0; l < NB; ++l) {   // t -= P_il conj(P_jl)
                const double2 a = P[i][l], b = P[j][l];
                t.x = fma(-a.x, b.x, fma(-a.y, b.y, t.x));
                t.y = fma(-a.y, b.x, fma(a.x, b.y, t.y));
            }
        }
        T[i][j] = t;
    }
    __syncthreads();   // this CTA's reads of the old diagonal block are done
    if (tid == 0) {
        __threadfence();
        last = atomicAdd(&st->ticket, 1) == (int)gridDim.x - 1;
    }
    if (!factor_block(T, d0s, rpiv, bad, k1, nb1, st)) return;
    if (tid < nb1) rs[tid] = 1.0 / sqrt(T[tid][tid].x);
    __syncthreads();
    for (int e = tid; e < NB * NB; e += DT) {   // L11 in place: columns scaled by d^-1/2, diagonal sqrt(d)
        const int i = e / NB, j = e % NB;
        if (i < nb1 && j < i) T[i][j] = make_double2(T[i][j].x * rs[j], T[i][j].y * rs[j]);
        else if (i < nb1 && j == i) T[i][i] = make_double2(T[i][i].x * rs[i], 0.0);
        else T[i][j] = zero;
    }
    __syncthreads();
    if (tid < nb1) rd[tid] = 1.0 / T[tid][tid].x;
    if (last) {
        for (int e = tid; e < nb1 * nb1; e += DT) {
            const int i = e / nb1, j = e % nb1;
            A[(int64_t)(k1 + i) * lda + (k1 + j)] = T[i][j];
        }
        if (tid == 0) st->ticket = 0;
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    if (warp >= PW) return;
    for (int r = blockIdx.x * PW + warp; r < rows; r += gridDim.x * PW) {
        double2 *row = A + (int64_t)(k1 + nb1 + r) * lda;
        const double2 lr = lane < NB ? row[k + lane] : zero;
        double2 acc = lane < nb1 ? row[k1 + lane] : zero;
        for (int l = 0; l < NB; ++l) {   // acc -= L[r, k + l] conj(P_cl)
            const double ax = __shfl_sync(0xffffffffu, lr.x, l), ay = __shfl_sync(0xffffffffu, lr.y, l);
            if (lane < nb1) {
                const double2 b = P[lane][l];
                acc.x = fma(-ax, b.x, fma(-ay, b.y, acc.x));
                acc.y = fma(-ay, b.x, fma(ax, b.y, acc.y));
            }
        }
        double2 x = zero;
        for (int c = 0; c < nb1; ++c) {   // forward substitution x L11^H = acc, as panel_solve
            double2 xs = make_double2(acc.x * rd[c], acc.y * rd[c]);
            xs.x = __shfl_sync(0xffffffffu, xs.x, c);
            xs.y = __shfl_sync(0xffffffffu, xs.y, c);
            if (lane == c) x = xs;
            if (lane > c && lane < nb1) {   // acc -= x_c conj(L_lc)
                const double2 b = T[lane][c];
                acc.x = fma(-xs.x, b.x, fma(-xs.y, b.y, acc.x));
                acc.y = fma(-xs.y, b.x, fma(xs.x, b.y, acc.y));
            }
        }
        if (lane < nb1) row[k1 + lane] = x;
    }
}

// Inverses of all diagonal blocks of L (one CTA each): with L^ = L D^-1 (unit
// diagonal), X = L^^-1 by elimination on [L^ | I] (step j: X_ic -= L^_ij X_jc,
// c <= j < i, one barrier per step), then L_kk^-1 = D^-1 X.
__global__ void __launch_bounds__(EW) inv_diag(const double2 *L, int64_t ld, double2 *Linv, int64_t ldi, int n,
                                              const DeviceStatus *st)
{
    __shared__ double2 T[NB][NB + 1];
    __shared__ double2 X[NB][NB + 1];
    __shared__ double rs[NB];   // 1 / L_jj
    if (st->code != 0) return;
    const int k = blockIdx.x * NB, nb = min(NB, n - k), tid = threadIdx.x;
    for (int e = tid; e < NB * NB; e += EW) {
        const int i = e / NB, j = e % NB;
        T[i][j] = (i < nb && j <= i) ? L[(int64_t)(k + i) * ld + (k + j)] : make_double2(0.0, 0.0);
        X[i][j] = make_double2(i == j && i < nb ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    if (tid < nb) rs[tid] = 1.0 / T[tid][tid].x;
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        const int nX = (nb - 1 - j) * (j + 1);   // at most 16 x 16 = 256 = EW
        for (int e = tid; e < nX; e += EW) {
            const int i = j + 1 + e / (j + 1), c = e % (j + 1);
            const double2 a = T[i][j], b = X[j][c];
            const double mx = a.x * rs[j], my = a.y * rs[j];
            double2 x = X[i][c];
            x.x = fma(-mx, b.x, fma(my, b.y, x.x));
            x.y = fma(-mx, b.y, fma(-my, b.x, x.y));
            X[i][c] = x;
        }
        __syncthreads();
    }
    for (int e = tid; e < nb * nb; e += EW) {
        const int i = e / nb, j = e % nb;
        Linv[(int64_t)(k + i) * ldi + (k + j)] =
            j <= i ? make_double2(X[i][j].x * rs[i], X[i][j].y * rs[i]) : make_double2(0.0, 0.0);
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

// FP64 product: on the tensor cores by exact slicing when the plan enables it, the
// shape is large enough to pay for the slicing and the scratch fits; else FP64 GEMM
isdf_status product(const ZGemm &g, double2 *part, size_t part_n, const isdf_plan *tp, cudaStream_t st)
{
    if (tp && tp->use_oz && (int64_t)g.M * g.N * (g.batch > 1 ? g.batch : 1) >= (int64_t)256 * 256 &&
        g.K >= 256 && oz_fits(g, tp->oz))
        return oz_zgemm(g, tp->oz, tp->oz_err, st);
    return zgemm_auto(g, part, part_n, st);
}

// L^-1 from the inverted diagonal blocks (NB wide) already in Linv, merging
// aligned groups of blocks bottom-up: at each level, every pair (left group
// of h rows at o, right group of r <= h rows at o + h) gets
//   tmp = L[o+h:, o:o+h] Linv[o:o+h, o:o+h],  Linv[o+h:, o:o+h] = -Linv[o+h:, o+h:] tmp,
// all full pairs of a level in one batched launch, a ragged last pair apart.
isdf_status tri_inv(const double2 *L, double2 *Linv, double2 *tmp, int64_t ld, int n, double2 *part,
                    size_t part_n, const isdf_plan *tp, cudaStream_t st)
{
    const int nblk = (n + NB - 1) / NB;
    for (int g = 1; g < nblk; g *= 2) {
        const int h = g * NB;
        const int full = n / (2 * h);
        const int64_t step = (int64_t)2 * h * (ld + 1);   // from one pair's diagonal block to the next
        if (full > 0) {
            ZGemm g1 = single(h, h, h, op(L + (int64_t)h * ld, ld, 1, 0), op(Linv, ld, 1, 0), tmp, h, 1.0, 0);
            g1.kmode = ZG_K_FROM_N0;   // Linv lower: k >= n
            g1.batch = full;
            g1.bsa = step;
            g1.bsb = step;
            g1.bsc = (int64_t)h * h;
            ISDF_TRY(product(g1, part, part_n, tp, st));
            ZGemm g2 = single(h, h, h, op(Linv + (int64_t)h * (ld + 1), ld, 1, 0), op(tmp, h, 1, 0),
                              Linv + (int64_t)h * ld, ld, -1.0, 0);
            g2.k_to_m_end = 1;         // Linv lower: k <= m
            g2.batch = full;
            g2.bsa = step;
            g2.bsb = (int64_t)h * h;
            g2.bsc = step;
            ISDF_TRY(product(g2, part, part_n, tp, st));
        }
        const int o = full * 2 * h, r = n - o - h;
        if (r > 0) {
            ZGemm g1 = single(r, h, h, op(L + (int64_t)(o + h) * ld + o, ld, 1, 0),
                              op(Linv + (int64_t)o * ld + o, ld, 1, 0), tmp, h, 1.0, 0);
            g1.kmode = ZG_K_FROM_N0;
            ISDF_TRY(product(g1, part, part_n, tp, st));
            ZGemm g2 = single(r, h, r, op(Linv + (int64_t)(o + h) * ld + (o + h), ld, 1, 0), op(tmp, h, 1, 0),
                              Linv + (int64_t)(o + h) * ld + o, ld, -1.0, 0);
            g2.k_to_m_end = 1;
            ISDF_TRY(product(g2, part, part_n, tp, st));
        }
    }
    return ISDF_OK;
}

// Right-looking blocked factorisation of the diagonal block L[o:o+m, o:o+m] in place (its lower
// triangle holds the matrix; earlier columns are already final). Look-ahead: after the panel of
// block k, a side stream updates block column k+1, factors its diagonal block and forms its panel
// (one chol_step launch) while this stream updates the rest of the block's trailing matrix
// (disjoint columns).
isdf_status chol_blocked(const double2 *M0, double2 *L, int64_t ld, int o, int m, double2 *part, size_t part_n,
                         DeviceStatus *st, cudaStream_t stream, isdf_plan *tp)
{
    const int end = o + m;
    cudaStream_t side = (tp && tp->side) ? tp->side : nullptr;
    {
        const int nb = m < NB ? m : NB;
        potrf_diag<<<1, DT, 0, stream>>>(L, ld, M0, o, nb, st); isdf_note_launch();
        ISDF_LAUNCH_CHECK();
        if (m - nb > 0) {
            const int g = (m - nb + PW - 1) / PW;
            panel_solve<<<g < 4096 ? g : 4096, 32 * PW, 0, stream>>>(L, ld, o, nb, m - nb, st); isdf_note_launch();
            ISDF_LAUNCH_CHECK();
        }
    }
    for (int k = o; k + NB < end; k += NB) {
        const int k1 = k + NB, rest = end - k1;            // next block at k1, rows below block k
        const int nb1 = rest < NB ? rest : NB, rest1 = rest - nb1;
        cudaStream_t s2 = side ? side : stream;
        StreamJoin fork;   // joins the side stream back on any early return below
        if (side) {
            ISDF_CUDA_TRY(cudaEventRecord(tp->ev_fork, stream));
            ISDF_CUDA_TRY(cudaStreamWaitEvent(side, tp->ev_fork, 0));
            fork.arm(stream, side, tp->ev_join);
        }
        // side: block column k1 updated by block column k, its diagonal block factored, its panel formed
        const int g = rest1 > 0 ? ((rest1 + PW - 1) / PW < kStepCtas ? (rest1 + PW - 1) / PW : kStepCtas) : 1;
        chol_step<<<g, DT, 0, s2>>>(L, ld, M0, k, k1, nb1, rest1, st); isdf_note_launch();
        ISDF_LAUNCH_CHECK();
        // this stream: A[k1+nb1:, k1+nb1:] -= L21[nb1:] L21[nb1:]^H (lower tiles)
        if (rest1 > 0) {
            const double2 *l21 = L + (int64_t)(k1 + nb1) * ld + k;
            ZGemm u = single(rest1, rest1, NB, op(l21, ld, 1, 0), op(l21, 1, ld, 1),
                             L + (int64_t)(k1 + nb1) * ld + (k1 + nb1), ld, -1.0, 1);
            u.lower_only = 1;
            ISDF_TRY(zgemm_auto(u, part, part_n, stream));
        }
        ISDF_CUDA_TRY(fork.join());
    }
    return ISDF_OK;
}

// The inverse of the factored diagonal block L[o:o+m, o:o+m] into Linv[o:o+m, o:o+m]: its NB-wide
// diagonal blocks inverted at once, then merged bottom-up (tri_inv).
isdf_status inverse_blocked(const double2 *L, double2 *Linv, double2 *tmp, int64_t ld, int o, int m, double2 *part,
                            size_t part_n, DeviceStatus *st, cudaStream_t stream, const isdf_plan *tp)
{
    const double2 *Lo = L + (int64_t)o * ld + o;
    double2 *Io = Linv + (int64_t)o * ld + o;
    inv_diag<<<(m + NB - 1) / NB, EW, 0, stream>>>(Lo, ld, Io, ld, m, st); isdf_note_launch();
    ISDF_LAUNCH_CHECK();
    return tri_inv(Lo, Io, tmp, ld, m, part, part_n, tp, stream);
}

// Recursive factorisation and inverse of the diagonal block [o, o+m) for large blocks, so that
// most of the (4/3) m^3 flops of each are in large products (on the tensor cores by exact slicing
// when the plan enables it): with the block split at m1,
//   L11 = chol(A11), L11^-1                 (recursively)
//   L21 = A21 L11^-H                        (product; L11^-1 is at hand)
//   A22 <- A22 - L21 L21^H                  (lower tiles)
//   L22 = chol(A22), L22^-1                 (recursively)
//   (L^-1)21 = -L22^-1 (L21 L11^-1)
// Blocks of at most kRecBase rows use the blocked factorisation and inverse above.
constexpr int kRecBase = 512;

isdf_status chol_rec(const double2 *M0, double2 *L, double2 *Linv, double2 *tmp, int64_t ld, int o, int m,
                     double2 *part, size_t part_n, DeviceStatus *st, cudaStream_t stream, isdf_plan *tp)
{
    if (m <= kRecBase) {
        ISDF_TRY(chol_blocked(M0, L, ld, o, m, part, part_n, st, stream, tp));
        return inverse_blocked(L, Linv, tmp, ld, o, m, part, part_n, st, stream, tp);
    }
    const int m1 = ((m / 2 + NB - 1) / NB) * NB, m2 = m - m1;
    ISDF_TRY(chol_rec(M0, L, Linv, tmp, ld, o, m1, part, part_n, st, stream, tp));
    double2 *A21 = L + (int64_t)(o + m1) * ld + o;
    const double2 *I11 = Linv + (int64_t)o * ld + o;
    // L21 = A21 L11^-H into tmp (m2 x m1), then back in place
    ZGemm g = single(m2, m1, m1, op(A21, ld, 1, 0), op(I11, 1, ld, 1), tmp, m1, 1.0, 0);
    ISDF_TRY(product(g, part, part_n, tp, stream));
    ISDF_CUDA_TRY(cudaMemcpy2DAsync(A21, sizeof(double2) * ld, tmp, sizeof(double2) * m1, sizeof(double2) * m1, m2,
                                    cudaMemcpyDeviceToDevice, stream));
    // A22 -= L21 L21^H (lower tiles)
    ZGemm u = single(m2, m2, m1, op(A21, ld, 1, 0), op(A21, 1, ld, 1), L + (int64_t)(o + m1) * (ld + 1), ld, -1.0, 1);
    u.lower_only = 1;
    ISDF_TRY(product(u, part, part_n, tp, stream));
    ISDF_TRY(chol_rec(M0, L, Linv, tmp, ld, o + m1, m2, part, part_n, st, stream, tp));
    // (L^-1)21 = -L22^-1 (L21 L11^-1)
    ZGemm g1 = single(m2, m1, m1, op(A21, ld, 1, 0), op(I11, ld, 1, 0), tmp, m1, 1.0, 0);
    g1.kmode = ZG_K_FROM_N0;   // L11^-1 lower: k >= n
    ISDF_TRY(product(g1, part, part_n, tp, stream));
    ZGemm g2 = single(m2, m1, m2, op(Linv + (int64_t)(o + m1) * (ld + 1), ld, 1, 0), op(tmp, m1, 1, 0),
                      Linv + (int64_t)(o + m1) * ld + o, ld, -1.0, 0);
    g2.k_to_m_end = 1;         // L22^-1 lower: k <= m
    return product(g2, part, part_n, tp, stream);
}

}  // namespace

isdf_status cholesky_inverse(const double2 *M0, double2 *L, double2 *Linv, double2 *W, double2 *tmp, int n,
                             double2 *part, size_t part_n, DeviceStatus *st, cudaStream_t stream,
                             isdf_plan *tp)
{
    const int64_t ld = n;
    if (tp) timer_start(tp, 3, stream);
    ISDF_CUDA_TRY(cudaMemsetAsync(Linv, 0, sizeof(double2) * (size_t)n * n, stream));
    const bool recursive = tp && tp->use_oz && n > kRecBase;
    if (recursive) {
        // factor and inverse together (timed as stage 3; stage 4 records nothing)
        ISDF_TRY(chol_rec(M0, L, Linv, tmp, ld, 0, n, part, part_n, st, stream, tp));
        const int64_t total = (int64_t)n * n;
        const unsigned gr = (unsigned)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
        zero_strict_upper<<<gr, 256, 0, stream>>>(L, n, ld); isdf_note_launch();
        ISDF_LAUNCH_CHECK();
        timer_stop(tp, 3, stream, n);
    } else {
        ISDF_TRY(chol_blocked(M0, L, ld, 0, n, part, part_n, st, stream, tp));
        const int64_t total = (int64_t)n * n;
        const unsigned gr = (unsigned)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
        zero_strict_upper<<<gr, 256, 0, stream>>>(L, n, ld); isdf_note_launch();
        // the inverted diagonal blocks of L, all at once (the first level of L^-1)
        inv_diag<<<(n + NB - 1) / NB, EW, 0, stream>>>(L, ld, Linv, ld, n, st); isdf_note_launch();
        ISDF_LAUNCH_CHECK();
        if (tp) {
            timer_stop(tp, 3, stream, n);
            timer_start(tp, 4, stream);
        }
        ISDF_TRY(tri_inv(L, Linv, tmp, ld, n, part, part_n, tp, stream));
        if (tp) timer_stop(tp, 4, stream, n);
    }
    if (tp) timer_start(tp, 5, stream);
    // W = Linv^H Linv: W_ij = sum_{k >= max(i, j)} conj(Linv_ki) Linv_kj (lower tiles, then mirrored)
    ZGemm w = single(n, n, n, op(Linv, 1, ld, 1), op(Linv, ld, 1, 0), W, ld, 1.0, 0);
    w.kmode = ZG_K_FROM_MAX_MN;
    w.lower_only = 1;
    ISDF_TRY(product(w, part, part_n, tp, stream));
    ISDF_TRY(hermitian_mirror(W, n, ld, stream));
    if (tp) timer_stop(tp, 5, stream, n);
    return ISDF_OK;
}
