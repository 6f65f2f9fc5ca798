// Interpolation points by QR with column pivoting (Sec. 2.1, Eq. QRCP), the
// accuracy comparator of the K-means selection. The N_phi N_psi x N_r matrix
// Z^T is replaced by its randomized sketch S^T, S = Z G with the Khatri-Rao
// random columns g_k = a_k (x) conj(b_k):
//     S = (Phi A) o conj(Psi B)      (N_r x p, FP64 products)
// and the first N_mu pivots of S^T's column-pivoted QR are found by greedy
// pivoted Gram-Schmidt: one launch per step normalises the pivot column,
// removes its component from every other column, recomputes their residual
// norms and leaves the next pivot (the largest residual norm) in a key word.
#include "common.cuh"
#include "zgemm.cuh"

namespace {

constexpr int QR_THREADS = 256;
constexpr int QR_IDX_BITS = 22;                       // grid rows < 2^22
constexpr unsigned long long QR_IDX_MASK = (1ull << QR_IDX_BITS) - 1;

// larger norm first, then the lower row: the norm's top 42 bits (sign, exponent, 30 mantissa
// bits of a non-negative double order like the value) above the complemented row index
__device__ __forceinline__ unsigned long long pivot_key(double nrm2, int64_t r)
{
    if (!(nrm2 > 0.0)) return 0ull;
    const unsigned long long b = (unsigned long long)__double_as_longlong(nrm2);
    return (b & ~QR_IDX_MASK) | (QR_IDX_MASK - (unsigned long long)r);
}

__device__ unsigned long long block_max(unsigned long long v)
{
    __shared__ unsigned long long red[QR_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, v, o);
        v = t > v ? t : v;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        v = 0ull;
        for (int i = 0; i < QR_THREADS / 32; ++i) v = red[i] > v ? red[i] : v;
    }
    return v;
}

// S <- S o conj(T) over a block of rows (both rows x p, leading dimension p)
__global__ void hadamard_conj(double2 *S, const double2 *T, int64_t total)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        S[e] = cmulc(S[e], T[e]);
}

// residual norms of every row of S and the first pivot
__global__ void qrcp_init(const double2 *S, int p, int64_t n_r, double *norms, unsigned long long *keys)
{
    const int lane = threadIdx.x & 31;
    unsigned long long best = 0ull;
    for (int64_t r = ((int64_t)blockIdx.x * QR_THREADS + threadIdx.x) / 32; r < n_r;
         r += (int64_t)gridDim.x * (QR_THREADS / 32)) {
        double s = 0.0;
        for (int i = lane; i < p; i += 32) {
            const double2 v = S[r * p + i];
            s += v.x * v.x + v.y * v.y;
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) norms[r] = s;
        const unsigned long long k = pivot_key(s, r);
        best = k > best ? k : best;
    }
    best = block_max(best);
    if (threadIdx.x == 0 && best) atomicMax(keys, best);
}

// step k: pivot j from keys[k % 3]; every other live row r loses (q^H s_r) q, q = s_j / |s_j|;
// the next pivot goes to keys[(k + 1) % 3]; keys[(k + 2) % 3] (read by step k - 1) is cleared
__global__ void __launch_bounds__(QR_THREADS) qrcp_step(double2 *S, int p, int64_t n_r, double *norms,
                                                       unsigned long long *keys, int k, int64_t *idx, double *rdiag,
                                                       int *err)
{
    extern __shared__ double2 q[];
    __shared__ double s_inv;
    const unsigned long long key = keys[k % 3];
    if (key == 0ull) {                    // every column is exhausted or chosen
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            idx[k] = -1;
            rdiag[k] = 0.0;
            atomicExch(err, 1);
        }
        return;
    }
    const int64_t j = (int64_t)(QR_IDX_MASK - (key & QR_IDX_MASK));
    // the pivot row is written by no one in this step, so every block reads the same values
    double s = 0.0;
    for (int i = threadIdx.x; i < p; i += QR_THREADS) {
        const double2 v = S[j * p + i];
        q[i] = v;
        s += v.x * v.x + v.y * v.y;
    }
    __shared__ double red[QR_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < QR_THREADS / 32; ++i) t += red[i];
        s_inv = 1.0 / sqrt(t);
        if (blockIdx.x == 0) {
            idx[k] = j;
            rdiag[k] = sqrt(t);
            keys[(k + 2) % 3] = 0ull;
        }
    }
    __syncthreads();
    const double inv = s_inv;
    for (int i = threadIdx.x; i < p; i += QR_THREADS) {
        q[i].x *= inv;
        q[i].y *= inv;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    unsigned long long best = 0ull;
    for (int64_t r = ((int64_t)blockIdx.x * QR_THREADS + threadIdx.x) / 32; r < n_r;
         r += (int64_t)gridDim.x * (QR_THREADS / 32)) {
        if (r == j) {
            if (lane == 0) norms[r] = -1.0;
            continue;
        }
        if (norms[r] < 0.0) continue;     // chosen earlier
        double2 *row = S + r * p;
        double cx = 0.0, cy = 0.0;        // c = q^H s_r
        for (int i = lane; i < p; i += 32) {
            const double2 a = q[i], v = row[i];
            cx += a.x * v.x + a.y * v.y;
            cy += a.x * v.y - a.y * v.x;
        }
        for (int o = 16; o > 0; o >>= 1) {
            cx += __shfl_xor_sync(0xffffffffu, cx, o);
            cy += __shfl_xor_sync(0xffffffffu, cy, o);
        }
        double nr = 0.0;
        for (int i = lane; i < p; i += 32) {
            const double2 a = q[i];
            double2 v = row[i];
            v.x -= a.x * cx - a.y * cy;
            v.y -= a.x * cy + a.y * cx;
            row[i] = v;
            nr += v.x * v.x + v.y * v.y;
        }
        for (int o = 16; o > 0; o >>= 1) nr += __shfl_xor_sync(0xffffffffu, nr, o);
        if (lane == 0) norms[r] = nr;
        const unsigned long long kk = pivot_key(nr, r);
        best = kk > best ? kk : best;
    }
    best = block_max(best);
    if (threadIdx.x == 0 && best) atomicMax(keys + (k + 1) % 3, best);
}

ZOperand opnd(const void *p, int64_t s0, int64_t s1, int type)
{
    ZOperand o;
    o.p = p;
    o.s0 = s0;
    o.s1 = s1;
    o.conj = 0;
    o.type = type;
    return o;
}

}  // namespace

extern "C" isdf_status isdf_qrcp_points(const void *phi, int64_t ld_phi, int32_t n_phi, const void *psi,
                                        int64_t ld_psi, int32_t n_psi, int64_t n_r, int32_t dtype, const void *A,
                                        const void *B, int32_t p, int32_t n_mu, int64_t *idx, double *rdiag,
                                        void *stream)
{
    if (!phi || !psi || !A || !B || !idx || !rdiag) return ISDF_ERR_INVALID_ARG;
    if (n_phi < 1 || n_psi < 1 || ld_phi < n_phi || ld_psi < n_psi || p < 1 || n_mu < 1 || n_mu > p || n_r < n_mu)
        return ISDF_ERR_INVALID_ARG;
    if (dtype != ISDF_C128 && dtype != ISDF_C64) return ISDF_ERR_INVALID_ARG;
    const size_t el = dtype == ISDF_C128 ? 16 : 8;
    if (!aligned(phi, el) || !aligned(psi, el) || !aligned(A, 16) || !aligned(B, 16) || !aligned(idx, 8) ||
        !aligned(rdiag, 8))
        return ISDF_ERR_INVALID_ARG;
    if (n_r > (int64_t)QR_IDX_MASK || p > 8192) return ISDF_ERR_UNSUPPORTED;
    cudaStream_t st = as_stream(stream);
    const int t = dtype == ISDF_C128 ? ZG_C128 : ZG_C64;
    const int64_t blk = n_r < 65536 ? n_r : 65536;
    double2 *S = nullptr, *T = nullptr;
    double *norms = nullptr;
    unsigned long long *keys = nullptr;
    int *err = nullptr;
    isdf_status s = ISDF_OK;
    auto take = [&](cudaError_t e) {
        if (s == ISDF_OK && e != cudaSuccess) s = ISDF_ERR_CUDA;
    };
    take(cudaMalloc((void **)&S, sizeof(double2) * (size_t)n_r * p));
    if (n_phi != n_psi) take(cudaMalloc((void **)&T, sizeof(double2) * (size_t)blk * p));
    take(cudaMalloc((void **)&norms, sizeof(double) * (size_t)n_r));
    take(cudaMalloc((void **)&keys, 3 * sizeof(unsigned long long)));
    take(cudaMalloc((void **)&err, sizeof(int)));
    if (s == ISDF_OK) {
        take(cudaMemsetAsync(keys, 0, 3 * sizeof(unsigned long long), st));
        take(cudaMemsetAsync(err, 0, sizeof(int), st));
    }
    // the sketch, in row blocks: S_b = (Phi_b A) o conj(Psi_b B)
    for (int64_t r0 = 0; s == ISDF_OK && r0 < n_r; r0 += blk) {
        const int rows = (int)(n_r - r0 < blk ? n_r - r0 : blk);
        const char *pb = static_cast<const char *>(phi) + r0 * ld_phi * el;
        const char *qb = static_cast<const char *>(psi) + r0 * ld_psi * el;
        double2 *Sb = S + r0 * p;
        ZGemm g{};
        g.M = rows;
        g.N = p;
        g.C = Sb;
        g.scm = p;
        g.scn = 1;
        g.ctype = ZG_C128;
        g.alpha = 1.0;
        g.splits = 1;
        if (n_phi == n_psi) {
            g.K = n_phi;
            g.dual = 1;
            g.A1 = opnd(pb, ld_phi, 1, t);
            g.B1 = opnd(A, p, 1, ZG_C128);
            g.A2 = opnd(qb, ld_psi, 1, t);
            g.B2 = opnd(B, p, 1, ZG_C128);
            s = zgemm(g, st);
        } else {
            g.K = n_phi;
            g.A1 = opnd(pb, ld_phi, 1, t);
            g.B1 = opnd(A, p, 1, ZG_C128);
            s = zgemm(g, st);
            if (s == ISDF_OK) {
                g.K = n_psi;
                g.A1 = opnd(qb, ld_psi, 1, t);
                g.B1 = opnd(B, p, 1, ZG_C128);
                g.C = T;
                s = zgemm(g, st);
            }
            if (s == ISDF_OK) {
                const int64_t tot = (int64_t)rows * p;
                hadamard_conj<<<(unsigned)((tot + 255) / 256 < 16384 ? (tot + 255) / 256 : 16384), 256, 0, st>>>(
                    Sb, T, tot);
                isdf_note_launch();
                take(cudaGetLastError());
            }
        }
    }
    const int64_t wblocks = (n_r + QR_THREADS / 32 - 1) / (QR_THREADS / 32);
    const unsigned grid = (unsigned)(wblocks < 152 * 8 ? wblocks : 152 * 8);
    const size_t smem = sizeof(double2) * (size_t)p;
    if (s == ISDF_OK) {
        take(cudaFuncSetAttribute(qrcp_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(double2) * 8192)));
        qrcp_init<<<grid, QR_THREADS, 0, st>>>(S, p, n_r, norms, keys);
        isdf_note_launch();
        take(cudaGetLastError());
    }
    for (int k = 0; s == ISDF_OK && k < n_mu; ++k) {
        qrcp_step<<<grid, QR_THREADS, smem, st>>>(S, p, n_r, norms, keys, k, idx, rdiag, err);
        isdf_note_launch();
        take(cudaGetLastError());
    }
    int h = 0;
    if (s == ISDF_OK) take(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (s == ISDF_OK) take(cudaStreamSynchronize(st));
    else cudaStreamSynchronize(st);
    cudaFree(S);
    cudaFree(T);
    cudaFree(norms);
    cudaFree(keys);
    cudaFree(err);
    if (s == ISDF_OK && h) s = ISDF_ERR_NOT_HPD;   // the sketch's rank is below n_mu
    return s;
}
