// Step 1: the K-means weight function (Sec. 2.2, Eq. weight function 2 for
// SSM and its alpha family, Eq. weight function for PSM).
//
// One thread owns one grid row and sums its moduli in ascending column order
// with explicitly rounded FP64 operations, so the result is bit-identical to
// the plain sequential definition. To keep HBM reads coalesced, a CTA stages
// a 256-row x 128-byte tile through shared memory with 16-byte vector loads
// (rows padded to 144 bytes so that the per-thread row reads are free of bank
// conflicts), then each thread consumes its row of the tile.
#include "common.cuh"

namespace {

constexpr int kRows = 256;          // rows per CTA (one per thread)
constexpr int kPieces = 8;          // 16-byte pieces per row per chunk (128 B)
constexpr int kStride = kPieces + 1;

template <int AK>  // 2: alpha = 2; 1, 3, 4: sqrt/product forms; 0: pow
__device__ __forceinline__ double modulus_pow(double m, double half_alpha)
{
    if (AK == 2) return m;
    if (AK == 1) return __dsqrt_rn(m);
    if (AK == 3) return __dmul_rn(m, __dsqrt_rn(m));
    if (AK == 4) return __dmul_rn(m, m);
    return pow(m, half_alpha);
}

// |z|^2 = re*re + im*im with each operation rounded. For complex64 input the
// products are exact in FP64, so one fused multiply-add gives the same bits.
__device__ __forceinline__ double mod2(double re, double im, bool exact_products)
{
    if (exact_products) return __fma_rn(re, re, __dmul_rn(im, im));
    return __dadd_rn(__dmul_rn(re, re), __dmul_rn(im, im));
}

// Sum of |x_j|^alpha over the n columns of one orbital set for this CTA's rows.
template <typename T, int AK>
__device__ double row_sum(const T *__restrict__ x, int64_t ld, int n, int64_t row0, int64_t n_r,
                          double half_alpha, uint4 (*tile)[kStride])
{
    constexpr int per_piece = 16 / (int)sizeof(T);   // complex elements per 16-byte piece
    constexpr int chunk = kPieces * per_piece;        // columns per chunk
    const int tid = threadIdx.x;
    const bool vec_ok = ((ld * (int64_t)sizeof(T)) % 16 == 0) && ((reinterpret_cast<uintptr_t>(x) & 15) == 0);
    double s = 0.0;
    for (int c0 = 0; c0 < n; c0 += chunk) {
        // cooperative coalesced load of kRows x chunk columns
#pragma unroll
        for (int it = 0; it < kPieces; ++it) {
            const int e = it * kRows + tid;
            const int r = e / kPieces, p = e % kPieces;
            const int64_t row = row0 + r;
            const int col = c0 + p * per_piece;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (row < n_r && col < n) {
                const T *src = x + row * ld + col;
                if (vec_ok && col + per_piece <= n) {
                    v = *reinterpret_cast<const uint4 *>(src);
                } else {
                    T tmp[per_piece];
#pragma unroll
                    for (int q = 0; q < per_piece; ++q) {
                        if (col + q < n) tmp[q] = src[q];
                        else memset(&tmp[q], 0, sizeof(T));
                    }
                    memcpy(&v, tmp, 16);
                }
            }
            tile[r][p] = v;
        }
        __syncthreads();
        const int cols = min(chunk, n - c0);
#pragma unroll 1
        for (int p = 0; p < kPieces; ++p) {
            if (p * per_piece >= cols) break;
            uint4 v = tile[tid][p];
            if (sizeof(T) == 16) {
                double2 z;
                memcpy(&z, &v, 16);
                s = __dadd_rn(s, modulus_pow<AK>(mod2(z.x, z.y, false), half_alpha));
            } else {
                float4 z;
                memcpy(&z, &v, 16);
                s = __dadd_rn(s, modulus_pow<AK>(mod2((double)z.x, (double)z.y, true), half_alpha));
                if (p * per_piece + 1 < cols)
                    s = __dadd_rn(s, modulus_pow<AK>(mod2((double)z.z, (double)z.w, true), half_alpha));
            }
        }
        __syncthreads();
    }
    return s;
}

template <typename T, int AK>
__global__ void __launch_bounds__(kRows) weights_kernel(const T *__restrict__ phi, int64_t ld_phi, int n_phi,
                                                       const T *__restrict__ psi, int64_t ld_psi, int n_psi,
                                                       int64_t n_r, int psm, double half_alpha,
                                                       double *__restrict__ w, int acc)
{
    __shared__ uint4 tile[kRows][kStride];
    const int64_t row0 = (int64_t)blockIdx.x * kRows;
    const double sa = row_sum<T, AK>(phi, ld_phi, n_phi, row0, n_r, half_alpha, tile);
    const double sb = row_sum<T, AK>(psi, ld_psi, n_psi, row0, n_r, half_alpha, tile);
    const int64_t row = row0 + threadIdx.x;
    if (row < n_r) {
        const double v = psm ? __dmul_rn(sa, sb) : __dadd_rn(sa, sb);
        w[row] = acc ? __dadd_rn(w[row], v) : v;   // shared weight of several pairs: one rounding per pair
    }
}

template <typename T>
isdf_status launch_weights(const void *phi, int64_t ld_phi, int n_phi, const void *psi, int64_t ld_psi,
                           int n_psi, int64_t n_r, int psm, double alpha, double *w, int acc, cudaStream_t st)
{
    const unsigned grid = (unsigned)((n_r + kRows - 1) / kRows);
    const T *a = static_cast<const T *>(phi);
    const T *b = static_cast<const T *>(psi);
    const double ha = 0.5 * alpha;
    if (psm || alpha == 2.0)
        weights_kernel<T, 2><<<grid, kRows, 0, st>>>(a, ld_phi, n_phi, b, ld_psi, n_psi, n_r, psm, ha, w, acc);
    else if (alpha == 1.0)
        weights_kernel<T, 1><<<grid, kRows, 0, st>>>(a, ld_phi, n_phi, b, ld_psi, n_psi, n_r, 0, ha, w, acc);
    else if (alpha == 3.0)
        weights_kernel<T, 3><<<grid, kRows, 0, st>>>(a, ld_phi, n_phi, b, ld_psi, n_psi, n_r, 0, ha, w, acc);
    else if (alpha == 4.0)
        weights_kernel<T, 4><<<grid, kRows, 0, st>>>(a, ld_phi, n_phi, b, ld_psi, n_psi, n_r, 0, ha, w, acc);
    else
        weights_kernel<T, 0><<<grid, kRows, 0, st>>>(a, ld_phi, n_phi, b, ld_psi, n_psi, n_r, 0, ha, w, acc);
    isdf_note_launch();
    ISDF_LAUNCH_CHECK();
    return ISDF_OK;
}

}  // namespace

extern "C" isdf_status isdf_weights(const void *phi, int64_t ld_phi, int32_t n_phi, const void *psi,
                                    int64_t ld_psi, int32_t n_psi, int64_t n_r, int32_t dtype, int32_t kind,
                                    double alpha, double *w, void *stream)
{
    if (n_r < 0 || n_phi < 1 || n_psi < 1 || ld_phi < n_phi || ld_psi < n_psi) return ISDF_ERR_INVALID_ARG;
    if (dtype != ISDF_C128 && dtype != ISDF_C64) return ISDF_ERR_INVALID_ARG;
    const int acc = (kind & ISDF_W_ACCUMULATE) ? 1 : 0;
    kind &= ~ISDF_W_ACCUMULATE;
    if (kind != ISDF_W_SSM && kind != ISDF_W_PSM) return ISDF_ERR_INVALID_ARG;
    if (!(alpha > 0.0) || alpha > 1e6) return ISDF_ERR_INVALID_ARG;
    if (n_r == 0) return ISDF_OK;
    if (!phi || !psi || !w) return ISDF_ERR_INVALID_ARG;
    const size_t el = dtype == ISDF_C128 ? 16 : 8;
    if (!aligned(phi, el) || !aligned(psi, el) || !aligned(w, 8)) return ISDF_ERR_INVALID_ARG;
    cudaStream_t st = as_stream(stream);
    if (dtype == ISDF_C128)
        return launch_weights<double2>(phi, ld_phi, n_phi, psi, ld_psi, n_psi, n_r, kind == ISDF_W_PSM, alpha, w, acc,
                                       st);
    return launch_weights<float2>(phi, ld_phi, n_phi, psi, ld_psi, n_psi, n_r, kind == ISDF_W_PSM, alpha, w, acc, st);
}

static unsigned long long g_launches = 0;

void isdf_note_launch() { __atomic_add_fetch(&g_launches, 1ull, __ATOMIC_RELAXED); }

extern "C" unsigned long long isdf_kernel_launches(void) { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

extern "C" const char *isdf_status_string(isdf_status s)
{
    switch (s) {
    case ISDF_OK: return "ok";
    case ISDF_ERR_INVALID_ARG: return "invalid argument";
    case ISDF_ERR_CUDA: return "CUDA runtime error";
    case ISDF_ERR_NOT_HPD: return "C C^H is not Hermitian positive definite";
    case ISDF_ERR_EMPTY_CLUSTER: return "empty K-means cluster";
    case ISDF_ERR_NONFINITE: return "non-finite value";
    case ISDF_ERR_TIMEOUT: return "bounded device wait timed out";
    case ISDF_ERR_WORKSPACE: return "workspace missing or too small";
    case ISDF_ERR_UNSUPPORTED: return "unsupported size";
    }
    return "unknown status";
}
