// Register-tiled complex FP64 GEMM on the FP64 pipe (GB300 has no FP64
// tensor-core MMA). 64 x 64 complex output tile per CTA, 256 threads, 4 x 4
// complex accumulators per thread, K staged through shared memory 8 complex
// at a time with the conjugation applied on the way in. The dual form keeps
// two products in registers and writes their Hadamard conjugate product,
// Y = (Phi Phi_mu^H) o conj(Psi Psi_mu^H) (Eq. muRownuCol), without storing
// either factor.
#include "zgemm.cuh"

namespace {

constexpr int BK = 8;

template <typename T>
__device__ __forceinline__ double2 ld_c(const void *p, int64_t i)
{
    return cload(static_cast<const T *>(p), i);
}

template <typename TA, typename TB, bool DUAL, int BM, int BN>
__device__ __forceinline__ void load_tiles(const ZGemm &g, int64_t oa, int64_t ob, int m0, int n0, int k0,
                                           int kend, double2 (*As)[BK][BM + 1], double2 (*Bs)[BK][BN + 1])
{
    const int tid = threadIdx.x;
#pragma unroll
    for (int pr = 0; pr < (DUAL ? 2 : 1); ++pr) {
        const ZOperand &A = pr ? g.A2 : g.A1;
        const ZOperand &B = pr ? g.B2 : g.B1;
        const bool a_k_contig = (A.s1 == 1);
        const bool b_n_contig = (B.s1 == 1);
#pragma unroll
        for (int it = 0; it < (BM * BK) / 256; ++it) {
            const int e = it * 256 + tid;
            int mi, ki;
            if (a_k_contig) { mi = e / BK; ki = e % BK; }
            else { mi = e % BM; ki = e / BM; }
            const int m = m0 + mi, k = k0 + ki;
            double2 v = make_double2(0.0, 0.0);
            if (m < g.M && k < kend) {
                v = ld_c<TA>(A.p, oa + (int64_t)m * A.s0 + (int64_t)k * A.s1);
                if (A.conj) v.y = -v.y;
            }
            As[pr][ki][mi] = v;
        }
#pragma unroll
        for (int it = 0; it < (BN * BK) / 256; ++it) {
            const int e = it * 256 + tid;
            int ni, ki;
            if (b_n_contig) { ni = e % BN; ki = e / BN; }
            else { ni = e / BK; ki = e % BK; }
            const int n = n0 + ni, k = k0 + ki;
            double2 v = make_double2(0.0, 0.0);
            if (n < g.N && k < kend) {
                v = ld_c<TB>(B.p, ob + (int64_t)k * B.s0 + (int64_t)n * B.s1);
                if (B.conj) v.y = -v.y;
            }
            Bs[pr][ki][ni] = v;
        }
    }
}

// T x T complex output tile (T = 64 or 32), 256 threads, (T/16) x (T/16) outputs per thread
template <typename TA, typename TB, typename TC, bool DUAL, int T>
__global__ void __launch_bounds__(256) zgemm_kernel(ZGemm g)
{
    constexpr int BM = T, BN = T, R = T / 16;
    __shared__ double2 As[DUAL ? 2 : 1][BK][BM + 1];
    __shared__ double2 Bs[DUAL ? 2 : 1][BK][BN + 1];
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    if (g.lower_only && m0 + BM <= n0) return;
    // blockIdx.z = batch index * splits + K partition
    const int nsplit = g.splits > 1 ? g.splits : 1;
    const int bz = blockIdx.z / nsplit, zs = blockIdx.z % nsplit;
    const int64_t oa = DUAL ? 0 : (int64_t)bz * g.bsa, ob = DUAL ? 0 : (int64_t)bz * g.bsb;
    const int64_t oc = DUAL ? 0 : (int64_t)bz * g.bsc;
    int kb = 0, ke = g.K;
    if (g.kmode == ZG_K_FROM_MAX_MN) kb = (max(m0, n0) / BK) * BK;
    else if (g.kmode == ZG_K_FROM_N0) kb = (n0 / BK) * BK;
    if (g.k_to_m_end) ke = min(ke, m0 + BM);
    if (g.splits > 1) {
        const int span = ke - kb;
        const int chunk = ((span + g.splits - 1) / g.splits + BK - 1) / BK * BK;
        kb = kb + zs * chunk;
        ke = min(ke, kb + chunk);
    }
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double2 acc1[R][R], acc2[DUAL ? R : 1][DUAL ? R : 1];
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc1[i][j] = make_double2(0.0, 0.0);
    if (DUAL) {
#pragma unroll
        for (int i = 0; i < (DUAL ? R : 1); ++i)
#pragma unroll
            for (int j = 0; j < (DUAL ? R : 1); ++j) acc2[i][j] = make_double2(0.0, 0.0);
    }
    for (int k0 = kb; k0 < ke; k0 += BK) {
        load_tiles<TA, TB, DUAL, BM, BN>(g, oa, ob, m0, n0, k0, ke, As, Bs);
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
#pragma unroll
            for (int pr = 0; pr < (DUAL ? 2 : 1); ++pr) {
                double2 a[R], b[R];
#pragma unroll
                for (int i = 0; i < R; ++i) a[i] = As[pr][kk][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < R; ++j) b[j] = Bs[pr][kk][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < R; ++i)
#pragma unroll
                    for (int j = 0; j < R; ++j) {
                        double2 &c = (DUAL && pr) ? acc2[DUAL ? i : 0][DUAL ? j : 0] : acc1[i][j];
                        c.x = fma(a[i].x, b[j].x, c.x);
                        c.x = fma(-a[i].y, b[j].y, c.x);
                        c.y = fma(a[i].x, b[j].y, c.y);
                        c.y = fma(a[i].y, b[j].x, c.y);
                    }
            }
        }
        __syncthreads();
    }
    // epilogue
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int m = m0 + ty + 16 * i;
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int n = n0 + tx + 16 * j;
            if (n >= g.N) continue;
            if (g.splits > 1) {
                g.partial[((int64_t)blockIdx.z * g.M + m) * g.N + n] = acc1[i][j];
                continue;
            }
            const int64_t ci = oc + (int64_t)m * g.scm + (int64_t)n * g.scn;
            double2 v;
            if (DUAL) {
                const double2 p1 = acc1[i][j], p2 = acc2[DUAL ? i : 0][DUAL ? j : 0];
                v = make_double2(p1.x * p2.x + p1.y * p2.y, p1.y * p2.x - p1.x * p2.y);
                if (g.C1) static_cast<double2 *>(g.C1)[ci] = p1;
                if (g.C2) static_cast<double2 *>(g.C2)[ci] = p2;
            } else {
                v = make_double2(g.alpha * acc1[i][j].x, g.alpha * acc1[i][j].y);
                if (g.beta) {
                    const double2 o = cload(static_cast<const TC *>(g.C), ci);
                    v.x += o.x;
                    v.y += o.y;
                }
            }
            cstore(static_cast<TC *>(g.C), ci, v);
        }
    }
}

template <typename TC>
__global__ void splitk_reduce(ZGemm g)
{
    const int64_t mn = (int64_t)g.M * g.N;
    const int nbatch = g.batch > 1 ? g.batch : 1;
    const int64_t total = mn * nbatch;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t bz = e / mn, r = e % mn;
        const int m = (int)(r / g.N), n = (int)(r % g.N);
        if (g.lower_only && (m / g.tile) < (n / g.tile)) continue;
        double2 s = make_double2(0.0, 0.0);
        for (int z = 0; z < g.splits; ++z) {
            const double2 v = g.partial[(bz * g.splits + z) * mn + r];
            s.x += v.x;
            s.y += v.y;
        }
        const int64_t ci = bz * g.bsc + (int64_t)m * g.scm + (int64_t)n * g.scn;
        double2 v = make_double2(g.alpha * s.x, g.alpha * s.y);
        if (g.beta) {
            const double2 o = cload(static_cast<const TC *>(g.C), ci);
            v.x += o.x;
            v.y += o.y;
        }
        cstore(static_cast<TC *>(g.C), ci, v);
    }
}

template <typename TA, typename TB, typename TC, bool DUAL>
isdf_status launch(const ZGemm &g, cudaStream_t st)
{
    const int splits = g.splits > 1 ? g.splits : 1;
    const int nbatch = g.batch > 1 ? g.batch : 1;
    const int T = g.tile == 32 ? 32 : 64;
    dim3 grid((g.N + T - 1) / T, (g.M + T - 1) / T, splits * nbatch);
    if (grid.y > 65535u || (int64_t)splits * nbatch > 65535) return ISDF_ERR_UNSUPPORTED;
    if (T == 32)
        zgemm_kernel<TA, TB, TC, DUAL, 32><<<grid, 256, 0, st>>>(g);
    else
        zgemm_kernel<TA, TB, TC, DUAL, 64><<<grid, 256, 0, st>>>(g);
    isdf_note_launch();
    ISDF_LAUNCH_CHECK();
    if (splits > 1) {
        const int64_t total = (int64_t)g.M * g.N * nbatch;
        const unsigned gr = (unsigned)((total + 255) / 256 < 8192 ? (total + 255) / 256 : 8192);
        splitk_reduce<TC><<<gr, 256, 0, st>>>(g); isdf_note_launch();
        ISDF_LAUNCH_CHECK();
    }
    return ISDF_OK;
}

__global__ void mirror_kernel(double2 *C, int n, int64_t ld)
{
    const int64_t total = (int64_t)n * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        if (j > i) {
            const double2 v = C[(int64_t)j * ld + i];
            C[(int64_t)i * ld + j] = make_double2(v.x, -v.y);
        }
    }
}

}  // namespace

isdf_status zgemm(const ZGemm &g_in, cudaStream_t st)
{
    ZGemm g = g_in;
    if (g.M <= 0 || g.N <= 0) return ISDF_OK;
    if (g.tile != 32) g.tile = 64;
    if (g.splits > 1 && (g.dual || !g.partial)) return ISDF_ERR_INVALID_ARG;
    if (g.batch > 1 && g.dual) return ISDF_ERR_INVALID_ARG;
    const int a = g.A1.type, b = g.B1.type, c = g.ctype;
    if (g.dual) {
        if (g.A2.type != a || g.B2.type != b || c != ZG_C128 || b != ZG_C128) return ISDF_ERR_UNSUPPORTED;
        if (a == ZG_C128) return launch<double2, double2, double2, true>(g, st);
        return launch<float2, double2, double2, true>(g, st);
    }
    if (a == ZG_C128 && b == ZG_C128 && c == ZG_C128) return launch<double2, double2, double2, false>(g, st);
    if (a == ZG_C64 && b == ZG_C128 && c == ZG_C128) return launch<float2, double2, double2, false>(g, st);
    if (a == ZG_C128 && b == ZG_C64 && c == ZG_C128) return launch<double2, float2, double2, false>(g, st);
    if (a == ZG_C128 && b == ZG_C128 && c == ZG_C64) return launch<double2, double2, float2, false>(g, st);
    return ISDF_ERR_UNSUPPORTED;
}

isdf_status zgemm_auto(const ZGemm &g_in, double2 *partial, size_t partial_elems, cudaStream_t st)
{
    ZGemm g = g_in;
    const int sms = 152;
    const size_t nbatch = g.batch > 1 ? (size_t)g.batch : 1;
    auto tiles = [&](int t) {
        const int tm = (g.M + t - 1) / t, tn = (g.N + t - 1) / t;
        return (g.lower_only ? (tm * (tn + 1)) / 2 : tm * tn) * (int)nbatch;
    };
    // tiles with a triangular K range carry up to twice the average work, so they get more
    // splits; the target is ~8 (triangular) or ~4 CTAs of balanced work per SM
    const int target = (g.kmode != ZG_K_ALL || g.k_to_m_end) ? 8 * sms : 4 * sms;
    auto splits_for = [&](int nt) {
        int s = 1;
        if (!g.dual && partial)
            while (s < 16 && nt * s * 2 <= target && g.K / (s * 2) >= 64 &&
                   (size_t)(s * 2) * g.M * g.N * nbatch <= partial_elems)
                s *= 2;
        return s;
    };
    // 64-wide tiles keep the FP64 pipe busier (4 x 4 accumulators a thread); take them whenever
    // they, with split-K, still give two CTAs per SM
    const int s64 = splits_for(tiles(64));
    if (tiles(64) * s64 >= 2 * sms) {
        g.tile = 64;
        g.splits = s64;
    } else {
        g.tile = 32;
        g.splits = splits_for(tiles(32));
    }
    if (g.splits > 1) g.partial = partial;
    return zgemm(g, st);
}

isdf_status hermitian_mirror(double2 *C, int n, int64_t ld, cudaStream_t st)
{
    const int64_t total = (int64_t)n * n;
    const unsigned gr = (unsigned)((total + 255) / 256 < 8192 ? (total + 255) / 256 : 8192);
    mirror_kernel<<<gr, 256, 0, st>>>(C, n, ld); isdf_note_launch();
    ISDF_LAUNCH_CHECK();
    return ISDF_OK;
}
