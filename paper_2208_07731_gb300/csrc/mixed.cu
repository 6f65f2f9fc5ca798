// Tensor-core path of the Theta fit (ISDF_MIXED): the two Gram GEMMs with
// the Hadamard conjugate product fused (Eq. muRownuCol) and the application
// of M^-1 (Eq. theta) on the tcgen05 tensor cores.
//
// Complex GEMMs as real GEMMs without a de-interleave pass: an interleaved
// complex row (re0, im0, re1, im1, ...) is a real row of length 2N, and for a
// complex matrix B the "rotated" real matrix Bh with rows
//     Bh[2v]   = (Re b_v1, Im b_v1, Re b_v2, ...)
//     Bh[2v+1] = (-Im b_v1, Re b_v1, -Im b_v2, ...)
// gives A Bh^T = interleaved (Re, Im) of A B^H. Both operands are K-major.
//
// Split precision: every operand x is scaled by an exact power of two s
// (so |x s| < 2^14) and split into FP16 hi = fp16(x s), lo = fp16(x s - hi);
// A B^T ~ Ahi Bhi^T + Ahi Blo^T + Alo Bhi^T, each product exact in the FP32
// accumulator (11 + 11 significant bits), leaving ~2^-22 relative error.
//
// GEMM kernel (tc_gemm_persist): 128 x 128 output tiles, K in chunks of 64
// FP16 (one 128-byte swizzle row), a 3-stage TMA/mbarrier ring, tcgen05.mma
// into a double-buffered TMEM accumulator and a TMEM epilogue. The Gram
// variant accumulates Phi_b Phi_mu^H and Psi_b Psi_mu^H into two TMEM
// accumulators and writes Y = P^phi o conj(P^psi), already scaled and split,
// as the A operand of the second GEMM Theta_b = Y_b M^-1, whose K loop runs
// in segments summed in registers.
#include <cudaTypedefs.h>

#include "mixed.cuh"
#include "tc.cuh"

namespace {

constexpr int TM = 128, TN = 128, TK = 64;
constexpr int STAGES = 3;
constexpr int TILE_A = TM * TK * 2;
constexpr int TILE_B = TN * TK * 2;
constexpr int STAGE_BYTES = 2 * TILE_A + 2 * TILE_B;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;
constexpr long long WAIT_BUDGET = 200000000LL;
constexpr int kApplySegment = 8;   // K chunks (of 64) per TMEM accumulation segment in the M^-1 GEMM
constexpr int kGramSegment = 8;    // the same for each of the two Gram products  // SM cycles (~0.1 s); normal waits take microseconds

struct MixScales {
    unsigned int maxabs_phi, maxrho_phi, maxabs_psi, maxrho_psi, maxabs_w;  // float bits
    float s_phi, s_psi, s_w, fy, ftheta;
    int err;
    int pad[5];
};

}  // namespace

struct MixedBuffers {
    __half *a1h, *a1l, *a2h, *a2l;   // N_r x 2N split orbitals
    __half *b1h, *b1l, *b2h, *b2l;   // 2 N_mu x 2N rotated Phi_mu, Psi_mu
    __half *bwh, *bwl;               // 2 N_mu x 2 N_mu rotated M^-1
    __half *yh, *yl;                 // max_rows x 2 N_mu split Y block
    MixScales *sc;
    CUtensorMap m_a1h, m_a1l, m_a2h, m_a2l, m_b1h, m_b1l, m_b2h, m_b2l, m_bwh, m_bwl, m_yh, m_yl;
};

namespace {

__device__ __forceinline__ void atomic_max_pos(unsigned int *p, float v) { atomicMax(p, __float_as_uint(v)); }

// max |Re|, |Im| over the matrix and max row density sum_i |x_ri|^2 (FP32 for
// complex64 input, FP64 for complex128; both are bounds used with margins)
template <typename T>
__global__ void absmax_rows(const T *x, int64_t ld, int n, int64_t n_r, unsigned int *maxabs, unsigned int *maxrho)
{
    float ma = 0.f, mr = 0.f;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < n_r; r += nwarps) {
        float rho;
        if (sizeof(T) == 8) {
            const float2 *xr = reinterpret_cast<const float2 *>(x) + r * ld;
            float acc = 0.f;
            for (int i = lane; i < n; i += 32) {
                const float2 v = xr[i];
                ma = fmaxf(ma, fmaxf(fabsf(v.x), fabsf(v.y)));
                acc = fmaf(v.x, v.x, fmaf(v.y, v.y, acc));
            }
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            rho = acc * (1.f + 1e-5f);
        } else {
            double acc = 0.0;
            for (int i = lane; i < n; i += 32) {
                const double2 v = cload(x, r * ld + i);
                ma = fmaxf(ma, (float)fmax(fabs(v.x), fabs(v.y)));
                acc += v.x * v.x + v.y * v.y;
            }
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            rho = (float)acc * (1.f + 1e-6f);
        }
        mr = fmaxf(mr, rho);
    }
    for (int o = 16; o > 0; o >>= 1) {
        ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, o));
        mr = fmaxf(mr, __shfl_xor_sync(0xffffffffu, mr, o));
    }
    if (lane == 0) {
        atomic_max_pos(maxabs, ma * 1.0001f);
        if (maxrho) atomic_max_pos(maxrho, mr);
    }
}

// s = 2^(14 - e) with v < 2^e: |x s| < 2^14 for every |x| <= v
__device__ int scale_exp(float v)
{
    if (!(v > 0.f)) return 0;
    int e;
    frexpf(v * 1.0001f, &e);
    return 14 - e;
}

__global__ void compute_scales(MixScales *sc)
{
    const float ma_phi = __uint_as_float(sc->maxabs_phi), ma_psi = __uint_as_float(sc->maxabs_psi);
    const float mr_phi = __uint_as_float(sc->maxrho_phi), mr_psi = __uint_as_float(sc->maxrho_psi);
    const float ma_w = __uint_as_float(sc->maxabs_w);
    const int e_phi = scale_exp(ma_phi), e_psi = scale_exp(ma_psi), e_w = scale_exp(ma_w);
    // |Y| = |P^phi||P^psi| <= max rho_phi * max rho_psi (Cauchy-Schwarz)
    const int e_y = scale_exp(mr_phi * mr_psi * 1.01f);
    sc->s_phi = ldexpf(1.f, e_phi);
    sc->s_psi = ldexpf(1.f, e_psi);
    sc->s_w = ldexpf(1.f, e_w);
    sc->fy = ldexpf(1.f, e_y - 2 * e_phi - 2 * e_psi);
    sc->ftheta = ldexpf(1.f, -e_y - e_w);
    if (!isfinite(ma_phi) || !isfinite(ma_psi) || !isfinite(ma_w) || !isfinite(mr_phi * mr_psi)) sc->err = 2;
}

// hi = fp16(x s), lo = fp16(x s - hi); s is a power of two, so for complex64
// input x s and x s - hi are exact in FP32 and no FP64 arithmetic is needed
template <typename T>
__global__ void split_orbitals(const T *x, int64_t ld, int n, int64_t n_r, const float *scale, __half *hi,
                               __half *lo)
{
    const int64_t total = n_r * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / n;
        const int i = (int)(e % n);
        __half ha, hb, la, lb;
        if (sizeof(T) == 8) {
            const float2 v = reinterpret_cast<const float2 *>(x)[r * ld + i];
            const float s = *scale;
            const float a = v.x * s, b = v.y * s;
            ha = __float2half_rn(a);
            hb = __float2half_rn(b);
            la = __float2half_rn(a - __half2float(ha));
            lb = __float2half_rn(b - __half2float(hb));
        } else {
            const double2 v = cload(x, r * ld + i);
            const double s = (double)*scale;
            const double a = v.x * s, b = v.y * s;
            ha = __double2half(a);
            hb = __double2half(b);
            la = __double2half(a - (double)__half2float(ha));
            lb = __double2half(b - (double)__half2float(hb));
        }
        reinterpret_cast<__half2 *>(hi)[r * n + i] = __halves2half2(ha, hb);
        reinterpret_cast<__half2 *>(lo)[r * n + i] = __halves2half2(la, lb);
    }
}

// rotated real matrix of a complex nb x n matrix X (complex128, leading dim ld), scaled and split
__global__ void build_rotated(const double2 *X, int64_t ld, int nb, int n, const float *scale, __half *hi,
                              __half *lo)
{
    const int64_t total = (int64_t)nb * n;
    const double s = (double)*scale;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int v = (int)(e / n), i = (int)(e % n);
        const double2 x = X[(int64_t)v * ld + i];
        const double a = x.x * s, b = x.y * s;
        const __half ha = __double2half(a), hb = __double2half(b);
        const __half la = __double2half(a - (double)__half2float(ha)), lb = __double2half(b - (double)__half2float(hb));
        __half2 *H = reinterpret_cast<__half2 *>(hi), *Lo = reinterpret_cast<__half2 *>(lo);
        H[(int64_t)(2 * v) * n + i] = __halves2half2(ha, hb);
        H[(int64_t)(2 * v + 1) * n + i] = __halves2half2(__hneg(hb), ha);
        Lo[(int64_t)(2 * v) * n + i] = __halves2half2(la, lb);
        Lo[(int64_t)(2 * v + 1) * n + i] = __halves2half2(__hneg(lb), la);
    }
}

struct EpiParams {
    __half *yh, *yl;      // Gram: split Y output, row pitch ldy halves
    int64_t ldy;
    float2 *theta;        // apply: complex64 output, leading dimension ld_theta
    int64_t ld_theta;
    const MixScales *sc;
    int *err;
};

// One persistent CTA per SM walks the output tiles (row-block major, so
// concurrently running CTAs share A tiles in L2). Warp 0 lane 0 feeds the
// 3-stage shared-memory ring with TMA, warp 1 lane 0 issues the MMAs, warps
// 2-9 run the epilogue (warp w reads TMEM lane quarter w % 4 and one half of
// the tile's columns). The K loop runs in segments of `seg` chunks; every
// segment accumulates into a fresh TMEM buffer (the tensor cores' internal
// FP32 accumulation never spans more than one segment) and the epilogue sums
// the segments in registers with IEEE FP32 adds. The TMEM buffer is double
// buffered (tfull / tempty barriers), so the epilogue of one segment overlaps
// the MMAs of the next. DUAL (the Gram-Hadamard kernel) accumulates the
// Phi and Psi products of a segment side by side and writes the split Y.
constexpr int EPI_WARPS = 8;
constexpr int GEMM_THREADS = 64 + 32 * EPI_WARPS;

template <bool DUAL>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    tc_gemm_persist(const __grid_constant__ CUtensorMap a1h, const __grid_constant__ CUtensorMap a1l,
                    const __grid_constant__ CUtensorMap b1h, const __grid_constant__ CUtensorMap b1l,
                    const __grid_constant__ CUtensorMap a2h, const __grid_constant__ CUtensorMap a2l,
                    const __grid_constant__ CUtensorMap b2h, const __grid_constant__ CUtensorMap b2l, int kchunks,
                    int a_row0, int rows, int n_tiles_n, int n_tiles, int seg, EpiParams ep)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[STAGES];
    __shared__ __align__(8) uint64_t empty_bar[STAGES];
    __shared__ __align__(8) uint64_t tfull[2];
    __shared__ __align__(8) uint64_t tempty[2];
    __shared__ __align__(8) uint64_t drain_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int failed;

    if (*(volatile int *)ep.err) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t raw = tc::smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *sbase = smem_raw + (base - raw);
    constexpr int PARTS = DUAL ? 2 : 1;
    constexpr uint32_t ACC = PARTS * TN;   // TMEM columns of one buffer
    constexpr uint32_t NCOLS = 2 * ACC;
    const int nseg = (kchunks + seg - 1) / seg;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&full_bar[s], 1);
            tc::mbar_init(&empty_bar[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            tc::mbar_init(&tfull[a], 1);
            tc::mbar_init(&tempty[a], EPI_WARPS);
        }
        tc::mbar_init(&drain_bar, 1);
        failed = 0;
        tc::fence_barrier_init();
    }
    if (warp == 0) tc::tmem_alloc(&tmem_slot, NCOLS);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            const CUtensorMap *maps[8] = {&a1h, &a1l, &b1h, &b1l, &a2h, &a2l, &b2h, &b2l};
            for (int i = 0; i < 4 * PARTS; ++i) tc::prefetch_map(maps[i]);
            int c = 0, issued = 0;
            for (int tile = blockIdx.x; tile < n_tiles && !failed; tile += gridDim.x) {
                const int m0 = (tile / n_tiles_n) * TM, n0 = (tile % n_tiles_n) * TN;
                for (int sg = 0; sg < nseg && !failed; ++sg)
                    for (int part = 0; part < PARTS && !failed; ++part)
                        for (int kc = sg * seg; kc < min(kchunks, (sg + 1) * seg); ++kc, ++c) {
                            const int s = c % STAGES, it = c / STAGES;
                            if (!tc::mbar_wait(&empty_bar[s], (it & 1) ^ 1, WAIT_BUDGET)) {
                                atomicExch(ep.err, 1);
                                failed = 1;
                                break;
                            }
                            const CUtensorMap *const *mp = maps + 4 * part;
                            uint8_t *st = sbase + s * STAGE_BYTES;
                            tc::mbar_expect_tx(&full_bar[s], STAGE_BYTES);
                            tc::tma_load_2d(st, mp[0], &full_bar[s], kc * TK, a_row0 + m0);
                            tc::tma_load_2d(st + TILE_A, mp[1], &full_bar[s], kc * TK, a_row0 + m0);
                            tc::tma_load_2d(st + 2 * TILE_A, mp[2], &full_bar[s], kc * TK, n0);
                            tc::tma_load_2d(st + 2 * TILE_A + TILE_B, mp[3], &full_bar[s], kc * TK, n0);
                            issued = c + 1;
                        }
            }
            for (int c2 = issued - STAGES > 0 ? issued - STAGES : 0; c2 < issued; ++c2)
                tc::mbar_wait(&full_bar[c2 % STAGES], (c2 / STAGES) & 1, WAIT_BUDGET);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_f16(TM, TN);
            int c = 0, tl = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < n_tiles && !failed && ok; tile += gridDim.x) {
                for (int sg = 0; sg < nseg && ok; ++sg, ++tl) {
                    const int acc = tl & 1, use = tl >> 1;
                    if (!tc::mbar_wait(&tempty[acc], (use & 1) ^ 1, WAIT_BUDGET)) {
                        atomicExch(ep.err, 1);
                        failed = 1;
                        ok = false;
                        break;
                    }
                    tc::fence_after();
                    for (int part = 0; part < PARTS && ok; ++part) {
                        const uint32_t d = tmem + (uint32_t)acc * ACC + (uint32_t)part * TN;
                        const int k0 = sg * seg, k1 = min(kchunks, (sg + 1) * seg);
                        for (int kc = k0; kc < k1; ++kc, ++c) {
                            const int s = c % STAGES, it = c / STAGES;
                            if (!tc::mbar_wait(&full_bar[s], it & 1, WAIT_BUDGET)) {
                                atomicExch(ep.err, 1);
                                failed = 1;
                                ok = false;
                                break;
                            }
                            tc::fence_after();
                            const uint32_t sa = base + s * STAGE_BYTES;
                            const uint64_t dah = tc::desc_sw128(sa), dal = tc::desc_sw128(sa + TILE_A);
                            const uint64_t dbh = tc::desc_sw128(sa + 2 * TILE_A),
                                           dbl = tc::desc_sw128(sa + 2 * TILE_A + TILE_B);
#pragma unroll
                            for (int kk = 0; kk < TK / 16; ++kk) {
                                const uint64_t o = (uint64_t)(2 * kk);
                                tc::mma_f16(d, dah + o, dbh + o, idesc, (kc > k0 || kk > 0) ? 1u : 0u);
                                tc::mma_f16(d, dah + o, dbl + o, idesc, 1u);
                                tc::mma_f16(d, dal + o, dbh + o, idesc, 1u);
                            }
                            tc::mma_commit(&empty_bar[s]);
                        }
                    }
                    if (!ok) break;
                    tc::mma_commit(&tfull[acc]);
                }
            }
            // no MMA may still be running when the TMEM is released
            tc::mma_commit(&drain_bar);
            tc::mbar_wait(&drain_bar, 0, WAIT_BUDGET);
        }
        __syncwarp();
    } else {
        const int quarter = warp & 3;          // TMEM lane quarter this warp may access
        const int half = (warp - 2) >> 2;      // which 64 of the tile's 128 columns
        constexpr int HC = TN / 2;
        int tl = 0;
        for (int tile = blockIdx.x; tile < n_tiles && !failed; tile += gridDim.x) {
            const int m0 = (tile / n_tiles_n) * TM, n0 = (tile % n_tiles_n) * TN;
            const int row = m0 + quarter * 32 + lane;
            float sa[HC], sb[DUAL ? HC : 1];
#pragma unroll
            for (int i = 0; i < HC; ++i) sa[i] = 0.f;
#pragma unroll
            for (int i = 0; i < (DUAL ? HC : 1); ++i) sb[i] = 0.f;
            bool ok = true;
            for (int sg = 0; sg < nseg; ++sg, ++tl) {
                const int acc = tl & 1, use = tl >> 1;
                if (!tc::mbar_wait(&tfull[acc], use & 1, WAIT_BUDGET)) {
                    atomicExch(ep.err, 1);
                    failed = 1;
                    ok = false;
                    break;
                }
                tc::fence_after();
                const uint32_t ta = tmem + (uint32_t)acc * ACC + ((uint32_t)(quarter * 32) << 16) + half * HC;
#pragma unroll
                for (int j = 0; j < HC / 16; ++j) {
                    uint32_t r[16];
                    tc::tmem_ld16(ta + 16 * j, r);
                    if (DUAL) {
                        uint32_t r2[16];
                        tc::tmem_ld16(ta + TN + 16 * j, r2);
                        tc::tmem_wait_ld();
#pragma unroll
                        for (int q = 0; q < 16; ++q) sb[(16 * j + q) % (DUAL ? HC : 1)] += __uint_as_float(r2[q]);
                    } else {
                        tc::tmem_wait_ld();
                    }
#pragma unroll
                    for (int q = 0; q < 16; ++q) sa[16 * j + q] += __uint_as_float(r[q]);
                }
                tc::fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&tempty[acc]);
            }
            if (!ok) break;
            if (row >= rows) continue;
            if (DUAL) {
                const float fy = ep.sc->fy;
#pragma unroll
                for (int j = 0; j < HC / 32; ++j) {
                    __half2 hv[16], lv[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const float ar = sa[32 * j + 2 * q], ai = sa[32 * j + 2 * q + 1];
                        const float br = sb[(32 * j + 2 * q) % (DUAL ? HC : 1)],
                                    bi = sb[(32 * j + 2 * q + 1) % (DUAL ? HC : 1)];
                        const float yr = (ar * br + ai * bi) * fy, yi = (ai * br - ar * bi) * fy;
                        const __half2 h = __floats2half2_rn(yr, yi);
                        const float2 hf = __half22float2(h);
                        hv[q] = h;
                        lv[q] = __floats2half2_rn(yr - hf.x, yi - hf.y);
                    }
                    uint4 *dh = reinterpret_cast<uint4 *>(ep.yh + row * ep.ldy + n0 + half * HC + 32 * j);
                    uint4 *dl = reinterpret_cast<uint4 *>(ep.yl + row * ep.ldy + n0 + half * HC + 32 * j);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        dh[q] = reinterpret_cast<const uint4 *>(hv)[q];
                        dl[q] = reinterpret_cast<const uint4 *>(lv)[q];
                    }
                }
            } else {
                const float ft = ep.sc->ftheta;
                float2 *dst = ep.theta + row * ep.ld_theta + ((n0 + half * HC) >> 1);
#pragma unroll
                for (int q = 0; q < HC / 2; ++q) dst[q] = make_float2(sa[2 * q] * ft, sa[2 * q + 1] * ft);
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, NCOLS);
}

int num_sms()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    }
    return n;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D FP16 map: `inner` halves per row, `rows` rows, box 64 x 128, 128-byte swizzle
bool make_map(CUtensorMap *m, const void *base, uint64_t inner, uint64_t rows)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[2] = {inner, rows};
    cuuint64_t strides[1] = {inner * 2};
    cuuint32_t box[2] = {TK, TM};
    cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

unsigned grid_for(int64_t total, unsigned cap = 8192)
{
    const int64_t g = (total + 255) / 256;
    return (unsigned)(g < 1 ? 1 : (g < cap ? g : cap));
}

template <typename T>
isdf_status halloc(T **p, size_t count)
{
    ISDF_CUDA_TRY(cudaMalloc((void **)p, sizeof(T) * (count ? count : 1)));
    return ISDF_OK;
}

}  // namespace

bool mixed_supported(int n, int n_mu, int64_t, int64_t, int)
{
    return n % 32 == 0 && n_mu % 64 == 0 && n >= 32 && n_mu >= 64;
}

static isdf_status mixed_alloc(isdf_plan *p)
{
    MixedBuffers *b = static_cast<MixedBuffers *>(calloc(1, sizeof(MixedBuffers)));
    if (!b) return ISDF_ERR_CUDA;
    p->mixed = b;
    const int n = p->n_phi, nm = p->n_mu;
    const size_t rowsA = (size_t)p->n_r * 2 * n;
    ISDF_TRY(halloc(&b->a1h, rowsA));
    ISDF_TRY(halloc(&b->a1l, rowsA));
    ISDF_TRY(halloc(&b->a2h, rowsA));
    ISDF_TRY(halloc(&b->a2l, rowsA));
    ISDF_TRY(halloc(&b->b1h, (size_t)2 * nm * 2 * n));
    ISDF_TRY(halloc(&b->b1l, (size_t)2 * nm * 2 * n));
    ISDF_TRY(halloc(&b->b2h, (size_t)2 * nm * 2 * n));
    ISDF_TRY(halloc(&b->b2l, (size_t)2 * nm * 2 * n));
    ISDF_TRY(halloc(&b->bwh, (size_t)2 * nm * 2 * nm));
    ISDF_TRY(halloc(&b->bwl, (size_t)2 * nm * 2 * nm));
    ISDF_TRY(halloc(&b->yh, (size_t)p->max_rows * 2 * nm));
    ISDF_TRY(halloc(&b->yl, (size_t)p->max_rows * 2 * nm));
    ISDF_TRY(halloc(&b->sc, 1));
    bool ok = true;
    ok &= make_map(&b->m_a1h, b->a1h, 2 * n, p->n_r);
    ok &= make_map(&b->m_a1l, b->a1l, 2 * n, p->n_r);
    ok &= make_map(&b->m_a2h, b->a2h, 2 * n, p->n_r);
    ok &= make_map(&b->m_a2l, b->a2l, 2 * n, p->n_r);
    ok &= make_map(&b->m_b1h, b->b1h, 2 * n, 2 * nm);
    ok &= make_map(&b->m_b1l, b->b1l, 2 * n, 2 * nm);
    ok &= make_map(&b->m_b2h, b->b2h, 2 * n, 2 * nm);
    ok &= make_map(&b->m_b2l, b->b2l, 2 * n, 2 * nm);
    ok &= make_map(&b->m_bwh, b->bwh, 2 * nm, 2 * nm);
    ok &= make_map(&b->m_bwl, b->bwl, 2 * nm, 2 * nm);
    ok &= make_map(&b->m_yh, b->yh, 2 * nm, p->max_rows);
    ok &= make_map(&b->m_yl, b->yl, 2 * nm, p->max_rows);
    if (!ok) return ISDF_ERR_CUDA;
    ISDF_CUDA_TRY(
        cudaFuncSetAttribute(tc_gemm_persist<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    ISDF_CUDA_TRY(
        cudaFuncSetAttribute(tc_gemm_persist<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    return ISDF_OK;
}

isdf_status mixed_prepare(isdf_plan *p, cudaStream_t st)
{
    if (!p->mixed) ISDF_TRY(mixed_alloc(p));
    MixedBuffers *b = p->mixed;
    const int n = p->n_phi, nm = p->n_mu;
    ISDF_CUDA_TRY(cudaMemsetAsync(b->sc, 0, sizeof(MixScales), st));

    const unsigned g = 152 * 8;
    if (p->dtype == ISDF_C128) {
        absmax_rows<double2><<<g, 256, 0, st>>>(static_cast<const double2 *>(p->phi), p->ld_phi, n, p->n_r,
                                                &b->sc->maxabs_phi, &b->sc->maxrho_phi); isdf_note_launch();
        absmax_rows<double2><<<g, 256, 0, st>>>(static_cast<const double2 *>(p->psi), p->ld_psi, n, p->n_r,
                                                &b->sc->maxabs_psi, &b->sc->maxrho_psi); isdf_note_launch();
    } else {
        absmax_rows<float2><<<g, 256, 0, st>>>(static_cast<const float2 *>(p->phi), p->ld_phi, n, p->n_r,
                                               &b->sc->maxabs_phi, &b->sc->maxrho_phi); isdf_note_launch();
        absmax_rows<float2><<<g, 256, 0, st>>>(static_cast<const float2 *>(p->psi), p->ld_psi, n, p->n_r,
                                               &b->sc->maxabs_psi, &b->sc->maxrho_psi); isdf_note_launch();
    }
    absmax_rows<double2><<<grid_for((int64_t)nm * 32), 256, 0, st>>>(p->W, nm, nm, nm, &b->sc->maxabs_w, nullptr); isdf_note_launch();
    compute_scales<<<1, 1, 0, st>>>(b->sc); isdf_note_launch();
    ISDF_LAUNCH_CHECK();
    const int64_t tot = p->n_r * n;
    if (p->dtype == ISDF_C128) {
        split_orbitals<double2><<<grid_for(tot, 152 * 64), 256, 0, st>>>(
            static_cast<const double2 *>(p->phi), p->ld_phi, n, p->n_r, &b->sc->s_phi, b->a1h, b->a1l); isdf_note_launch();
        split_orbitals<double2><<<grid_for(tot, 152 * 64), 256, 0, st>>>(
            static_cast<const double2 *>(p->psi), p->ld_psi, n, p->n_r, &b->sc->s_psi, b->a2h, b->a2l); isdf_note_launch();
    } else {
        split_orbitals<float2><<<grid_for(tot, 152 * 64), 256, 0, st>>>(
            static_cast<const float2 *>(p->phi), p->ld_phi, n, p->n_r, &b->sc->s_phi, b->a1h, b->a1l); isdf_note_launch();
        split_orbitals<float2><<<grid_for(tot, 152 * 64), 256, 0, st>>>(
            static_cast<const float2 *>(p->psi), p->ld_psi, n, p->n_r, &b->sc->s_psi, b->a2h, b->a2l); isdf_note_launch();
    }
    build_rotated<<<grid_for((int64_t)nm * n), 256, 0, st>>>(p->phi_mu, n, nm, n, &b->sc->s_phi, b->b1h, b->b1l); isdf_note_launch();
    build_rotated<<<grid_for((int64_t)nm * n), 256, 0, st>>>(p->psi_mu, n, nm, n, &b->sc->s_psi, b->b2h, b->b2l); isdf_note_launch();
    build_rotated<<<grid_for((int64_t)nm * nm), 256, 0, st>>>(p->W, nm, nm, nm, &b->sc->s_w, b->bwh, b->bwl); isdf_note_launch();
    ISDF_LAUNCH_CHECK();
    return ISDF_OK;
}

isdf_status mixed_fit(isdf_plan *p, int64_t row_begin, int64_t row_count, void *theta, int64_t ld_theta,
                      cudaStream_t st)
{
    MixedBuffers *b = p->mixed;
    const int n = p->n_phi, nm = p->n_mu;
    int *err = &b->sc->err;
    for (int64_t r0 = row_begin; r0 < row_begin + row_count; r0 += p->max_rows) {
        const int rows =
            (int)((row_begin + row_count - r0) < p->max_rows ? (row_begin + row_count - r0) : p->max_rows);
        EpiParams ep{};
        ep.yh = b->yh;
        ep.yl = b->yl;
        ep.ldy = 2 * nm;
        ep.sc = b->sc;
        ep.err = err;
        const int n_tiles_n = (2 * nm) / TN, m_tiles = (rows + TM - 1) / TM;
        const int n_tiles = n_tiles_n * m_tiles;
        const unsigned grid = (unsigned)(n_tiles < num_sms() ? n_tiles : num_sms());
        const unsigned threads = GEMM_THREADS;
        // a10: Y_b = (Phi_b Phi_mu^H) o conj(Psi_b Psi_mu^H), written split for the next GEMM
        timer_start(p, 0, st);
        tc_gemm_persist<true><<<grid, threads, SMEM_BYTES, st>>>(b->m_a1h, b->m_a1l, b->m_b1h, b->m_b1l, b->m_a2h,
                                                                 b->m_a2l, b->m_b2h, b->m_b2l, (2 * n) / TK, (int)r0,
                                                                 rows, n_tiles_n, n_tiles, kGramSegment, ep); isdf_note_launch();
        timer_stop(p, 0, st, rows);
        ISDF_LAUNCH_CHECK();
        // a11: Theta_b = Y_b M^-1
        ep.theta = static_cast<float2 *>(theta) + (r0 - row_begin) * ld_theta;
        ep.ld_theta = ld_theta;
        timer_start(p, 1, st);
        tc_gemm_persist<false><<<grid, threads, SMEM_BYTES, st>>>(b->m_yh, b->m_yl, b->m_bwh, b->m_bwl, b->m_yh,
                                                                  b->m_yl, b->m_bwh, b->m_bwl, (2 * nm) / TK, 0, rows,
                                                                  n_tiles_n, n_tiles, kApplySegment, ep); isdf_note_launch();
        timer_stop(p, 1, st, rows);
        ISDF_LAUNCH_CHECK();
    }
    return ISDF_OK;
}

isdf_status mixed_status(isdf_plan *p, int32_t *code)
{
    *code = 0;
    if (!p->mixed) return ISDF_OK;
    int h = 0;
    ISDF_CUDA_TRY(cudaMemcpy(&h, &p->mixed->sc->err, sizeof(int), cudaMemcpyDeviceToHost));
    *code = h == 1 ? ISDF_ERR_TIMEOUT : (h == 2 ? ISDF_ERR_NONFINITE : 0);
    return ISDF_OK;
}

void mixed_release(isdf_plan *p)
{
    MixedBuffers *b = p->mixed;
    if (!b) return;
    void *bufs[] = {b->a1h, b->a1l, b->a2h, b->a2l, b->b1h, b->b1l, b->b2h,
                    b->b2l, b->bwh, b->bwl, b->yh,  b->yl,  b->sc};
    for (void *x : bufs)
        if (x) cudaFree(x);
    free(b);
    p->mixed = nullptr;
}
