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

#include <cfloat>

#include "mixed.cuh"
#include "tc.cuh"

namespace {

// K chunk of 64 FP16 (one 128-byte row per tile row, 128-byte swizzle) in a 3-stage ring of 64 KB
// (a 6-stage ring of 32-element chunks with 64-byte swizzle was 13-17 % slower at N_mu = 4096)
constexpr int TM = 128, TN = 128, TK = 64;
constexpr int STAGES = 3;
constexpr int TILE_A = TM * TK * 2;
constexpr int TILE_B = TN * TK * 2;
constexpr int STAGE_BYTES = 2 * TILE_A + 2 * TILE_B;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;
constexpr long long WAIT_BUDGET = 200000000LL;   // SM cycles (~0.1 s); normal waits take microseconds
// K per TMEM accumulation segment (segments are summed in FP32 registers). Measured on silica-like orbitals
// (80^3, N = 1024, N_mu = 4096; Theta against the FP64 mode on 16,384 rows): Gram segments of 512 give 5.4e-6, one
// segment over the whole K 2.3e-5; M^-1 segments of 512 or 1024 give 5.4e-6 / 5.3e-6, one segment 1.2e-5. The
// longer M^-1 segments drain TMEM half as often (7.45 -> 7.05 ms per 32,768 rows).
constexpr int kGramSegmentK = 512, kApplySegmentK = 1024;
constexpr int kApplySegment = kApplySegmentK / TK;   // K chunks per segment in the M^-1 GEMM
constexpr int kGramSegment = kGramSegmentK / TK;     // the same for each of the two Gram products

struct MixScales {
    unsigned int maxabs_phi, maxrho_phi, maxabs_psi, maxrho_psi, maxabs_w;  // float bits
    float s_phi, s_psi, s_w, fy, ftheta;
    float s_y, inv_phi2, inv_psi2;   // scale of the split Y; 1/s_phi^2, 1/s_psi^2
    int err;
    int pad[2];
};

}  // namespace

struct MixedBuffers {
    __half *a1h, *a1l, *a2h, *a2l;   // N_r x 2N split orbitals
    __half *b1h, *b1l, *b2h, *b2l;   // 2 N_mu x 2N rotated Phi_mu, Psi_mu
    __half *bwh, *bwl;               // 2 N_mu x 2 N_mu rotated M^-1
    __half *yh, *yl;                 // max_rows x 2 N_mu split Y block
    MixScales *sc;
    CUtensorMap m_a1h, m_a1l, m_a2h, m_a2l, m_b1h, m_b1l, m_b2h, m_b2l, m_bwh, m_bwl, m_yh, m_yl;
    // the Gram operands B in 64-row boxes: each CTA of a pair loads half of a 128-column tile
    CUtensorMap m_b1h_half, m_b1l_half, m_b2h_half, m_b2l_half;
    // adjoint (allocated on the first backward call)
    float2 *ac, *bc, *tc, *gc, *ybc;      // max_rows x N_mu complex64: P^phi, P^psi, Theta, G, Ybar
    __half *oah, *oal;                    // split A operand scratch (max(R 2N_mu, N_mu 2R) halves)
    __half *obh, *obl;                    // split B operand scratch (2 max(N, N_mu) x 2R halves)
    __half *kh, *kl;                      // rotated K^T (2N_mu x 2N_mu)
    __half *pmh, *pml, *qmh, *qml;        // rotated Phi_mu^H, Psi_mu^H (2N x 2N_mu)
    float *adj_sc;                        // per-operand scales (see the adjoint code)
    unsigned int *adj_max;                // per-operand max |.| (float bits)
};

namespace {

__device__ __forceinline__ void atomic_max_pos(unsigned int *p, float v) { atomicMax(p, __float_as_uint(v)); }

// max |Re|, |Im| over the matrix and max row density sum_i |x_ri|^2 (FP32 for
// complex64 input, FP64 for complex128; both are bounds used with margins)
template <typename T>
__global__ void absmax_rows(const T *x, int64_t ld, int n, int64_t n_r, unsigned int *maxabs, unsigned int *maxrho)
{
    float ma = 0.f, mr = 0.f;
    bool bad = false;   // an infinite or NaN entry
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
                // fmaxf drops a NaN operand: NaN entries are flagged separately
                bad |= !(fabsf(v.x) <= FLT_MAX) || !(fabsf(v.y) <= FLT_MAX);
                ma = fmaxf(ma, fmaxf(fabsf(v.x), fabsf(v.y)));
                acc = fmaf(v.x, v.x, fmaf(v.y, v.y, acc));
            }
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            rho = acc * (1.f + 1e-5f);
        } else {
            // converted to float first: the bounds only set power-of-two scales
            float acc = 0.f;
            for (int i = lane; i < n; i += 32) {
                const double2 v = cload(x, r * ld + i);
                const float a = d2f_int(v.x), b = d2f_int(v.y);
                bad |= !(fabsf(a) <= FLT_MAX) || !(fabsf(b) <= FLT_MAX);
                ma = fmaxf(ma, fmaxf(fabsf(a), fabsf(b)));
                acc = fmaf(a, a, fmaf(b, b, acc));
            }
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            rho = acc * (1.f + 1e-4f);
        }
        mr = fmaxf(mr, rho);
    }
    for (int o = 16; o > 0; o >>= 1) {
        ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, o));
        mr = fmaxf(mr, __shfl_xor_sync(0xffffffffu, mr, o));
    }
    // a non-finite entry makes the bound infinite, which compute_scales reports as ISDF_ERR_NONFINITE
    if (__any_sync(0xffffffffu, bad)) ma = INFINITY;
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
    sc->s_y = ldexpf(1.f, e_y);
    sc->inv_phi2 = ldexpf(1.f, -2 * e_phi);
    sc->inv_psi2 = ldexpf(1.f, -2 * e_psi);
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
            // one rounding to float (2^-24), below the split's own 2^-22; s is a power of two
            const double2 v = cload(x, r * ld + i);
            const float s = *scale;
            const float a = d2f_int(v.x) * s, b = d2f_int(v.y) * s;
            ha = __float2half_rn(a);
            hb = __float2half_rn(b);
            la = __float2half_rn(a - __half2float(ha));
            lb = __float2half_rn(b - __half2float(hb));
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

enum { OUT_C64 = 0, OUT_ADD_C128 = 1, OUT_ATOMIC_C128 = 2, OUT_C128 = 3, OUT_SPLIT_HV = 4 };

struct EpiParams {
    // Gram-Hadamard (DUAL): split Y, and optionally P^phi, P^psi as complex64
    __half *yh, *yl;      // row pitch ldy halves
    int64_t ldy;
    float2 *aout, *bout;  // or NULL; leading dimension ldab (complex)
    int64_t ldab;
    // single product: result = alpha * acc / (*sa * *sb), stored per out_mode
    int out_mode;
    void *out;            // complex64 (OUT_C64) or complex128, leading dimension ldo (complex)
    int64_t ldo;
    const float *sa, *sb;
    float alpha;
    int ksplit;           // K partitions, each a separate tile (OUT_ATOMIC_C128 only)
    int ncols;            // valid real output columns (multiple of 64)
    const MixScales *sc;
    int *err;
    // OUT_SPLIT_HV: H = (acc * *fvh) o V written split (hi + lo FP16) to yh / yl like Y
    const float2 *vmat;   // complex64, leading dimension ldv (complex), row 0 = the block's first row
    int64_t ldv;
    const float *fvh;
    long long budget;     // cycle budget of the pipeline waits; 0: WAIT_BUDGET (the drain waits keep it);
                          // < 0: test hook, see isdf_plan_set_wait_budget
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

// Output tile order: groups of kGroupM row tiles, all column tiles of a group before the next
// group, row tile fastest within the group. The ~152 tiles in flight then cover ~kGroupM row tiles
// x ~152/kGroupM column tiles, so both operands' panels are shared in L2 by several CTAs; with the
// plain row-major order they span ~2 row tiles x every column tile, and a B operand larger than L2
// (e.g. the 268 MB split M^-1 at N_mu = 4096) is re-read from HBM every ~2 row tiles.
constexpr int kGroupM = 16;
constexpr int kGroupPairM = 8;   // pair tiles are 256 rows: 8 of them hold the same 2,048 rows of A as 16 single tiles

__device__ __forceinline__ void tile_coords(int mn, int n_tiles_n, int m_tiles, int &m0, int &n0, int group = kGroupM)
{
    const int per_group = group * n_tiles_n;
    const int g = mn / per_group, r = mn - g * per_group;
    const int gm0 = g * group;
    const int gm = min(group, m_tiles - gm0);
    m0 = (gm0 + r % gm) * TM;
    n0 = (r / gm) * TN;
}

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
    __shared__ __align__(8) uint64_t never_bar;   // signalled by nothing (the test hook waits on it)
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int failed;

    if (*(volatile int *)ep.err) return;
    const long long budget = ep.budget > 0 ? ep.budget : WAIT_BUDGET;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t raw = tc::smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *sbase = smem_raw + (base - raw);
    constexpr int PARTS = DUAL ? 2 : 1;
    constexpr uint32_t ACC = PARTS * TN;   // TMEM columns of one buffer
    constexpr uint32_t NCOLS = 2 * ACC;
    const int ksplit = (DUAL || ep.ksplit < 1) ? 1 : ep.ksplit;
    const int kper = (kchunks + ksplit - 1) / ksplit;   // K chunks of one split
    const int n_work = n_tiles * ksplit;

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
        tc::mbar_init(&never_bar, 1);
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
            for (int t = blockIdx.x; t < n_work && !failed; t += gridDim.x) {
                const int mn = t / ksplit, ks = t % ksplit;
                int m0, n0;
                tile_coords(mn, n_tiles_n, n_tiles / n_tiles_n, m0, n0);
                const int kb = ks * kper, ke = min(kchunks, kb + kper);
                for (int s0 = kb; s0 < ke && !failed; s0 += seg)
                    for (int part = 0; part < PARTS && !failed; ++part)
                        for (int kc = s0; kc < min(ke, s0 + seg); ++kc, ++c) {
                            const int s = c % STAGES, it = c / STAGES;
                            if (!tc::mbar_wait(&empty_bar[s], (it & 1) ^ 1, budget)) {
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
            // test hook (negative budget): a wait on a barrier that nothing signals runs out after
            // -budget cycles and takes the timeout path before any MMA is issued
            if (ep.budget < 0 && !tc::mbar_wait(&never_bar, 0, -ep.budget)) {
                atomicExch(ep.err, 1);
                failed = 1;
                ok = false;
            }
            for (int t = blockIdx.x; t < n_work && !failed && ok; t += gridDim.x) {
                const int ks = t % ksplit;
                const int kb = ks * kper, ke = min(kchunks, kb + kper);
                for (int s0 = kb; s0 < ke && ok; s0 += seg, ++tl) {
                    const int acc = tl & 1, use = tl >> 1;
                    if (!tc::mbar_wait(&tempty[acc], (use & 1) ^ 1, budget)) {
                        atomicExch(ep.err, 1);
                        failed = 1;
                        ok = false;
                        break;
                    }
                    tc::fence_after();
                    const int s1 = min(ke, s0 + seg);
                    for (int part = 0; part < PARTS && ok; ++part) {
                        const uint32_t d = tmem + (uint32_t)acc * ACC + (uint32_t)part * TN;
                        for (int kc = s0; kc < s1; ++kc, ++c) {
                            const int s = c % STAGES, it = c / STAGES;
                            if (!tc::mbar_wait(&full_bar[s], it & 1, budget)) {
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
                                tc::mma_f16(d, dah + o, dbh + o, idesc, (kc > s0 || kk > 0) ? 1u : 0u);
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
        for (int t = blockIdx.x; t < n_work && !failed; t += gridDim.x) {
            const int mn = t / ksplit, ks = t % ksplit;
            int m0, n0;
            tile_coords(mn, n_tiles_n, n_tiles / n_tiles_n, m0, n0);
            const int kb = ks * kper, ke = min(kchunks, kb + kper);
            const int row = m0 + quarter * 32 + lane;
            float sa[HC], sb[DUAL ? HC : 1];
#pragma unroll
            for (int i = 0; i < HC; ++i) sa[i] = 0.f;
#pragma unroll
            for (int i = 0; i < (DUAL ? HC : 1); ++i) sb[i] = 0.f;
            bool ok = true;
            for (int s0 = kb; s0 < ke; s0 += seg, ++tl) {
                const int acc = tl & 1, use = tl >> 1;
                if (!tc::mbar_wait(&tfull[acc], use & 1, budget)) {
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
            if (row >= rows || ke <= kb || n0 + half * HC >= ep.ncols) continue;
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
                if (ep.aout) {
                    // the two products themselves (for the adjoint), unscaled, as complex64
                    const float fa = ep.sc->inv_phi2, fb = ep.sc->inv_psi2;
                    float2 *da = ep.aout + row * ep.ldab + ((n0 + half * HC) >> 1);
                    float2 *db = ep.bout + row * ep.ldab + ((n0 + half * HC) >> 1);
#pragma unroll
                    for (int q = 0; q < HC / 2; ++q) {
                        da[q] = make_float2(sa[2 * q] * fa, sa[2 * q + 1] * fa);
                        db[q] = make_float2(sb[(2 * q) % (DUAL ? HC : 1)] * fb, sb[(2 * q + 1) % (DUAL ? HC : 1)] * fb);
                    }
                }
            } else if (ep.out_mode == OUT_SPLIT_HV) {
                // exchange: H = P o V for the next product, P = acc / s^2 carried in *fvh with H's scale
                const float f = *ep.fvh;
                const float2 *vr = ep.vmat + row * ep.ldv + ((n0 + half * HC) >> 1);
#pragma unroll
                for (int j = 0; j < HC / 32; ++j) {
                    __half2 hv[16], lv[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const float2 vv = vr[16 * j + q];
                        const float ar = sa[32 * j + 2 * q] * f, ai = sa[32 * j + 2 * q + 1] * f;
                        const float yr = ar * vv.x - ai * vv.y, yi = ar * vv.y + ai * vv.x;
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
                const float f = ep.alpha / ((*ep.sa) * (*ep.sb));
                const int64_t col = (n0 + half * HC) >> 1;
                if (ep.out_mode == OUT_C128) {
                    double2 *dst = static_cast<double2 *>(ep.out) + row * ep.ldo + col;
#pragma unroll
                    for (int q = 0; q < HC / 2; ++q)
                        dst[q] = make_double2((double)(sa[2 * q] * f), (double)(sa[2 * q + 1] * f));
                } else if (ep.out_mode == OUT_C64) {
                    float2 *dst = static_cast<float2 *>(ep.out) + row * ep.ldo + col;
#pragma unroll
                    for (int q = 0; q < HC / 2; ++q) dst[q] = make_float2(sa[2 * q] * f, sa[2 * q + 1] * f);
                } else if (ep.out_mode == OUT_ADD_C128) {
                    double2 *dst = static_cast<double2 *>(ep.out) + row * ep.ldo + col;
#pragma unroll
                    for (int q = 0; q < HC / 2; ++q) {
                        double2 v = dst[q];
                        v.x += (double)(sa[2 * q] * f);
                        v.y += (double)(sa[2 * q + 1] * f);
                        dst[q] = v;
                    }
                } else {
                    double *dst = reinterpret_cast<double *>(static_cast<double2 *>(ep.out) + row * ep.ldo + col);
#pragma unroll
                    for (int q = 0; q < HC; ++q) atomicAdd(dst + q, (double)(sa[q] * f));
                }
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, NCOLS);
}

// ---------------------------------------------------------------- CTA-pair GEMM
// The same products on CTA pairs (clusters of two, cta_group::2): one MMA of M = 256 rows covers the
// pair's two 128-row halves, each CTA holding its 128 rows of A, half of the BN rows of B and its
// 128 rows of the accumulator in its own TMEM. Per SM and per FLOP this halves the B bytes loaded
// from L2 and the operand bytes the tensor core reads from shared memory (the single-CTA kernel is
// bound by that operand feed). Roles:
//  * rank 0 (leader): warp 0 lane 0 loads the leader's stages and adds both CTAs' bytes to the
//    leader's full barrier of each stage; warp 1 lane 0 issues the pair's MMAs and commits them to
//    both CTAs' empty and tfull barriers; warps 2-9 run the epilogue of the leader's rows;
//  * rank 1 (peer): warp 0 lane 0 loads the peer's stages into its own shared memory, completing on
//    the leader's full barrier, as soon as the slot is empty (the barrier's transaction count is
//    signed, so the peer's bytes may land before the leader's expect: the phase still needs the
//    leader's arrival and every byte); at the end it reports its stage count to the leader, which
//    drains every copy of both CTAs before the pair exits; warps 2-9 run the epilogue of the peer's
//    rows and release the accumulator with a remote arrive on the leader's tempty.
// Every wait is bounded as in tc_gemm_persist; the pair decides to run or to skip (an earlier
// failure) once, from the leader's reading, so both CTAs always meet at the cluster barriers.
template <bool DUAL, int BN>
struct PairCfg {
    static constexpr int BH = BN / 2;                       // B rows per CTA
    static constexpr int TILE_BH = BH * TK * 2;
    static constexpr int STAGE = 2 * TILE_A + 2 * TILE_BH;  // per CTA
    static constexpr int NSTAGE = (192 * 1024) / STAGE;     // 4 (BN = 128) or 3 (BN = 256)
    static constexpr int SMEM = NSTAGE * STAGE + 1024;
    static constexpr int PARTS = DUAL ? 2 : 1;
    static constexpr uint32_t ACC = PARTS * BN;             // TMEM columns of one accumulator buffer
    static constexpr uint32_t NCOLS = 2 * ACC;
    static constexpr int HC = BN / 2;                       // columns per epilogue thread
    static_assert(NCOLS <= 512, "TMEM");
};

template <bool DUAL, int BN>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(GEMM_THREADS, 1)
    tc_gemm_pair(const __grid_constant__ CUtensorMap a1h, const __grid_constant__ CUtensorMap a1l,
                 const __grid_constant__ CUtensorMap b1h, const __grid_constant__ CUtensorMap b1l,
                 const __grid_constant__ CUtensorMap a2h, const __grid_constant__ CUtensorMap a2l,
                 const __grid_constant__ CUtensorMap b2h, const __grid_constant__ CUtensorMap b2l, int kchunks,
                 int a_row0, int rows, int n_tiles_n, int n_tiles, int seg, EpiParams ep)
{
    using C = PairCfg<DUAL, BN>;
    constexpr int S = C::NSTAGE;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[S];
    __shared__ __align__(8) uint64_t empty_bar[S];
    __shared__ __align__(8) uint64_t peer_bar;   // leader: the peer's producer has finished (count below)
    __shared__ volatile int peer_issued;          // leader: stages the peer's producer loaded
    __shared__ __align__(8) uint64_t tfull[2];
    __shared__ __align__(8) uint64_t tempty[2];
    __shared__ __align__(8) uint64_t drain_bar;
    __shared__ __align__(8) uint64_t never_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int failed;
    __shared__ uint32_t skip;

    const uint32_t rank = tc::cluster_rank();
    const bool leader = rank == 0;
    const long long budget = ep.budget > 0 ? ep.budget : WAIT_BUDGET;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t raw = tc::smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *sbase = smem_raw + (base - raw);
    const int n_pairs = gridDim.x >> 1, pair = blockIdx.x >> 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(&full_bar[s], 1);
            tc::mbar_init(&empty_bar[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            tc::mbar_init(&tfull[a], 1);
            tc::mbar_init(&tempty[a], 2 * EPI_WARPS);
        }
        tc::mbar_init(&drain_bar, 1);
        tc::mbar_init(&never_bar, 1);
        tc::mbar_init(&peer_bar, 1);
        failed = 0;
        skip = *(volatile int *)ep.err ? 1u : 0u;   // only the leader's reading is used
        tc::fence_barrier_init();
    }
    __syncthreads();
    tc::cluster_sync();   // both CTAs' barriers initialised before any remote arrive
    const bool run = tc::ld_shared_cluster(tc::map_shared(&skip, 0)) == 0u;
    if (warp == 0) tc::tmem_alloc_pair(&tmem_slot, C::NCOLS);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_slot;
    const int m_ptiles = n_tiles / n_tiles_n;
    const int n_work = run ? n_tiles : 0;

    if (warp == 0) {
        if (lane == 0) {
            const CUtensorMap *maps[8] = {&a1h, &a1l, &b1h, &b1l, &a2h, &a2l, &b2h, &b2l};
            for (int i = 0; i < 4 * C::PARTS; ++i) tc::prefetch_map(maps[i]);
            const uint32_t full0 = tc::map_shared(&full_bar[0], 0);   // the leader's full barriers
            int c = 0, issued = 0;
            for (int t = pair; t < n_work && !failed; t += n_pairs) {
                int m0, n0;
                tile_coords(t, n_tiles_n, m_ptiles, m0, n0, kGroupPairM);          // m0 in pair tiles of TM, n0 in TN units
                m0 = (m0 / TM) * (2 * TM) + (int)rank * TM;           // this CTA's 128 rows of the pair's 256
                n0 = (n0 / TN) * BN + (int)rank * C::BH;              // this CTA's half of the pair's BN columns
                for (int s0 = 0; s0 < kchunks && !failed; s0 += seg)
                    for (int part = 0; part < C::PARTS && !failed; ++part)
                        for (int kc = s0; kc < min(kchunks, s0 + seg); ++kc, ++c) {
                            const int s = c % S, it = c / S;
                            if (!tc::mbar_wait(&empty_bar[s], (it & 1) ^ 1, budget)) {
                                atomicExch(ep.err, 1);
                                failed = 1;
                                break;
                            }
                            if (leader) tc::mbar_expect_tx(&full_bar[s], 2 * C::STAGE);   // both CTAs' bytes
                            const CUtensorMap *const *mp = maps + 4 * part;
                            uint8_t *st = sbase + s * C::STAGE;
                            const uint32_t fb = full0 + (uint32_t)(s * sizeof(uint64_t));
                            tc::tma_load_2d_pair(st, mp[0], fb, kc * TK, a_row0 + m0);
                            tc::tma_load_2d_pair(st + TILE_A, mp[1], fb, kc * TK, a_row0 + m0);
                            tc::tma_load_2d_pair(st + 2 * TILE_A, mp[2], fb, kc * TK, n0);
                            tc::tma_load_2d_pair(st + 2 * TILE_A + C::TILE_BH, mp[3], fb, kc * TK, n0);
                            issued = c + 1;
                        }
            }
            // Every copy of either CTA completes on a leader barrier, so the leader drains them all before the
            // pair exits: the peer reports how many stages it loaded, and the leader waits for the last S
            // stages of either CTA, arming for the peer's bytes alone the stages only the peer loaded (after a
            // failure the peer can run up to S stages ahead of the leader's producer, never more: it loads a
            // stage only after the MMA released the slot's previous stage, which the leader loaded).
            if (!leader) {
                tc::st_shared_cluster(tc::map_shared((const void *)&peer_issued, 0), (uint32_t)issued);
                tc::mbar_arrive_cluster(tc::map_shared(&peer_bar, 0));
            } else {
                int hi = issued;
                if (tc::mbar_wait_cluster(&peer_bar, 0, WAIT_BUDGET)) hi = max(hi, (int)peer_issued);
                for (int c2 = hi - S > 0 ? hi - S : 0; c2 < hi; ++c2) {
                    if (c2 >= issued) tc::mbar_expect_tx(&full_bar[c2 % S], C::STAGE);
                    tc::mbar_wait(&full_bar[c2 % S], (c2 / S) & 1, WAIT_BUDGET);
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0 && leader) {
            constexpr uint32_t idesc = tc::idesc_f16(2 * TM, BN);
            int c = 0, tl = 0;
            bool ok = true;
            if (ep.budget < 0 && !tc::mbar_wait(&never_bar, 0, -ep.budget)) {
                atomicExch(ep.err, 1);
                failed = 1;
                ok = false;
            }
            for (int t = pair; t < n_work && !failed && ok; t += n_pairs) {
                for (int s0 = 0; s0 < kchunks && ok; s0 += seg, ++tl) {
                    const int acc = tl & 1, use = tl >> 1;
                    if (!tc::mbar_wait(&tempty[acc], (use & 1) ^ 1, budget)) {
                        atomicExch(ep.err, 1);
                        failed = 1;
                        ok = false;
                        break;
                    }
                    tc::fence_after();
                    const int s1 = min(kchunks, s0 + seg);
                    for (int part = 0; part < C::PARTS && ok; ++part) {
                        const uint32_t d = tmem + (uint32_t)acc * C::ACC + (uint32_t)part * BN;
                        for (int kc = s0; kc < s1; ++kc, ++c) {
                            const int s = c % S, it = c / S;
                            if (!tc::mbar_wait(&full_bar[s], it & 1, budget)) {
                                atomicExch(ep.err, 1);
                                failed = 1;
                                ok = false;
                                break;
                            }
                            tc::fence_after();
                            const uint32_t sa = base + s * C::STAGE;
                            const uint64_t dah = tc::desc_sw128(sa), dal = tc::desc_sw128(sa + TILE_A);
                            const uint64_t dbh = tc::desc_sw128(sa + 2 * TILE_A),
                                           dbl = tc::desc_sw128(sa + 2 * TILE_A + C::TILE_BH);
#pragma unroll
                            for (int kk = 0; kk < TK / 16; ++kk) {
                                const uint64_t o = (uint64_t)(2 * kk);
                                tc::mma_f16_pair(d, dah + o, dbh + o, idesc, (kc > s0 || kk > 0) ? 1u : 0u);
                                tc::mma_f16_pair(d, dah + o, dbl + o, idesc, 1u);
                                tc::mma_f16_pair(d, dal + o, dbh + o, idesc, 1u);
                            }
                            tc::mma_commit_pair(&empty_bar[s], 0x3);
                        }
                    }
                    if (!ok) break;
                    tc::mma_commit_pair(&tfull[acc], 0x3);
                }
            }
            // no MMA of the pair may still be running when either CTA releases its TMEM
            tc::mma_commit_pair(&drain_bar, 0x1);
            tc::mbar_wait(&drain_bar, 0, WAIT_BUDGET);
        }
        __syncwarp();
    } else {
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        constexpr int HC = C::HC;
        const uint32_t tempty0 = tc::map_shared(&tempty[0], 0);
        int tl = 0;
        for (int t = pair; t < n_work && !failed; t += n_pairs) {
            int m0, n0;
            tile_coords(t, n_tiles_n, m_ptiles, m0, n0, kGroupPairM);
            m0 = (m0 / TM) * (2 * TM) + (int)rank * TM;
            n0 = (n0 / TN) * BN;
            const int row = m0 + quarter * 32 + lane;
            float sa[HC], sb[DUAL ? HC : 1];
#pragma unroll
            for (int i = 0; i < HC; ++i) sa[i] = 0.f;
#pragma unroll
            for (int i = 0; i < (DUAL ? HC : 1); ++i) sb[i] = 0.f;
            bool ok = true;
            for (int s0 = 0; s0 < kchunks; s0 += seg, ++tl) {
                const int acc = tl & 1, use = tl >> 1;
                if (!tc::mbar_wait(&tfull[acc], use & 1, budget)) {
                    atomicExch(ep.err, 1);
                    failed = 1;
                    ok = false;
                    break;
                }
                tc::fence_after();
                const uint32_t ta = tmem + (uint32_t)acc * C::ACC + ((uint32_t)(quarter * 32) << 16) + half * HC;
#pragma unroll
                for (int j = 0; j < HC / 16; ++j) {
                    uint32_t r[16];
                    tc::tmem_ld16(ta + 16 * j, r);
                    if (DUAL) {
                        uint32_t r2[16];
                        tc::tmem_ld16(ta + BN + 16 * j, r2);
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
                if (lane == 0) tc::mbar_arrive_cluster(tempty0 + (uint32_t)(acc * sizeof(uint64_t)));
            }
            if (!ok) break;
            if (row >= rows || n0 + half * HC >= ep.ncols) continue;
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
                const float f = ep.alpha / ((*ep.sa) * (*ep.sb));
                float2 *dst = static_cast<float2 *>(ep.out) + row * ep.ldo + ((n0 + half * HC) >> 1);
#pragma unroll
                for (int q = 0; q < HC / 2; ++q) dst[q] = make_float2(sa[2 * q] * f, sa[2 * q + 1] * f);
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::cluster_sync();   // both CTAs done with TMEM, shared memory and the remote barriers
    if (warp == 0) tc::tmem_dealloc_pair(tmem, C::NCOLS);
}

// ---------------------------------------------------------------- adjoint helpers
// s = 2^(14 - e) from a max |.| held as float bits (a power of two, so scaling is exact)
__global__ void scale_from_max(const unsigned int *maxbits, float *scale, int n)
{
    const int i = threadIdx.x;
    if (i < n) scale[i] = ldexpf(1.f, scale_exp(__uint_as_float(maxbits[i])));
}

// Transposed split operands of a complex R x C matrix X (leading dimension ld):
//   TRANSPOSE_A:  row c of the output = (Re, Im) of x[r][c] for r = 0..R-1 (an A operand for X^T-shaped products)
//   ROTATED:      rows 2c, 2c+1 = (Re x, Im x), (-Im x, Re x) of x[r][c] (a B operand)
// with x = conj(X) when conj is set, scaled by *scale and split into FP16 hi + lo.
// 32 x 32 tiles are transposed through shared memory so that reads and writes are coalesced.
template <typename T, bool ROTATED>
__global__ void split_transposed(const T *X, int64_t ld, int R, int C, int conj, const float *scale, __half *hi,
                                 __half *lo, int64_t out_pitch)
{
    __shared__ float2 tile[32][33];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
    const float s = *scale;
    for (int i = ty; i < 32; i += 8) {
        const int r = r0 + i, c = c0 + tx;
        float2 v = make_float2(0.f, 0.f);
        if (r < R && c < C) {
            float fx, fy;
            if (sizeof(T) == 8) {
                const float2 f = reinterpret_cast<const float2 *>(X)[(int64_t)r * ld + c];
                fx = f.x;
                fy = f.y;
            } else {
                const double2 d = cload(X, (int64_t)r * ld + c);
                fx = d2f_int(d.x);
                fy = d2f_int(d.y);
            }
            v = make_float2(fx * s, (conj ? -fy : fy) * s);
        }
        tile[i][tx] = v;
    }
    __syncthreads();
    __half2 *H = reinterpret_cast<__half2 *>(hi), *L = reinterpret_cast<__half2 *>(lo);
    const int64_t pitch2 = out_pitch / 2;   // in half2
    for (int i = ty; i < 32; i += 8) {
        const int c = c0 + i, r = r0 + tx;
        if (c >= C || r >= R) continue;
        const float2 v = tile[tx][i];
        const __half ha = __float2half_rn(v.x), hb = __float2half_rn(v.y);
        const __half la = __float2half_rn(v.x - __half2float(ha)), lb = __float2half_rn(v.y - __half2float(hb));
        if (ROTATED) {
            H[(int64_t)(2 * c) * pitch2 + r] = __halves2half2(ha, hb);
            H[(int64_t)(2 * c + 1) * pitch2 + r] = __halves2half2(__hneg(hb), ha);
            L[(int64_t)(2 * c) * pitch2 + r] = __halves2half2(la, lb);
            L[(int64_t)(2 * c + 1) * pitch2 + r] = __halves2half2(__hneg(lb), la);
        } else {
            H[(int64_t)c * pitch2 + r] = __halves2half2(ha, hb);
            L[(int64_t)c * pitch2 + r] = __halves2half2(la, lb);
        }
    }
}

// Abar = Ybar o B (into A's place), Bbar = conj(Ybar) o A (into B's place), complex64
__global__ void hadamard_adjoint_c64(const float2 *Yb, float2 *A, float2 *B, int64_t total)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const float2 y = Yb[e], a = A[e], b = B[e];
        A[e] = make_float2(y.x * b.x - y.y * b.y, y.x * b.y + y.y * b.x);
        B[e] = make_float2(y.x * a.x + y.y * a.y, y.x * a.y - y.y * a.x);
    }
}

// loss += 1/2 Re sum conj(Theta) o G over a rows x n block (complex64, leading dimension ld)
__global__ void loss_c64(const float2 *T, const float2 *G, int64_t total, double *loss)
{
    __shared__ double red[8];
    // compensated FP32 sum per thread (error ~2^-24 whatever the count), then FP64 across threads
    float sum = 0.f, comp = 0.f;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const float2 t = T[e], g = G[e];
        const float y = fmaf(t.x, g.x, t.y * g.y) - comp;
        const float u = sum + y;
        comp = (u - sum) - y;
        sum = u;
    }
    double acc = (double)sum - (double)comp;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) b += red[i];
        atomicAdd(loss, 0.5 * b);
    }
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

// 2-D FP16 map: `inner` halves per row (row pitch `pitch` halves, default inner), `rows`
// rows, box TK x box_rows (128 bytes x 128 rows by default), 128-byte swizzle
bool make_map(CUtensorMap *m, const void *base, uint64_t inner, uint64_t rows, uint64_t pitch = 0,
              uint32_t box_rows = TM)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[2] = {inner, rows};
    cuuint64_t strides[1] = {(pitch ? pitch : inner) * 2};
    cuuint32_t box[2] = {TK, box_rows};
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
    ok &= make_map(&b->m_b1h_half, b->b1h, 2 * n, 2 * nm, 0, TM / 2);
    ok &= make_map(&b->m_b1l_half, b->b1l, 2 * n, 2 * nm, 0, TM / 2);
    ok &= make_map(&b->m_b2h_half, b->b2h, 2 * n, 2 * nm, 0, TM / 2);
    ok &= make_map(&b->m_b2l_half, b->b2l, 2 * n, 2 * nm, 0, TM / 2);
    if (!ok) return ISDF_ERR_CUDA;
    ISDF_CUDA_TRY(
        cudaFuncSetAttribute(tc_gemm_persist<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    ISDF_CUDA_TRY(
        cudaFuncSetAttribute(tc_gemm_persist<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    ISDF_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_pair<true, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       PairCfg<true, 128>::SMEM));
    ISDF_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_pair<false, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       PairCfg<false, 256>::SMEM));
    return ISDF_OK;
}

// The part that depends on the orbitals only: their scale bounds and FP16 hi/lo splits
// (the Gram kernel's A operands). It may run concurrently with the FP64 plan update.
isdf_status mixed_prepare_orbitals(isdf_plan *p, cudaStream_t st)
{
    if (!p->mixed) ISDF_TRY(mixed_alloc(p));
    MixedBuffers *b = p->mixed;
    const int n = p->n_phi;
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
    compute_scales<<<1, 1, 0, st>>>(b->sc); isdf_note_launch();   // s_phi, s_psi (final); M^-1's later
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
    ISDF_LAUNCH_CHECK();
    return ISDF_OK;
}

// The rest, after M^-1: its scale (compute_scales again: the orbital scales come out the same)
// and the rotated B operands of Phi_mu, Psi_mu and M^-1.
isdf_status mixed_prepare(isdf_plan *p, cudaStream_t st)
{
    MixedBuffers *b = p->mixed;
    const int n = p->n_phi, nm = p->n_mu;
    absmax_rows<double2><<<grid_for((int64_t)nm * 32), 256, 0, st>>>(p->W, nm, nm, nm, &b->sc->maxabs_w, nullptr); isdf_note_launch();
    compute_scales<<<1, 1, 0, st>>>(b->sc); isdf_note_launch();
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
        ep.budget = p->wait_budget;
        ep.ksplit = 1;
        ep.ncols = 2 * nm;
        const int n_tiles_n = (2 * nm) / TN, m_tiles = (rows + TM - 1) / TM;
        const int n_tiles = n_tiles_n * m_tiles;
        const unsigned grid = (unsigned)(n_tiles < num_sms() ? n_tiles : num_sms());
        const unsigned threads = GEMM_THREADS;
        // CTA pairs for the M^-1 application: 256 x 256 tiles (each CTA 128 rows and 128 B rows). The Gram
        // product stays on single CTAs: as 256 x 128 pair tiles (two accumulators per tile leave no room for
        // 256 columns) it ran 1.5x slower than the single-CTA kernel at N = 1024, N_mu = 4096.
        const int m_ptiles = (rows + 2 * TM - 1) / (2 * TM);
        const int pn_gram = (2 * nm) / TN, pn_apply = (2 * nm) / 256;
        const int pairs = num_sms() / 2;
        const bool use_pairs = (2 * nm) % 256 == 0;
        constexpr bool kGramPairs = false;
        // a10: Y_b = (Phi_b Phi_mu^H) o conj(Psi_b Psi_mu^H), written split for the next GEMM
        timer_start(p, 0, st);
        if (use_pairs && kGramPairs) {
            const int pt = pn_gram * m_ptiles;
            tc_gemm_pair<true, 128><<<2 * (pt < pairs ? pt : pairs), threads, PairCfg<true, 128>::SMEM, st>>>(
                b->m_a1h, b->m_a1l, b->m_b1h_half, b->m_b1l_half, b->m_a2h, b->m_a2l, b->m_b2h_half, b->m_b2l_half,
                (2 * n) / TK, (int)r0, rows, pn_gram, pt, kGramSegment, ep);
        } else {
            tc_gemm_persist<true><<<grid, threads, SMEM_BYTES, st>>>(b->m_a1h, b->m_a1l, b->m_b1h, b->m_b1l, b->m_a2h,
                                                                     b->m_a2l, b->m_b2h, b->m_b2l, (2 * n) / TK,
                                                                     (int)r0, rows, n_tiles_n, n_tiles, kGramSegment,
                                                                     ep);
        }
        isdf_note_launch();
        timer_stop(p, 0, st, rows);
        ISDF_LAUNCH_CHECK();
        // a11: Theta_b = Y_b M^-1
        ep.out_mode = OUT_C64;
        ep.out = static_cast<float2 *>(theta) + (r0 - row_begin) * ld_theta;
        ep.ldo = ld_theta;
        ep.sa = &b->sc->s_y;
        ep.sb = &b->sc->s_w;
        ep.alpha = 1.f;
        timer_start(p, 1, st);
        if (use_pairs) {
            const int pt = pn_apply * m_ptiles;
            tc_gemm_pair<false, 256><<<2 * (pt < pairs ? pt : pairs), threads, PairCfg<false, 256>::SMEM, st>>>(
                b->m_yh, b->m_yl, b->m_bwh, b->m_bwl, b->m_yh, b->m_yl, b->m_bwh, b->m_bwl, (2 * nm) / TK, 0, rows,
                pn_apply, pt, kApplySegment, ep);
        } else {
            tc_gemm_persist<false><<<grid, threads, SMEM_BYTES, st>>>(b->m_yh, b->m_yl, b->m_bwh, b->m_bwl, b->m_yh,
                                                                      b->m_yl, b->m_bwh, b->m_bwl, (2 * nm) / TK, 0,
                                                                      rows, n_tiles_n, n_tiles, kApplySegment, ep);
        }
        isdf_note_launch();
        timer_stop(p, 1, st, rows);
        ISDF_LAUNCH_CHECK();
    }
    return ISDF_OK;
}


namespace {

// one tensor-core GEMM launch: C (rows x ncols real) = A (rows x K) Bh^T over kchunks chunks of TK
isdf_status run_gemm(const CUtensorMap &ah, const CUtensorMap &al, const CUtensorMap &bh, const CUtensorMap &bl,
                     int kchunks, int rows, int ncols, EpiParams ep, cudaStream_t st)
{
    const int n_tiles_n = (ncols + TN - 1) / TN, m_tiles = (rows + TM - 1) / TM;
    const int n_tiles = n_tiles_n * m_tiles;
    if (ep.ksplit < 1) ep.ksplit = 1;
    const int work = n_tiles * ep.ksplit;
    const unsigned grid = (unsigned)(work < num_sms() ? work : num_sms());
    ep.ncols = ncols;
    tc_gemm_persist<false><<<grid, GEMM_THREADS, SMEM_BYTES, st>>>(ah, al, bh, bl, ah, al, bh, bl, kchunks, 0, rows,
                                                                   n_tiles_n, n_tiles, kApplySegment, ep);
    isdf_note_launch();
    ISDF_LAUNCH_CHECK();
    return ISDF_OK;
}

// split-K factor for a long reduction with few output tiles: ~3 CTAs of work per SM, >= 1024 K each
int ksplit_for(int rows, int ncols, int kchunks)
{
    const int tiles = ((rows + TM - 1) / TM) * ((ncols + TN - 1) / TN);
    int k = (3 * num_sms() + tiles - 1) / tiles;
    const int kmax = kchunks / (1024 / TK) > 1 ? kchunks / (1024 / TK) : 1;
    return k < 1 ? 1 : (k > kmax ? kmax : k);
}

// max |.| of a complex matrix into adj_max[slot], then the power-of-two scale into adj_sc[slot]
template <typename T>
isdf_status operand_scale(MixedBuffers *b, int slot, const T *x, int64_t ld, int cols, int64_t rows, cudaStream_t st)
{
    ISDF_CUDA_TRY(cudaMemsetAsync(b->adj_max + slot, 0, sizeof(unsigned int), st));
    absmax_rows<T><<<grid_for(rows * 32, 152 * 8), 256, 0, st>>>(x, ld, cols, rows, b->adj_max + slot, nullptr);
    isdf_note_launch();
    scale_from_max<<<1, 32, 0, st>>>(b->adj_max + slot, b->adj_sc + slot, 1);
    isdf_note_launch();
    ISDF_LAUNCH_CHECK();
    return ISDF_OK;
}

template <typename T, bool ROT>
isdf_status transposed_operand(const T *x, int64_t ld, int R, int C, int conj, const float *scale, __half *hi,
                               __half *lo, int64_t pitch, cudaStream_t st)
{
    dim3 grid((R + 31) / 32, (C + 31) / 32);
    split_transposed<T, ROT><<<grid, 256, 0, st>>>(x, ld, R, C, conj, scale, hi, lo, pitch);
    isdf_note_launch();
    ISDF_LAUNCH_CHECK();
    return ISDF_OK;
}

enum { SC_THETA = 0, SC_G = 1, SC_ABAR = 2, SC_BBAR = 3, SC_YBAR = 4, SC_K = 5, SC_SLOTS = 8 };

isdf_status adjoint_alloc(isdf_plan *p)
{
    MixedBuffers *b = p->mixed;
    const int64_t R = p->max_rows, nm = p->n_mu, n = p->n_phi;
    const int64_t Rp = (R + 7) & ~(int64_t)7;   // row pitch of the transposed operands (16-byte multiple)
    const size_t blk = (size_t)R * nm;
    ISDF_TRY(halloc(&b->ac, blk));
    ISDF_TRY(halloc(&b->bc, blk));
    ISDF_TRY(halloc(&b->tc, blk));
    ISDF_TRY(halloc(&b->gc, blk));
    ISDF_TRY(halloc(&b->ybc, blk));
    const size_t oa = (size_t)2 * Rp * nm;
    const size_t ob = (size_t)4 * Rp * (nm > n ? nm : n);
    ISDF_TRY(halloc(&b->oah, oa));
    ISDF_TRY(halloc(&b->oal, oa));
    ISDF_TRY(halloc(&b->obh, ob));
    ISDF_TRY(halloc(&b->obl, ob));
    ISDF_TRY(halloc(&b->kh, (size_t)4 * nm * nm));
    ISDF_TRY(halloc(&b->kl, (size_t)4 * nm * nm));
    ISDF_TRY(halloc(&b->pmh, (size_t)4 * n * nm));
    ISDF_TRY(halloc(&b->pml, (size_t)4 * n * nm));
    ISDF_TRY(halloc(&b->qmh, (size_t)4 * n * nm));
    ISDF_TRY(halloc(&b->qml, (size_t)4 * n * nm));
    ISDF_TRY(halloc(&b->adj_sc, SC_SLOTS));
    ISDF_TRY(halloc(&b->adj_max, SC_SLOTS));
    return ISDF_OK;
}

}  // namespace

// Adjoint of Theta(Phi, Psi) at fixed points on the tensor cores (ISDF_MIXED). Per
// block of rows: recompute P^phi, P^psi and Y (Gram kernel), Theta = Y M^-1, G (given
// or 2 dV Theta conj(K)), Ybar = G M^-1, Abar = Ybar o B, Bbar = conj(Ybar) o A, then
// grad_phi rows += Abar Phi_mu, Phibar_mu += Abar^H Phi_b (and Psi likewise), and
// Mbar -= Theta^H Ybar. The three reductions over grid rows use transposed split
// copies and split-K partitions accumulated with FP64 atomics.
isdf_status mixed_backward(isdf_plan *p, int64_t row_begin, int64_t row_count, const void *grad_theta,
                           int64_t ld_grad, const void *K, double dV, void *grad_phi, int64_t ld_gphi,
                           void *grad_psi, int64_t ld_gpsi, double *loss, cudaStream_t st)
{
    MixedBuffers *b = p->mixed;
    if (!b->ac) ISDF_TRY(adjoint_alloc(p));
    const int n = p->n_phi, nm = p->n_mu;
    const int64_t R = p->max_rows, Rp = (R + 7) & ~(int64_t)7;
    const size_t es = p->dtype == ISDF_C128 ? 16 : 8;
    int *err = &b->sc->err;
    bool ok = true;
    // per call: rotated K^T, Phi_mu^H, Psi_mu^H
    CUtensorMap mkh, mkl, mph, mpl, mqh, mql;
    if (!grad_theta) {
        ISDF_TRY(operand_scale<double2>(b, SC_K, static_cast<const double2 *>(K), nm, nm, nm, st));
        ISDF_TRY((transposed_operand<double2, true>(static_cast<const double2 *>(K), nm, nm, nm, 0, b->adj_sc + SC_K,
                                                    b->kh, b->kl, 2 * nm, st)));
        ok &= make_map(&mkh, b->kh, 2 * nm, 2 * nm);
        ok &= make_map(&mkl, b->kl, 2 * nm, 2 * nm);
    }
    ISDF_TRY((transposed_operand<double2, true>(p->phi_mu, n, nm, n, 1, &b->sc->s_phi, b->pmh, b->pml, 2 * nm, st)));
    ISDF_TRY((transposed_operand<double2, true>(p->psi_mu, n, nm, n, 1, &b->sc->s_psi, b->qmh, b->qml, 2 * nm, st)));
    ok &= make_map(&mph, b->pmh, 2 * nm, 2 * n);
    ok &= make_map(&mpl, b->pml, 2 * nm, 2 * n);
    ok &= make_map(&mqh, b->qmh, 2 * nm, 2 * n);
    ok &= make_map(&mql, b->qml, 2 * nm, 2 * n);
    CUtensorMap moah, moal;   // row-block A operand (rows x 2 N_mu)
    ok &= make_map(&moah, b->oah, 2 * nm, R);
    ok &= make_map(&moal, b->oal, 2 * nm, R);
    if (!ok) return ISDF_ERR_CUDA;

    for (int64_t r0 = row_begin; r0 < row_begin + row_count; r0 += R) {
        const int rows = (int)((row_begin + row_count - r0) < R ? (row_begin + row_count - r0) : R);
        const int64_t tot = (int64_t)rows * nm;
        // 1. P^phi, P^psi and the split Y of this block
        {
            EpiParams ep{};
            ep.yh = b->yh;
            ep.yl = b->yl;
            ep.ldy = 2 * nm;
            ep.aout = b->ac;
            ep.bout = b->bc;
            ep.ldab = nm;
            ep.sc = b->sc;
            ep.err = err;
            ep.budget = p->wait_budget;
            ep.ksplit = 1;
            ep.ncols = 2 * nm;
            const int n_tiles_n = (2 * nm) / TN, m_tiles = (rows + TM - 1) / TM;
            const int n_tiles = n_tiles_n * m_tiles;
            const unsigned grid = (unsigned)(n_tiles < num_sms() ? n_tiles : num_sms());
            tc_gemm_persist<true><<<grid, GEMM_THREADS, SMEM_BYTES, st>>>(
                b->m_a1h, b->m_a1l, b->m_b1h, b->m_b1l, b->m_a2h, b->m_a2l, b->m_b2h, b->m_b2l, (2 * n) / TK,
                (int)r0, rows, n_tiles_n, n_tiles, kGramSegment, ep);
            isdf_note_launch();
            ISDF_LAUNCH_CHECK();
        }
        EpiParams e{};
        e.sc = b->sc;
        e.err = err;
        e.budget = p->wait_budget;
        e.ksplit = 1;
        // 2. Theta = Y M^-1 (complex64)
        e.out_mode = OUT_C64;
        e.out = b->tc;
        e.ldo = nm;
        e.sa = &b->sc->s_y;
        e.sb = &b->sc->s_w;
        e.alpha = 1.f;
        ISDF_TRY(run_gemm(b->m_yh, b->m_yl, b->m_bwh, b->m_bwl, (2 * nm) / TK, rows, 2 * nm, e, st));
        ISDF_TRY(operand_scale<float2>(b, SC_THETA, b->tc, nm, nm, rows, st));
        // 3. G = 2 dV Theta conj(K), or the given dL/dTheta
        if (!grad_theta) {
            split_orbitals<float2><<<grid_for(tot, 152 * 64), 256, 0, st>>>(b->tc, nm, nm, rows, b->adj_sc + SC_THETA,
                                                                            b->oah, b->oal);
            isdf_note_launch();
            e.out = b->gc;
            e.sa = b->adj_sc + SC_THETA;
            e.sb = b->adj_sc + SC_K;
            e.alpha = (float)(2.0 * dV);
            ISDF_TRY(run_gemm(moah, moal, mkh, mkl, (2 * nm) / TK, rows, 2 * nm, e, st));
            if (loss) {
                loss_c64<<<grid_for(tot, 2048), 256, 0, st>>>(b->tc, b->gc, tot, loss);
                isdf_note_launch();
            }
        } else {
            ISDF_CUDA_TRY(cudaMemcpy2DAsync(b->gc, sizeof(float2) * nm,
                                            static_cast<const char *>(grad_theta) + (r0 - row_begin) * ld_grad * 8,
                                            sizeof(float2) * ld_grad, sizeof(float2) * nm, rows,
                                            cudaMemcpyDeviceToDevice, st));
        }
        // 4. Ybar = G M^-1
        ISDF_TRY(operand_scale<float2>(b, SC_G, b->gc, nm, nm, rows, st));
        split_orbitals<float2><<<grid_for(tot, 152 * 64), 256, 0, st>>>(b->gc, nm, nm, rows, b->adj_sc + SC_G, b->oah,
                                                                        b->oal);
        isdf_note_launch();
        e.out = b->ybc;
        e.sa = b->adj_sc + SC_G;
        e.sb = &b->sc->s_w;
        e.alpha = 1.f;
        ISDF_TRY(run_gemm(moah, moal, b->m_bwh, b->m_bwl, (2 * nm) / TK, rows, 2 * nm, e, st));
        // 5. Abar = Ybar o B, Bbar = conj(Ybar) o A
        hadamard_adjoint_c64<<<grid_for(tot), 256, 0, st>>>(b->ybc, b->ac, b->bc, tot);
        isdf_note_launch();
        ISDF_TRY(operand_scale<float2>(b, SC_ABAR, b->ac, nm, nm, rows, st));
        ISDF_TRY(operand_scale<float2>(b, SC_BBAR, b->bc, nm, nm, rows, st));
        ISDF_TRY(operand_scale<float2>(b, SC_YBAR, b->ybc, nm, nm, rows, st));
        // 6. grad_phi rows += Abar Phi_mu, grad_psi rows += Bbar Psi_mu
        for (int side = 0; side < 2; ++side) {
            const float2 *src = side ? b->bc : b->ac;
            const int slot = side ? SC_BBAR : SC_ABAR;
            split_orbitals<float2><<<grid_for(tot, 152 * 64), 256, 0, st>>>(src, nm, nm, rows, b->adj_sc + slot,
                                                                            b->oah, b->oal);
            isdf_note_launch();
            EpiParams g{};
            g.sc = b->sc;
            g.err = err;
            g.ksplit = 1;
            g.out_mode = OUT_ADD_C128;
            g.out = side ? static_cast<double2 *>(grad_psi) + r0 * ld_gpsi : static_cast<double2 *>(grad_phi) + r0 * ld_gphi;
            g.ldo = side ? ld_gpsi : ld_gphi;
            g.sa = b->adj_sc + slot;
            g.sb = side ? &b->sc->s_psi : &b->sc->s_phi;
            g.alpha = 1.f;
            ISDF_TRY(run_gemm(moah, moal, side ? mqh : mph, side ? mql : mpl, (2 * nm) / TK, rows, 2 * n, g, st));
        }
        // 7. Phibar_mu += Abar^H Phi_b, Psibar_mu += Bbar^H Psi_b (reductions over the block's rows)
        const int kch = (2 * rows + TK - 1) / TK;
        CUtensorMap mah, mal, mbh, mbl;
        ok &= make_map(&mah, b->oah, 2 * rows, nm, 2 * Rp);
        ok &= make_map(&mal, b->oal, 2 * rows, nm, 2 * Rp);
        for (int side = 0; side < 2 && ok; ++side) {
            const float2 *src = side ? b->bc : b->ac;
            const int slot = side ? SC_BBAR : SC_ABAR;
            ISDF_TRY((transposed_operand<float2, false>(src, nm, rows, nm, 1, b->adj_sc + slot, b->oah, b->oal, 2 * Rp,
                                                        st)));
            const void *orb = side ? p->psi : p->phi;
            const int64_t ldo = side ? p->ld_psi : p->ld_phi;
            const float *so = side ? &b->sc->s_psi : &b->sc->s_phi;
            const char *src_rows = static_cast<const char *>(orb) + r0 * ldo * es;
            if (p->dtype == ISDF_C128)
                ISDF_TRY((transposed_operand<double2, true>(reinterpret_cast<const double2 *>(src_rows), ldo, rows, n,
                                                            1, so, b->obh, b->obl, 2 * Rp, st)));
            else
                ISDF_TRY((transposed_operand<float2, true>(reinterpret_cast<const float2 *>(src_rows), ldo, rows, n, 1,
                                                           so, b->obh, b->obl, 2 * Rp, st)));
            ok &= make_map(&mbh, b->obh, 2 * rows, 2 * n, 2 * Rp);
            ok &= make_map(&mbl, b->obl, 2 * rows, 2 * n, 2 * Rp);
            if (!ok) break;
            EpiParams g{};
            g.sc = b->sc;
            g.err = err;
            g.out_mode = OUT_ATOMIC_C128;
            g.out = side ? p->gpsi_mu : p->gphi_mu;
            g.ldo = n;
            g.sa = b->adj_sc + slot;
            g.sb = so;
            g.alpha = 1.f;
            g.ksplit = ksplit_for(nm, 2 * n, kch);
            ISDF_TRY(run_gemm(mah, mal, mbh, mbl, kch, nm, 2 * n, g, st));
        }
        // 8. Mbar -= Theta^H Ybar
        if (ok) {
            ISDF_TRY((transposed_operand<float2, false>(b->tc, nm, rows, nm, 1, b->adj_sc + SC_THETA, b->oah, b->oal,
                                                        2 * Rp, st)));
            ISDF_TRY((transposed_operand<float2, true>(b->ybc, nm, rows, nm, 1, b->adj_sc + SC_YBAR, b->obh, b->obl,
                                                       2 * Rp, st)));
            ok &= make_map(&mbh, b->obh, 2 * rows, 2 * nm, 2 * Rp);
            ok &= make_map(&mbl, b->obl, 2 * rows, 2 * nm, 2 * Rp);
            EpiParams g{};
            g.sc = b->sc;
            g.err = err;
            g.out_mode = OUT_ATOMIC_C128;
            g.out = p->Mbar;
            g.ldo = nm;
            g.sa = b->adj_sc + SC_THETA;
            g.sb = b->adj_sc + SC_YBAR;
            g.alpha = -1.f;
            g.ksplit = ksplit_for(nm, 2 * nm, kch);
            if (ok) ISDF_TRY(run_gemm(mah, mal, mbh, mbl, kch, nm, 2 * nm, g, st));
        }
        if (!ok) return ISDF_ERR_CUDA;
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
    void *bufs[] = {b->a1h, b->a1l, b->a2h, b->a2l, b->b1h, b->b1l, b->b2h, b->b2l, b->bwh, b->bwl,
                    b->yh,  b->yl,  b->sc,  b->ac,  b->bc,  b->tc,  b->gc,  b->ybc, b->oah, b->oal,
                    b->obh, b->obl, b->kh,  b->kl,  b->pmh, b->pml, b->qmh, b->qml, b->adj_sc, b->adj_max};
    for (void *x : bufs)
        if (x) cudaFree(x);
    free(b);
    p->mixed = nullptr;
}


// ---------------------------------------------------------------- exchange application (Eq. v2)
struct MixedExchange {
    __half *ah, *al;      // n_r x 2 N_phi split Phi
    __half *bh, *bl;      // 2 N_mu x 2 N_phi rotated Phi_mu
    __half *hh, *hl;      // max_rows x 2 N_mu split H = (Phi_b Phi_mu^H) o V_b
    __half *qh, *ql;      // 2 N_psi x 2 N_mu rotated Psi_mu^H
    unsigned int *mx;     // max |Phi|, max rho_Phi, max |V|, max |Psi_mu| (float bits)
    float *sc;            // s_phi, s_h, s_q, f_vh = s_h / s_phi^2
    int *err;
    int64_t n_r, max_rows;
    int n_phi, n_psi, n_mu;
    CUtensorMap m_ah, m_al, m_bh, m_bl, m_hh, m_hl, m_qh, m_ql;
};

namespace {

// power-of-two scales of the exchange products from the maxima (bounds with margins):
// |Re, Im of H| <= |P| |V| <= max rho_Phi * sqrt(2) max |V| (Cauchy-Schwarz on P = Phi_b Phi_mu^H)
__global__ void exchange_scales(const unsigned int *mx, float *sc, int *err)
{
    const float ma_phi = __uint_as_float(mx[0]), mr_phi = __uint_as_float(mx[1]);
    const float ma_v = __uint_as_float(mx[2]), ma_q = __uint_as_float(mx[3]);
    const int e_phi = scale_exp(ma_phi), e_q = scale_exp(ma_q);
    const int e_h = scale_exp(mr_phi * ma_v * 1.4143f * 1.01f);
    sc[0] = ldexpf(1.f, e_phi);
    sc[1] = ldexpf(1.f, e_h);
    sc[2] = ldexpf(1.f, e_q);
    sc[3] = ldexpf(1.f, e_h - 2 * e_phi);
    if (!isfinite(ma_phi) || !isfinite(mr_phi) || !isfinite(ma_v) || !isfinite(ma_q)) atomicExch(err, 2);
}

}  // namespace

bool mixed_exchange_supported(int n_phi, int n_psi, int n_mu)
{
    return n_phi % 32 == 0 && n_phi >= 32 && n_psi % 32 == 0 && n_psi >= 32 && n_mu % 64 == 0 && n_mu >= 64;
}

isdf_status mixed_exchange_create(MixedExchange **out, int64_t n_r, int n_phi, int n_psi, int n_mu, int64_t max_rows)
{
    *out = nullptr;
    MixedExchange *x = static_cast<MixedExchange *>(calloc(1, sizeof(MixedExchange)));
    if (!x) return ISDF_ERR_CUDA;
    x->n_r = n_r;
    x->max_rows = max_rows;
    x->n_phi = n_phi;
    x->n_psi = n_psi;
    x->n_mu = n_mu;
    isdf_status s = ISDF_OK;
    auto take = [&](isdf_status t) {
        if (s == ISDF_OK) s = t;
    };
    take(halloc(&x->ah, (size_t)n_r * 2 * n_phi));
    take(halloc(&x->al, (size_t)n_r * 2 * n_phi));
    take(halloc(&x->bh, (size_t)2 * n_mu * 2 * n_phi));
    take(halloc(&x->bl, (size_t)2 * n_mu * 2 * n_phi));
    take(halloc(&x->hh, (size_t)max_rows * 2 * n_mu));
    take(halloc(&x->hl, (size_t)max_rows * 2 * n_mu));
    take(halloc(&x->qh, (size_t)2 * n_psi * 2 * n_mu));
    take(halloc(&x->ql, (size_t)2 * n_psi * 2 * n_mu));
    take(halloc(&x->mx, 4));
    take(halloc(&x->sc, 4));
    take(halloc(&x->err, 1));
    if (s == ISDF_OK && cudaMemset(x->err, 0, sizeof(int)) != cudaSuccess) s = ISDF_ERR_CUDA;
    if (s == ISDF_OK) {
        bool ok = true;
        ok &= make_map(&x->m_ah, x->ah, 2 * n_phi, n_r);
        ok &= make_map(&x->m_al, x->al, 2 * n_phi, n_r);
        ok &= make_map(&x->m_bh, x->bh, 2 * n_phi, 2 * n_mu);
        ok &= make_map(&x->m_bl, x->bl, 2 * n_phi, 2 * n_mu);
        ok &= make_map(&x->m_hh, x->hh, 2 * n_mu, max_rows);
        ok &= make_map(&x->m_hl, x->hl, 2 * n_mu, max_rows);
        ok &= make_map(&x->m_qh, x->qh, 2 * n_mu, 2 * n_psi);
        ok &= make_map(&x->m_ql, x->ql, 2 * n_mu, 2 * n_psi);
        if (!ok) s = ISDF_ERR_CUDA;
    }
    if (s == ISDF_OK &&
        (cudaFuncSetAttribute(tc_gemm_persist<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES) !=
         cudaSuccess))
        s = ISDF_ERR_CUDA;
    if (s != ISDF_OK) {
        mixed_exchange_release(x);
        return s;
    }
    *out = x;
    return ISDF_OK;
}

template <typename T>
static isdf_status exchange_operands(MixedExchange *x, const T *phi, int64_t ld_phi, const double2 *phi_mu,
                                     const double2 *psi_mu, const float2 *V, int64_t ld_v, int64_t row_begin,
                                     int64_t row_count, cudaStream_t st)
{
    const int n = x->n_phi, nm = x->n_mu;
    ISDF_CUDA_TRY(cudaMemsetAsync(x->mx, 0, 4 * sizeof(unsigned int), st));
    // every row of Phi bounds rho(r_mu); the split covers the requested rows only
    absmax_rows<T><<<grid_for(x->n_r * 32, 152 * 8), 256, 0, st>>>(phi, ld_phi, n, x->n_r, x->mx, x->mx + 1);
    absmax_rows<float2><<<grid_for(row_count * 32, 152 * 8), 256, 0, st>>>(V + row_begin * ld_v, ld_v, nm,
                                                                           row_count, x->mx + 2, nullptr);
    absmax_rows<double2><<<grid_for((int64_t)nm * 32, 152 * 8), 256, 0, st>>>(psi_mu, x->n_psi, x->n_psi, nm,
                                                                              x->mx + 3, nullptr);
    exchange_scales<<<1, 1, 0, st>>>(x->mx, x->sc, x->err);
    for (int i = 0; i < 4; ++i) isdf_note_launch();
    split_orbitals<T><<<grid_for(row_count * n), 256, 0, st>>>(phi + row_begin * ld_phi, ld_phi, n, row_count, x->sc,
                                                              x->ah + row_begin * 2 * n, x->al + row_begin * 2 * n);
    build_rotated<<<grid_for((int64_t)nm * n), 256, 0, st>>>(phi_mu, n, nm, n, x->sc, x->bh, x->bl);
    // B of the second product: rotated X = Psi_mu^H, i.e. x[mu][j] = conj(Psi_mu[mu][j]) read transposed
    dim3 tg((nm + 31) / 32, (x->n_psi + 31) / 32);
    split_transposed<double2, true><<<tg, 256, 0, st>>>(psi_mu, x->n_psi, nm, x->n_psi, 1, x->sc + 2, x->qh, x->ql,
                                                         2 * (int64_t)nm);
    for (int i = 0; i < 3; ++i) isdf_note_launch();
    ISDF_LAUNCH_CHECK();
    return ISDF_OK;
}

isdf_status mixed_exchange_apply(MixedExchange *x, const void *phi, int64_t ld_phi, int orb_dtype,
                                 const double2 *phi_mu, const double2 *psi_mu, const float2 *V, int64_t ld_v,
                                 int64_t row_begin, int64_t row_count, double2 *out, int64_t ld_out, cudaStream_t st)
{
    const int n = x->n_phi, nm = x->n_mu;
    if (orb_dtype == ISDF_C128)
        ISDF_TRY(exchange_operands<double2>(x, static_cast<const double2 *>(phi), ld_phi, phi_mu, psi_mu, V, ld_v,
                                            row_begin, row_count, st));
    else
        ISDF_TRY(exchange_operands<float2>(x, static_cast<const float2 *>(phi), ld_phi, phi_mu, psi_mu, V, ld_v,
                                           row_begin, row_count, st));
    for (int64_t r0 = row_begin; r0 < row_begin + row_count; r0 += x->max_rows) {
        const int rows = (int)((row_begin + row_count - r0) < x->max_rows ? (row_begin + row_count - r0) : x->max_rows);
        // H_b = (Phi_b Phi_mu^H) o V_b, split for the next product
        EpiParams e1{};
        e1.out_mode = OUT_SPLIT_HV;
        e1.yh = x->hh;
        e1.yl = x->hl;
        e1.ldy = 2 * nm;
        e1.vmat = V + r0 * ld_v;
        e1.ldv = ld_v;
        e1.fvh = x->sc + 3;
        e1.err = x->err;
        e1.ksplit = 1;
        e1.ncols = 2 * nm;
        const int n_tiles_n = (2 * nm) / TN, m_tiles = (rows + TM - 1) / TM;
        const int n_tiles = n_tiles_n * m_tiles;
        const unsigned grid = (unsigned)(n_tiles < num_sms() ? n_tiles : num_sms());
        tc_gemm_persist<false><<<grid, GEMM_THREADS, SMEM_BYTES, st>>>(x->m_ah, x->m_al, x->m_bh, x->m_bl, x->m_ah,
                                                                       x->m_al, x->m_bh, x->m_bl, (2 * n) / TK, (int)r0,
                                                                       rows, n_tiles_n, n_tiles, kGramSegment, e1);
        isdf_note_launch();
        ISDF_LAUNCH_CHECK();
        // out_b = -H_b Psi_mu
        EpiParams e2{};
        e2.out_mode = OUT_C128;
        e2.out = out + (r0 - row_begin) * ld_out;
        e2.ldo = ld_out;
        e2.sa = x->sc + 1;
        e2.sb = x->sc + 2;
        e2.alpha = -1.f;
        e2.err = x->err;
        e2.ksplit = 1;
        ISDF_TRY(run_gemm(x->m_hh, x->m_hl, x->m_qh, x->m_ql, (2 * nm) / TK, rows, 2 * x->n_psi, e2, st));
    }
    return ISDF_OK;
}

int mixed_exchange_error(MixedExchange *x)
{
    int h = 0;
    if (cudaMemcpy(&h, x->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return ISDF_ERR_CUDA;
    return h == 1 ? ISDF_ERR_TIMEOUT : (h == 2 ? ISDF_ERR_NONFINITE : 0);
}

void mixed_exchange_release(MixedExchange *x)
{
    if (!x) return;
    void *bufs[] = {x->ah, x->al, x->bh, x->bl, x->hh, x->hl, x->qh, x->ql, x->mx, x->sc, x->err};
    for (void *b : bufs)
        if (b) cudaFree(b);
    free(x);
}
