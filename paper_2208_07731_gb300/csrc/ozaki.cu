// FP64 complex GEMM on the tcgen05 tensor cores by exact integer slicing
// (Ozaki, Ogita, Oishi and Rump, 2012; on FP16 tensor cores whose integer
// products are exact: Mukunoki, Ozaki, Ogita and Imamura, 2020).
//
// Real form: an interleaved complex row of op(A) is a real row of length 2K;
// for x = conj(op(B)(k, n)) the rotated real rows
//     Bh[2n] = (Re x, Im x, ...),   Bh[2n+1] = (-Im x, Re x, ...)
// make (A Bh^T)[m][2n + p] part p of (op(A) op(B))[m][n].
//
// Slicing: every real row r gets E_r with max |x| < 2^E_r, and each entry is
// rounded to F = round(x 2^(56 - E_r)) and written in balanced base 256,
// F = sum_{s=1..7} d_s 2^(56 - 8 s) with d_2..d_7 in [-128, 127] and
// |d_1| <= 256, so x = sum_s d_s 2^(E_r - 8 s) up to a rounding below
// 2^(E_r - 57); integer operations only, no FP64 arithmetic.
//
// Products: for every pair (s, t) with s + t <= 8 (28 pairs), the FP16 GEMM
// of the digit matrices over a K segment of 256 real terms is a sum of
// integers of magnitude at most 256 * 256 * 128 = 2^23, exact in the FP32
// accumulator in any order. The epilogue converts each segment to int32 and
// adds the segments of one group g = s + t exactly, then adds
// alpha 2^(E_m + E_n - 8 g) times that integer to the FP64 output. The
// neglected pairs (s + t > 8, digits of either sign) and the rounding of the
// operands stay below ~2^-55 K max|a| max|b| per output, the size of an
// FP64 GEMM's rounding error.
//
// Kernel: persistent, one CTA per SM, 320 threads - a TMA warp (6-stage ring
// of one 128 x 64 digit tile of A and one of B), an MMA warp (one elected
// thread issues tcgen05.mma kind::f16, M = N = 128) and 8 epilogue warps; the
// TMEM accumulator is double buffered per K segment. Every wait is bounded.
#include <cudaTypedefs.h>

#include "ozaki.cuh"
#include "tc.cuh"

namespace {

constexpr int OTM = 128, OTN = 128, OTK = 64;   // tile rows, tile real columns, K chunk (halves)
constexpr int OSTAGES = 6;
constexpr int OTILE = OTM * OTK * 2;            // bytes of one digit tile
constexpr int OSTAGE = 2 * OTILE;
constexpr int OSMEM = OSTAGES * OSTAGE + 1024;
constexpr int NSLICE = 7, BETA = 8, GMAX = NSLICE + 1;
constexpr int SEG = 4;                           // K chunks per TMEM accumulation (256 real terms)
constexpr int FLUSH_AT = 200;                    // pair-segments per int32 group sum (200 * 2^23 < 2^31)
constexpr int OEPI = 8;
constexpr int OTHREADS = 64 + 32 * OEPI;
constexpr long long OWAIT = 200000000LL;         // SM cycles (~0.1 s)

struct OzArgs {
    int M, N, K;            // complex sizes
    int Ra, Rb;             // padded real rows of one slice of A / of Bh
    int kchunks;            // padded real K / 64
    int batch, n_tm, n_tn;  // tiles per batch product
    int kmode, k_to_m_end, lower_only, beta;
    double alpha;
    double2 *C;
    int64_t ldc, bsc;
    const unsigned long long *ma, *mb;   // row maxima (batch-major: M and N per product)
    int *gsum;              // buffered epilogue: exact group sums [b][g - 2][M][2N] (int32), or NULL
    int *err;               // 1: a bounded wait gave up; 2: a non-finite operand entry
    long long budget;       // cycle budget of the pipeline waits (the drain waits keep OWAIT)
    long long never;        // > 0: test hook, the MMA issuer first waits this long on a barrier nothing signals
};

__device__ __forceinline__ int row_exp(unsigned long long maxbits) { return (int)(maxbits >> 52) - 1022; }

// 2^e as a double (ldexp for the rare exponents outside the normal range)
__device__ __forceinline__ double pow2(int e)
{
    if (e < -1022 || e > 1023) return ldexp(1.0, e);
    return __longlong_as_double((long long)(e + 1023) << 52);
}

// the 7 balanced base-256 digits of x relative to 2^E (|x| < 2^E), from the bits of x:
// F = round(x 2^(56 - E)) (half away from zero), then d_7 .. d_2 in [-128, 127] taken from
// the bottom and d_1 = what remains (|d_1| <= 256), so that x ~ sum_s d_s 2^(E - 8 s)
__device__ __forceinline__ void digits(double x, int E, int (&d)[NSLICE])
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ef = (int)((b >> 52) & 0x7FF);
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (ef ? (1ull << 52) : 0ull);
    const int sh = (ef ? ef : 1) - 1019 - E;   // |x| 2^(56 - E) = m 2^sh
    long long f = 0;
    if (sh >= 0 && sh < 8) f = (long long)(m << sh);
    else if (sh < 0 && sh > -64) f = (long long)((m + (1ull << (-sh - 1))) >> (-sh));
    if (b >> 63) f = -f;
#pragma unroll
    for (int s = NSLICE - 1; s > 0; --s) {
        const long long r = ((f + 128) & 255) - 128;
        d[s] = (int)r;
        f = (f - r) >> 8;
    }
    d[0] = (int)f;
}

// complex128 entry, or complex64 widened exactly by moving bits (no FP64 instruction)
__device__ __forceinline__ double2 load_c(const double2 *p, int64_t i) { return p[i]; }
__device__ __forceinline__ double2 load_c(const float2 *p, int64_t i)
{
    const float2 v = p[i];
    return make_double2(f2d_int(v.x), f2d_int(v.y));
}

// per-row max |Re|, |Im| (as double bits) of the operand rows r, entries X[r sr + k sk],
// one 32 x 32 (r, k) tile per block of 32 x 8 threads, batch in blockIdx.z
template <typename T>
__global__ void oz_rowmax(const T *X, int64_t sr, int64_t sk, int64_t bsx, int R, int K, unsigned long long *maxbits,
                          int *err)
{
    __shared__ unsigned long long t[32][33];
    const int k0 = blockIdx.x * 32, r0 = blockIdx.y * 32, b = blockIdx.z;
    const T *Xb = X + (int64_t)b * bsx;
    const bool kfast = (sk == 1);
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int r = kfast ? r0 + i : r0 + (int)threadIdx.x, k = kfast ? k0 + (int)threadIdx.x : k0 + i;
        unsigned long long v = 0ull;
        if (r < R && k < K) {
            const double2 x = load_c(Xb, (int64_t)r * sr + (int64_t)k * sk);
            const unsigned long long a = (unsigned long long)__double_as_longlong(x.x) & 0x7FFFFFFFFFFFFFFFull;
            const unsigned long long c = (unsigned long long)__double_as_longlong(x.y) & 0x7FFFFFFFFFFFFFFFull;
            v = a > c ? a : c;
        }
        if (kfast) t[i][threadIdx.x] = v;
        else t[threadIdx.x][i] = v;
    }
    __syncthreads();
    if (threadIdx.y == 0) {
        unsigned long long m = 0ull;
        for (int j = 0; j < 32; ++j) m = t[threadIdx.x][j] > m ? t[threadIdx.x][j] : m;
        const int r = r0 + (int)threadIdx.x;
        if (r < R && m) atomicMax(&maxbits[(int64_t)b * R + r], m);
        // an infinity or NaN (exponent field all ones) cannot be sliced: recorded, not computed on
        if (m >= 0x7FF0000000000000ull) atomicCAS(err, 0, 2);
    }
}

// digit slices of the operand rows: plain (A role: real row r = (Re, Im) interleaved over k)
// or rotated (B role: rows 2r and 2r+1 of Bh for x = value); slice s of row r of product b
// at out[((b NSLICE + s) Rp + row) Kp + column]
template <typename T>
__global__ void oz_slice(const T *X, int64_t sr, int64_t sk, int64_t bsx, int R, int K, int conj, int rotated,
                         const unsigned long long *maxbits, __half *out, int64_t Rp, int64_t Kp)
{
    __shared__ double2 t[32][33];
    const int k0 = blockIdx.x * 32, r0 = blockIdx.y * 32, b = blockIdx.z;
    const T *Xb = X + (int64_t)b * bsx;
    const bool kfast = (sk == 1);
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int r = kfast ? r0 + i : r0 + (int)threadIdx.x, k = kfast ? k0 + (int)threadIdx.x : k0 + i;
        double2 v = make_double2(0.0, 0.0);
        if (r < R && k < K) {
            v = load_c(Xb, (int64_t)r * sr + (int64_t)k * sk);
            if (conj) v.y = -v.y;
        }
        if (kfast) t[i][threadIdx.x] = v;
        else t[threadIdx.x][i] = v;
    }
    __syncthreads();
    __half2 *o2 = reinterpret_cast<__half2 *>(out);
    const int64_t kp2 = Kp / 2;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int r = r0 + i, k = k0 + (int)threadIdx.x;
        if (r >= R || k >= K) continue;
        const double2 v = t[i][threadIdx.x];
        const int E = row_exp(maxbits[(int64_t)b * R + r]);
        int dx[NSLICE], dy[NSLICE];
        digits(v.x, E, dx);
        digits(v.y, E, dy);
#pragma unroll
        for (int s = 0; s < NSLICE; ++s) {
            const int64_t sl = (int64_t)b * NSLICE + s;
            if (!rotated) {
                o2[(sl * Rp + r) * kp2 + k] = __halves2half2(__int2half_rn(dx[s]), __int2half_rn(dy[s]));
            } else {
                o2[(sl * Rp + 2 * r) * kp2 + k] = __halves2half2(__int2half_rn(dx[s]), __int2half_rn(dy[s]));
                o2[(sl * Rp + 2 * r + 1) * kp2 + k] = __halves2half2(__int2half_rn(-dy[s]), __int2half_rn(dx[s]));
            }
        }
    }
}

// the K range of a tile in chunks of 64 real terms (complex rows m0.., complex columns c0..)
__device__ __forceinline__ void tile_krange(const OzArgs &a, int m0, int c0, int &kb, int &ke)
{
    int kmin = 0, kmax = a.K;
    if (a.kmode == ZG_K_FROM_MAX_MN) kmin = max(m0, c0);
    else if (a.kmode == ZG_K_FROM_N0) kmin = c0;
    if (a.k_to_m_end) kmax = min(kmax, m0 + OTM);
    kb = (2 * kmin) / OTK;
    ke = (2 * kmax + OTK - 1) / OTK;
    if (ke > a.kchunks) ke = a.kchunks;
}

// decode work item t: batch b, complex row start m0, real column start n0; false if skipped
__device__ __forceinline__ bool tile_of(const OzArgs &a, int t, int &b, int &m0, int &n0)
{
    const int per = a.n_tm * a.n_tn;
    b = t / per;
    const int rem = t % per;
    m0 = (rem / a.n_tn) * OTM;
    n0 = (rem % a.n_tn) * OTN;
    return !(a.lower_only && n0 / 2 > m0 + OTM - 1);
}

__global__ void __launch_bounds__(OTHREADS, 1)
    oz_gemm(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, OzArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[OSTAGES];
    __shared__ __align__(8) uint64_t empty_bar[OSTAGES];
    __shared__ __align__(8) uint64_t tfull[2];
    __shared__ __align__(8) uint64_t tempty[2];
    __shared__ __align__(8) uint64_t drain_bar;
    __shared__ __align__(8) uint64_t never_bar;   // signalled by nothing (the test hook waits on it)
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int failed;

    if (*(volatile int *)a.err) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t raw = tc::smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *sbase = smem_raw + (base - raw);
    const int n_work = a.batch * a.n_tm * a.n_tn;

    if (threadIdx.x == 0) {
        for (int s = 0; s < OSTAGES; ++s) {
            tc::mbar_init(&full_bar[s], 1);
            tc::mbar_init(&empty_bar[s], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&tfull[i], 1);
            tc::mbar_init(&tempty[i], OEPI);
        }
        tc::mbar_init(&drain_bar, 1);
        tc::mbar_init(&never_bar, 1);
        failed = 0;
        tc::fence_barrier_init();
    }
    if (warp == 0) tc::tmem_alloc(&tmem_slot, 2 * OTN);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            tc::prefetch_map(&ta);
            tc::prefetch_map(&tb);
            int c = 0, issued = 0;
            for (int t = blockIdx.x; t < n_work && !failed; t += gridDim.x) {
                int b, m0, n0, kb, ke;
                if (!tile_of(a, t, b, m0, n0)) continue;
                tile_krange(a, m0, n0 / 2, kb, ke);
                for (int g = 2; g <= GMAX && !failed; ++g)
                    for (int s = max(1, g - NSLICE); s <= min(NSLICE, g - 1) && !failed; ++s) {
                        const int ya = (b * NSLICE + s - 1) * a.Ra + m0, yb = (b * NSLICE + g - s - 1) * a.Rb + n0;
                        for (int kc = kb; kc < ke; ++kc, ++c) {
                            const int st = c % OSTAGES, it = c / OSTAGES;
                            if (!tc::mbar_wait(&empty_bar[st], (it & 1) ^ 1, a.budget)) {
                                atomicExch(a.err, 1);
                                failed = 1;
                                break;
                            }
                            uint8_t *sp = sbase + st * OSTAGE;
                            tc::mbar_expect_tx(&full_bar[st], OSTAGE);
                            tc::tma_load_2d(sp, &ta, &full_bar[st], kc * OTK, ya);
                            tc::tma_load_2d(sp + OTILE, &tb, &full_bar[st], kc * OTK, yb);
                            issued = c + 1;
                        }
                    }
            }
            for (int c2 = issued - OSTAGES > 0 ? issued - OSTAGES : 0; c2 < issued; ++c2)
                tc::mbar_wait(&full_bar[c2 % OSTAGES], (c2 / OSTAGES) & 1, OWAIT);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_f16(OTM, OTN);
            int c = 0, tl = 0;
            bool ok = true;
            if (a.never > 0 && !tc::mbar_wait(&never_bar, 0, a.never)) {
                atomicExch(a.err, 1);
                failed = 1;
                ok = false;
            }
            for (int t = blockIdx.x; t < n_work && ok && !failed; t += gridDim.x) {
                int b, m0, n0, kb, ke;
                if (!tile_of(a, t, b, m0, n0)) continue;
                tile_krange(a, m0, n0 / 2, kb, ke);
                for (int g = 2; g <= GMAX && ok; ++g)
                    for (int s = max(1, g - NSLICE); s <= min(NSLICE, g - 1) && ok; ++s)
                        for (int s0 = kb; s0 < ke && ok; s0 += SEG, ++tl) {
                            const int acc = tl & 1, use = tl >> 1;
                            if (!tc::mbar_wait(&tempty[acc], (use & 1) ^ 1, a.budget)) {
                                atomicExch(a.err, 1);
                                failed = 1;
                                ok = false;
                                break;
                            }
                            tc::fence_after();
                            const uint32_t d = tmem + (uint32_t)acc * OTN;
                            const int s1 = min(ke, s0 + SEG);
                            for (int kc = s0; kc < s1; ++kc, ++c) {
                                const int st = c % OSTAGES, it = c / OSTAGES;
                                if (!tc::mbar_wait(&full_bar[st], it & 1, a.budget)) {
                                    atomicExch(a.err, 1);
                                    failed = 1;
                                    ok = false;
                                    break;
                                }
                                tc::fence_after();
                                const uint32_t sa = base + st * OSTAGE;
                                const uint64_t da = tc::desc_sw128(sa), db = tc::desc_sw128(sa + OTILE);
#pragma unroll
                                for (int kk = 0; kk < OTK / 16; ++kk)
                                    tc::mma_f16(d, da + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk), idesc,
                                                (kc > s0 || kk > 0) ? 1u : 0u);
                                tc::mma_commit(&empty_bar[st]);
                            }
                            if (!ok) break;
                            tc::mma_commit(&tfull[acc]);
                        }
            }
            tc::mma_commit(&drain_bar);
            tc::mbar_wait(&drain_bar, 0, OWAIT);
        }
        __syncwarp();
    } else {
        const int quarter = warp & 3;          // TMEM lane quarter this warp may access
        const int half = (warp - 2) >> 2;      // which 64 of the tile's 128 real columns
        int tl = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < n_work && ok && !failed; t += gridDim.x) {
            int b, m0, n0, kb, ke;
            if (!tile_of(a, t, b, m0, n0)) continue;
            tile_krange(a, m0, n0 / 2, kb, ke);
            const int row = m0 + quarter * 32 + lane;
            const int cb = n0 / 2 + half * 32;   // first complex column of this thread
            const bool rv = row < a.M;
            double2 *crow = a.C + (int64_t)b * a.bsc + (int64_t)row * a.ldc;
            const int ea = rv ? row_exp(a.ma[(int64_t)b * a.M + row]) : 0;
            bool first = true;   // no group added to C yet: C = beta C + ...
            if (kb >= ke) {      // empty K range: the product is zero
                if (rv && !a.beta)
                    for (int j = 0; j < 32; ++j)
                        if (cb + j < a.N) crow[cb + j] = make_double2(0.0, 0.0);
                continue;
            }
            for (int g = 2; g <= GMAX && ok; ++g) {
                int acc32[64];
#pragma unroll
                for (int i = 0; i < 64; ++i) acc32[i] = 0;
                int pending = 0;
                const int s_lo = max(1, g - NSLICE), s_hi = min(NSLICE, g - 1);
                for (int s = s_lo; s <= s_hi && ok; ++s)
                    for (int s0 = kb; s0 < ke; s0 += SEG, ++tl) {
                        const int accb = tl & 1, use = tl >> 1;
                        if (!tc::mbar_wait(&tfull[accb], use & 1, a.budget)) {
                            atomicExch(a.err, 1);
                            failed = 1;
                            ok = false;
                            break;
                        }
                        tc::fence_after();
                        const uint32_t ta0 = tmem + (uint32_t)accb * OTN + ((uint32_t)(quarter * 32) << 16) + half * 64;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            uint32_t r[16];
                            tc::tmem_ld16(ta0 + 16 * j, r);
                            tc::tmem_wait_ld();
#pragma unroll
                            for (int q = 0; q < 16; ++q) acc32[16 * j + q] += __float2int_rn(__uint_as_float(r[q]));
                        }
                        tc::fence_before();
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(&tempty[accb]);
                        ++pending;
                        const bool last = (s == s_hi) && (s0 + SEG >= ke);
                        if (a.gsum && last) {
                            // buffered: the group's exact sums go out as integers; oz_combine
                            // forms the FP64 result (no FP64 work and no reads of C here)
                            if (rv) {
                                int *gr = a.gsum + (((int64_t)b * NSLICE + (g - 2)) * a.M + row) * (2 * (int64_t)a.N);
                                const int c0r = 2 * cb;
                                if (c0r + 64 <= 2 * a.N && (a.N % 2) == 0) {
#pragma unroll
                                    for (int q = 0; q < 16; ++q)
                                        reinterpret_cast<int4 *>(gr + c0r)[q] =
                                            make_int4(acc32[4 * q], acc32[4 * q + 1], acc32[4 * q + 2], acc32[4 * q + 3]);
                                } else {
#pragma unroll
                                    for (int q = 0; q < 64; ++q)
                                        if (c0r + q < 2 * a.N) gr[c0r + q] = acc32[q];
                                }
                            }
                            pending = 0;
#pragma unroll
                            for (int i = 0; i < 64; ++i) acc32[i] = 0;
                        } else if (!a.gsum && (pending == FLUSH_AT || last)) {
                            // C += alpha 2^(E_row + E_col - 8 g) * (exact integer sum)
                            if (rv) {
#pragma unroll
                                for (int j = 0; j < 32; ++j) {
                                    const int cc = cb + j;
                                    if (cc >= a.N) continue;
                                    const int eb = row_exp(a.mb[(int64_t)b * a.N + cc]);
                                    const double sc = a.alpha * pow2(ea + eb - BETA * g);
                                    double2 o = make_double2(0.0, 0.0);
                                    if (!first || a.beta) o = crow[cc];
                                    o.x = fma((double)acc32[2 * j], sc, o.x);
                                    o.y = fma((double)acc32[2 * j + 1], sc, o.y);
                                    crow[cc] = o;
                                }
                            }
                            first = false;
                            pending = 0;
#pragma unroll
                            for (int i = 0; i < 64; ++i) acc32[i] = 0;
                        }
                    }
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 2 * OTN);
}

// FP64 result of a buffered product: C = beta C + alpha sum_g 2^(E_m + E_n - 8 g) S_g, one
// thread per complex output of the computed tiles (the GEMM's tile and K-range rules)
__global__ void oz_combine(OzArgs a)
{
    const int64_t total = (int64_t)a.batch * a.M * a.N;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(e / ((int64_t)a.M * a.N));
        const int64_t rem = e % ((int64_t)a.M * a.N);
        const int row = (int)(rem / a.N), c = (int)(rem % a.N);
        const int m0 = (row / OTM) * OTM, n0 = ((2 * c) / OTN) * OTN;
        if (a.lower_only && n0 / 2 > m0 + OTM - 1) continue;   // tile not computed: C untouched
        int kb, ke;
        tile_krange(a, m0, n0 / 2, kb, ke);
        double2 *cp = a.C + (int64_t)b * a.bsc + (int64_t)row * a.ldc + c;
        double2 o = a.beta ? *cp : make_double2(0.0, 0.0);
        if (kb < ke) {
            const int ea = row_exp(a.ma[(int64_t)b * a.M + row]), eb = row_exp(a.mb[(int64_t)b * a.N + c]);
            const int *gp = a.gsum + ((int64_t)b * NSLICE * a.M + row) * (2 * (int64_t)a.N) + 2 * c;
            const int64_t gstride = (int64_t)a.M * 2 * a.N;
            double vx = 0.0, vy = 0.0;
#pragma unroll
            for (int g = 2; g <= GMAX; ++g) {
                const int2 sg = *reinterpret_cast<const int2 *>(gp + (g - 2) * gstride);
                const double sc = pow2(ea + eb - BETA * g);
                vx = fma((double)sg.x, sc, vx);
                vy = fma((double)sg.y, sc, vy);
            }
            o.x = fma(a.alpha, vx, o.x);
            o.y = fma(a.alpha, vy, o.y);
        }
        *cp = o;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 oz_encode()
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

bool oz_map(CUtensorMap *m, const void *base, uint64_t inner, uint64_t rows)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = oz_encode();
    if (!enc) return false;
    cuuint64_t dims[2] = {inner, rows};
    cuuint64_t strides[1] = {inner * 2};
    cuuint32_t box[2] = {OTK, OTM};
    cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int oz_sms()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    }
    return n;
}

isdf_status oz_attributes()
{
    static bool done[64] = {false};
    int dev = 0;
    ISDF_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return ISDF_ERR_CUDA;
    if (done[dev]) return ISDF_OK;
    ISDF_CUDA_TRY(cudaFuncSetAttribute(oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, OSMEM));
    done[dev] = true;
    return ISDF_OK;
}

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace

void oz_sizes(int M, int N, int K, int batch, size_t *halves_a, size_t *halves_b, size_t *rows_a, size_t *rows_b)
{
    const int64_t Ra = round_up(M, OTM), Rb = round_up(2 * (int64_t)N, OTN), Kp = round_up(2 * (int64_t)K, OTK);
    *halves_a = (size_t)batch * NSLICE * Ra * Kp;
    *halves_b = (size_t)batch * NSLICE * Rb * Kp;
    *rows_a = (size_t)batch * M;
    *rows_b = (size_t)batch * N;
}

bool oz_fits(const ZGemm &g, const OzWork &w)
{
    if (g.dual || g.ctype != ZG_C128 || g.scn != 1) return false;
    if (g.M < 1 || g.N < 1 || g.K < 1 || !w.sa || !w.sb || !w.ma || !w.mb) return false;
    const int batch = g.batch > 1 ? g.batch : 1;
    size_t ha, hb, ra, rb;
    oz_sizes(g.M, g.N, g.K, batch, &ha, &hb, &ra, &rb);
    return ha <= w.cap_a && hb <= w.cap_b && ra <= w.cap_ma && rb <= w.cap_mb;
}

isdf_status oz_zgemm(const ZGemm &g, const OzWork &w, int *err, cudaStream_t st)
{
    if (!oz_fits(g, w) || !err) return ISDF_ERR_INVALID_ARG;
    ISDF_TRY(oz_attributes());
    const int batch = g.batch > 1 ? g.batch : 1;
    const int64_t Ra = round_up(g.M, OTM), Rb = round_up(2 * (int64_t)g.N, OTN), Kp = round_up(2 * (int64_t)g.K, OTK);
    // zero padding rows / columns only when they exist
    if (Ra != g.M || Kp != 2 * (int64_t)g.K)
        ISDF_CUDA_TRY(cudaMemsetAsync(w.sa, 0, sizeof(__half) * (size_t)batch * NSLICE * Ra * Kp, st));
    if (Rb != 2 * (int64_t)g.N || Kp != 2 * (int64_t)g.K)
        ISDF_CUDA_TRY(cudaMemsetAsync(w.sb, 0, sizeof(__half) * (size_t)batch * NSLICE * Rb * Kp, st));
    ISDF_CUDA_TRY(cudaMemsetAsync(w.ma, 0, sizeof(unsigned long long) * (size_t)batch * g.M, st));
    ISDF_CUDA_TRY(cudaMemsetAsync(w.mb, 0, sizeof(unsigned long long) * (size_t)batch * g.N, st));
    const dim3 blk(32, 8);
    // A role: rows m, entries A[m s0 + k s1]; B role: rows n, entries B[k s0 + n s1]
    const dim3 ga((g.K + 31) / 32, (g.M + 31) / 32, batch), gb((g.K + 31) / 32, (g.N + 31) / 32, batch);
    auto slice = [&](const ZOperand &o, dim3 grid, int64_t sr, int64_t sk, int64_t bs, int R, int conj, int rot,
                     unsigned long long *mx, __half *out, int64_t Rp) {
        if (o.type == ZG_C64) {
            const float2 *X = static_cast<const float2 *>(o.p);
            oz_rowmax<float2><<<grid, blk, 0, st>>>(X, sr, sk, bs, R, g.K, mx, err);
            isdf_note_launch();
            oz_slice<float2><<<grid, blk, 0, st>>>(X, sr, sk, bs, R, g.K, conj, rot, mx, out, Rp, Kp);
            isdf_note_launch();
        } else {
            const double2 *X = static_cast<const double2 *>(o.p);
            oz_rowmax<double2><<<grid, blk, 0, st>>>(X, sr, sk, bs, R, g.K, mx, err);
            isdf_note_launch();
            oz_slice<double2><<<grid, blk, 0, st>>>(X, sr, sk, bs, R, g.K, conj, rot, mx, out, Rp, Kp);
            isdf_note_launch();
        }
    };
    slice(g.A1, ga, g.A1.s0, g.A1.s1, g.bsa, g.M, g.A1.conj, 0, w.ma, w.sa, Ra);
    // Bh is built from x = conj(op(B))
    slice(g.B1, gb, g.B1.s1, g.B1.s0, g.bsb, g.N, !g.B1.conj, 1, w.mb, w.sb, Rb);
    ISDF_LAUNCH_CHECK();
    CUtensorMap ta, tb;
    if (!oz_map(&ta, w.sa, (uint64_t)Kp, (uint64_t)batch * NSLICE * Ra) ||
        !oz_map(&tb, w.sb, (uint64_t)Kp, (uint64_t)batch * NSLICE * Rb))
        return ISDF_ERR_CUDA;
    OzArgs a;
    a.M = g.M;
    a.N = g.N;
    a.K = g.K;
    a.Ra = (int)Ra;
    a.Rb = (int)Rb;
    a.kchunks = (int)(Kp / OTK);
    a.batch = batch;
    a.n_tm = (int)(Ra / OTM);
    a.n_tn = (int)(Rb / OTN);
    a.kmode = g.kmode;
    a.k_to_m_end = g.k_to_m_end;
    a.lower_only = g.lower_only;
    a.beta = g.beta;
    a.alpha = g.alpha;
    a.C = static_cast<double2 *>(g.C);
    a.ldc = g.scm;
    a.bsc = g.bsc;
    a.ma = w.ma;
    a.mb = w.mb;
    a.err = err;
    a.budget = w.wait_budget > 0 ? w.wait_budget : OWAIT;
    a.never = w.wait_budget < 0 ? -w.wait_budget : 0;
    // buffered epilogue when the group sums fit the scratch and no group needs a partial flush
    const int64_t segs = (a.kchunks + SEG - 1) / SEG;
    const size_t gneed = (size_t)batch * NSLICE * g.M * 2 * (size_t)g.N;
    a.gsum = (w.gsum && gneed <= w.cap_g && NSLICE * segs <= FLUSH_AT) ? w.gsum : nullptr;
    const int work = batch * a.n_tm * a.n_tn;
    const unsigned grid = (unsigned)(work < oz_sms() ? work : oz_sms());
    oz_gemm<<<grid, OTHREADS, OSMEM, st>>>(ta, tb, a);
    isdf_note_launch();
    if (a.gsum) {
        const int64_t tot = (int64_t)batch * g.M * g.N;
        const unsigned gc = (unsigned)((tot + 255) / 256 < 8192 ? (tot + 255) / 256 : 8192);
        oz_combine<<<gc, 256, 0, st>>>(a);
        isdf_note_launch();
    }
    ISDF_LAUNCH_CHECK();
    return ISDF_OK;
}
