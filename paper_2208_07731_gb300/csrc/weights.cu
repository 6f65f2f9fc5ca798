// Step 1: the K-means weight function (Sec. 2.2, Eq. weight function 2 for
// SSM and its alpha family, Eq. weight function for PSM).
//
// Every sum of the weight is the exact sum of its terms rounded once, so the
// result does not depend on summation order (and equals the oracle bit for
// bit). For alpha = 2 the terms are the exact squares x^2 of the real
// components x = Re z, Im z: with E = max floor(log2|x|) over the row's
// non-zero components,
//     sum = RN( sum_x floor(x^2 2^(110 - 2E)) ) 2^(2E - 110),
// where x = m 2^p (integer mantissa m, exponent p of its format) makes each
// term the integer m^2 shifted by 2p + 110 - 2E, accumulated in 128 bits with
// integer instructions only. For alpha != 2 the terms are |z|^alpha in FP64
// and the same exact summation runs on floor(t 2^(110 - E_t)).
//
// One warp owns one grid row: pass 1 reads the row and reduces the exponent
// window E, pass 2 reads it again (from L1/L2: the row was just read) and
// accumulates; the 128-bit lane sums are added across the warp with carries.
// GB300 issues FP64 at about 2 operations per clock per SM, so the integer
// formulation keeps the kernel on the memory system instead of the FP64 pipe.
//
// Complex64 rows take a shorter integer path. A float component x = m 2^p
// (p = max(b, 1) - 150 for the biased exponent b) has the term
// floor((m 2^k)^2) with k = p + 55 - E. Whenever k >= 0 (every normal
// component within 2^32 of the row maximum) y = m 2^k is an integer below
// 2^56, and with y = yh 2^28 + yl,
//     y^2 = yh^2 2^56 + yh yl 2^29 + yl^2,
// three products below 2^56 that each lane sums in plain 64-bit registers
// (128 of them stay below 2^63) and folds into its 128-bit sum every 128
// terms. Pass 1 finds the smallest magnitude of the row as well as the
// largest; a row whose components are all normal with k >= 0 runs a loop
// without branches (k <= 32 there, so yh and yl are two clamped funnel
// shifts of m 2^4), any other row checks each component and gives zeros,
// subnormals and components with k < 0 (whose term is floored) the general
// formula. The integer sum, hence the weight, is the same either way. Pass 1
// marks the row's L2 lines evict-last and pass 2 evict-first, so that the
// second read finds them in L2.
#include <type_traits>

#include "common.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kNoExp = -0x40000000;   // no non-zero component seen

struct U128 {
    unsigned long long lo, hi;
};

// L2 eviction priorities for the two reads of a row: the first read marks its lines evict-last so
// that they are still in L2 for the second, which marks them evict-first
__device__ __forceinline__ unsigned long long l2_evict_last()
{
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ unsigned long long l2_evict_first()
{
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ uint4 ld_policy(const uint4 *p, unsigned long long pol)
{
    uint4 r;
    asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p), "l"(pol));
    return r;
}

__device__ __forceinline__ void add_u128(U128 &a, unsigned long long lo, unsigned long long hi)
{
    const unsigned long long l = a.lo + lo;
    a.hi += hi + (l < lo ? 1ull : 0ull);
    a.lo = l;
}

// a += floor(v 2^sh) for a 64-bit v and sh <= 64
__device__ __forceinline__ void add_shifted64(U128 &a, unsigned long long v, int sh)
{
    if (sh >= 0) {
        if (sh == 0) add_u128(a, v, 0ull);
        else if (sh < 64) add_u128(a, v << sh, v >> (64 - sh));
        else add_u128(a, 0ull, v);
    } else if (sh > -64) {
        add_u128(a, v >> (-sh), 0ull);
    }
}

// a += floor((vhi:vlo) 2^sh) for sh <= 63
__device__ __forceinline__ void add_shifted128(U128 &a, unsigned long long vlo, unsigned long long vhi, int sh)
{
    if (sh >= 0) {
        if (sh == 0) add_u128(a, vlo, vhi);
        else add_u128(a, vlo << sh, (vhi << sh) | (vlo >> (64 - sh)));
    } else {
        const int t = -sh;
        if (t < 64) add_u128(a, (vlo >> t) | (vhi << (64 - t)), vhi >> t);
        else if (t < 128) add_u128(a, vhi >> (t - 64), 0ull);
    }
}

// floor(log2|x|) and the integer form |x| = m 2^p of a float / a double (x != 0)
__device__ __forceinline__ int exp_of(uint32_t u)
{
    const int b = (int)((u >> 23) & 0xFF);
    const uint32_t f = u & 0x7FFFFFu;
    if (b) return b - 127;
    return f ? (31 - __clz((int)f)) - 149 : kNoExp;
}
__device__ __forceinline__ int exp_of(unsigned long long u)
{
    const int b = (int)((u >> 52) & 0x7FF);
    const unsigned long long f = u & 0xFFFFFFFFFFFFFull;
    if (b) return b - 1023;
    return f ? (63 - __clzll((long long)f)) - 1074 : kNoExp;
}

// the term floor(x^2 2^(110 - 2E)) of one component, added to a
__device__ __forceinline__ void add_square(U128 &a, uint32_t u, int E)
{
    const int b = (int)((u >> 23) & 0xFF);
    const uint32_t f = u & 0x7FFFFFu;
    if (!b && !f) return;
    const uint32_t m = b ? (f | 0x800000u) : f;
    const int p = b ? b - 150 : -149;
    add_shifted64(a, (unsigned long long)m * m, 2 * p + 110 - 2 * E);   // m^2 < 2^48, shift <= 64
}
__device__ __forceinline__ void add_square(U128 &a, unsigned long long u, int E)
{
    const int b = (int)((u >> 52) & 0x7FF);
    const unsigned long long f = u & 0xFFFFFFFFFFFFFull;
    if (!b && !f) return;
    const unsigned long long m = b ? (f | (1ull << 52)) : f;
    const int p = b ? b - 1075 : -1074;
    add_shifted128(a, m * m, __umul64hi(m, m), 2 * p + 110 - 2 * E);     // m^2 < 2^106, shift <= 6
}

// round-to-nearest-even of a 128-bit integer, times 2^scale
__device__ __forceinline__ double u128_scaled(U128 a, int scale)
{
    double d;
    if (a.hi == 0ull) {
        d = __ull2double_rn(a.lo);
    } else {
        const int n = __clzll((long long)a.hi);
        unsigned long long top = n ? ((a.hi << n) | (a.lo >> (64 - n))) : a.hi;
        if (a.lo << n) top |= 1ull;   // sticky: the bits below top decide ties
        d = ldexp(__ull2double_rn(top), 64 - n);
    }
    return ldexp(d, scale);
}

__device__ __forceinline__ U128 warp_sum(U128 a)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long lo = __shfl_xor_sync(0xffffffffu, a.lo, o);
        const unsigned long long hi = __shfl_xor_sync(0xffffffffu, a.hi, o);
        add_u128(a, lo, hi);
    }
    return a;
}

// The component bits of one orbital row, visited by the lanes of a warp: complex64 rows as 16-byte
// pieces (two elements) when the row start is 16-byte aligned, else element by element.
template <typename F>
__device__ __forceinline__ void for_components(const float2 *row, int n, int lane, F &&fn)
{
    if ((reinterpret_cast<uintptr_t>(row) & 15) == 0) {
        const uint4 *v = reinterpret_cast<const uint4 *>(row);
        const int n2 = n >> 1;
#pragma unroll 4
        for (int i = lane; i < n2; i += 32) {
            const uint4 q = __ldg(v + i);
            fn(q.x);
            fn(q.y);
            fn(q.z);
            fn(q.w);
        }
        if ((n & 1) && lane == 0) {
            const uint2 q = __ldg(reinterpret_cast<const uint2 *>(row) + (n - 1));
            fn(q.x);
            fn(q.y);
        }
    } else {
        for (int i = lane; i < n; i += 32) {
            const uint2 q = __ldg(reinterpret_cast<const uint2 *>(row) + i);
            fn(q.x);
            fn(q.y);
        }
    }
}
template <typename F>
__device__ __forceinline__ void for_components(const double2 *row, int n, int lane, F &&fn)
{
    const ulonglong2 *v = reinterpret_cast<const ulonglong2 *>(row);
#pragma unroll 4
    for (int i = lane; i < n; i += 32) {
        const ulonglong2 q = __ldg(v + i);
        fn(q.x);
        fn(q.y);
    }
}

// floor(log2 max |x|) over a row's components from the largest magnitude bit pattern (the bit
// patterns of non-negative floats / doubles order like their values), kNoExp for an all-zero row
__device__ __forceinline__ int exp_of_max(uint32_t m) { return m ? exp_of(m) : kNoExp; }
__device__ __forceinline__ int exp_of_max(unsigned long long m) { return m ? exp_of(m) : kNoExp; }

template <typename T>
__device__ __forceinline__ int row_exp(const T *row, int n, int lane)
{
    using B = typename std::conditional<sizeof(T) == 8, uint32_t, unsigned long long>::type;
    constexpr B mag = sizeof(T) == 8 ? (B)0x7FFFFFFFu : (B)0x7FFFFFFFFFFFFFFFull;
    B m = 0;
    for_components(row, n, lane, [&](B u) { m = max(m, (B)(u & mag)); });
    return __reduce_max_sync(0xffffffffu, exp_of_max(m));
}

// The complex64 terms of one lane between two folds: sums of yh^2, yh yl, yl^2 and of the floored
// terms (each below 2^46)
struct Sq64 {
    unsigned long long a2, a1, a0, as;
};

__device__ __forceinline__ void add_y(Sq64 &q, uint32_t m, int k)   // y = m 2^k < 2^56
{
    const unsigned long long y = (unsigned long long)m << k;
    const uint32_t yh = (uint32_t)(y >> 28), yl = (uint32_t)y & 0xFFFFFFFu;
    q.a2 += (unsigned long long)yh * yh;
    q.a1 += (unsigned long long)yh * yl;
    q.a0 += (unsigned long long)yl * yl;
}

// one component: k = max(b, 1) - 95 - E; zeros, subnormals and components far below the row maximum
// (k < 0: the term is floor(m^2 2^(2k)), m^2 < 2^48) leave the common branch
__device__ __forceinline__ void add_square_c64(Sq64 &q, uint32_t u, int kbase)
{
    const int b = (int)((u >> 23) & 0xFFu);
    uint32_t m = (u | 0x800000u) & 0xFFFFFFu;
    int k = b + kbase;
    if (b == 0 || k < 0) {
        if (b == 0) {
            m = u & 0x7FFFFFu;
            k = 1 + kbase;
        }
        if (k < 0) {
            if (k > -24) q.as += ((unsigned long long)m * m) >> (-2 * k);
            return;
        }
    }
    add_y(q, m, k);
}

__device__ __forceinline__ void fold(U128 &a, Sq64 &q)
{
    add_u128(a, q.a2 << 56, q.a2 >> 8);
    add_u128(a, q.a1 << 29, q.a1 >> 35);
    add_u128(a, q.a0, 0ull);
    add_u128(a, q.as, 0ull);
    q = Sq64{0ull, 0ull, 0ull, 0ull};
}

// A normal component with k = b - 95 - E >= 0 (then k <= 32, since y = m 2^k < 2^56 and m >= 2^23):
// yh and yl come from m 2^4 < 2^28 by two clamped funnel shifts, without a branch.
__device__ __forceinline__ void add_normal_c64(Sq64 &q, uint32_t u, int kbase)
{
    const uint32_t m4 = ((u << 4) & 0x7FFFFF0u) | 0x8000000u;
    const unsigned k = (unsigned)((int)((u >> 23) & 0xFFu) + kbase);
    const uint32_t yh = __funnelshift_lc(m4, 0u, k);        // floor(m 2^(k - 28))
    const uint32_t yl = __funnelshift_lc(0u, m4, k) >> 4;   // (m 2^k) mod 2^28
    q.a2 += (unsigned long long)yh * yh;
    q.a1 += (unsigned long long)yh * yl;
    q.a0 += (unsigned long long)yl * yl;
}

// The terms of one complex64 row in the window E, added to a; every lane folds after at most 128 terms.
// NORMAL: every component of the row is normal and within 2^32 of the maximum (checked by the caller).
template <bool NORMAL>
__device__ __forceinline__ void row_squares_c64(const float2 *row, int n, int lane, int E, U128 &a,
                                                unsigned long long pol)
{
    const int kbase = -95 - E;
    Sq64 q{0ull, 0ull, 0ull, 0ull};
    auto add = [&](uint32_t u) {
        if (NORMAL) add_normal_c64(q, u, kbase);
        else add_square_c64(q, u, kbase);
    };
    if ((reinterpret_cast<uintptr_t>(row) & 15) == 0) {
        const uint4 *v = reinterpret_cast<const uint4 *>(row);
        const int n2 = n >> 1;
        for (int c0 = 0; c0 < n2; c0 += 32 * 32) {
            const int c1 = min(n2, c0 + 32 * 32);
#pragma unroll 4
            for (int i = c0 + lane; i < c1; i += 32) {
                const uint4 t = ld_policy(v + i, pol);
                add(t.x);
                add(t.y);
                add(t.z);
                add(t.w);
            }
            fold(a, q);
        }
        if ((n & 1) && lane == 0) {
            const uint2 t = __ldg(reinterpret_cast<const uint2 *>(row) + (n - 1));
            add(t.x);
            add(t.y);
            fold(a, q);
        }
    } else {
        for (int c0 = 0; c0 < n; c0 += 64 * 32) {
            const int c1 = min(n, c0 + 64 * 32);
            for (int i = c0 + lane; i < c1; i += 32) {
                const uint2 t = __ldg(reinterpret_cast<const uint2 *>(row) + i);
                add(t.x);
                add(t.y);
            }
            fold(a, q);
        }
    }
}

// The largest and smallest component magnitudes of a complex64 row as bit patterns (lane-local; the
// caller reduces them over the warp)
__device__ __forceinline__ void row_range_c64(const float2 *row, int n, int lane, unsigned long long pol,
                                              uint32_t &mx, uint32_t &mn)
{
    auto see = [&](uint32_t u) {
        const uint32_t v = u & 0x7FFFFFFFu;
        mx = max(mx, v);
        mn = min(mn, v);
    };
    if ((reinterpret_cast<uintptr_t>(row) & 15) == 0) {
        const uint4 *v = reinterpret_cast<const uint4 *>(row);
        const int n2 = n >> 1;
#pragma unroll 4
        for (int i = lane; i < n2; i += 32) {
            const uint4 q = ld_policy(v + i, pol);
            see(q.x);
            see(q.y);
            see(q.z);
            see(q.w);
        }
        if ((n & 1) && lane == 0) {
            const uint2 q = __ldg(reinterpret_cast<const uint2 *>(row) + (n - 1));
            see(q.x);
            see(q.y);
        }
    } else {
        for (int i = lane; i < n; i += 32) {
            const uint2 q = __ldg(reinterpret_cast<const uint2 *>(row) + i);
            see(q.x);
            see(q.y);
        }
    }
}

// row window E and whether the row takes the branch-free path: the smallest magnitude is a normal
// number with k = b_min - 95 - E >= 0
__device__ __forceinline__ bool all_normal(uint32_t mn, int E) { return (int)(mn >> 23) >= max(1, 95 + E); }

template <bool NORMAL>
__device__ __forceinline__ void row_pair_c64(const float2 *a, int na, const float2 *b, int nb, int lane, int E,
                                             bool both, U128 &s, unsigned long long pol)
{
    row_squares_c64<NORMAL>(a, na, lane, E, s, pol);
    if (both) row_squares_c64<NORMAL>(b, nb, lane, E, s, pol);
}

// alpha = 2 on complex64 rows: SSM (one window over both sets) or PSM (one per set, multiplied)
__global__ void __launch_bounds__(kThreads, 4) weights_squares_c64(const float2 *__restrict__ phi, int64_t ld_phi,
                                                                int n_phi, const float2 *__restrict__ psi,
                                                                int64_t ld_psi, int n_psi, int64_t n_r, int psm,
                                                                double *__restrict__ w, int acc)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned long long keep = l2_evict_last(), drop = l2_evict_first();
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n_r; r += nw) {
        const float2 *a = phi + r * ld_phi, *b = psi + r * ld_psi;
        uint32_t mxa = 0u, mna = 0xFFFFFFFFu, mxb = 0u, mnb = 0xFFFFFFFFu;
        row_range_c64(a, n_phi, lane, keep, mxa, mna);
        row_range_c64(b, n_psi, lane, keep, mxb, mnb);
        mxa = __reduce_max_sync(0xffffffffu, mxa);
        mna = __reduce_min_sync(0xffffffffu, mna);
        mxb = __reduce_max_sync(0xffffffffu, mxb);
        mnb = __reduce_min_sync(0xffffffffu, mnb);
        const int ea = exp_of_max(mxa), eb = exp_of_max(mxb);
        double v;
        if (!psm) {
            const int E = max(ea, eb);
            U128 s{0ull, 0ull};
            if (E != kNoExp) {
                if (all_normal(min(mna, mnb), E)) row_pair_c64<true>(a, n_phi, b, n_psi, lane, E, true, s, drop);
                else row_pair_c64<false>(a, n_phi, b, n_psi, lane, E, true, s, drop);
            }
            s = warp_sum(s);
            v = E == kNoExp ? 0.0 : u128_scaled(s, 2 * E - 110);
        } else {
            U128 sa{0ull, 0ull}, sb{0ull, 0ull};
            if (ea != kNoExp) {
                if (all_normal(mna, ea)) row_pair_c64<true>(a, n_phi, b, n_psi, lane, ea, false, sa, drop);
                else row_pair_c64<false>(a, n_phi, b, n_psi, lane, ea, false, sa, drop);
            }
            if (eb != kNoExp) {
                if (all_normal(mnb, eb)) row_pair_c64<true>(b, n_psi, a, n_phi, lane, eb, false, sb, drop);
                else row_pair_c64<false>(b, n_psi, a, n_phi, lane, eb, false, sb, drop);
            }
            sa = warp_sum(sa);
            sb = warp_sum(sb);
            const double xa = ea == kNoExp ? 0.0 : u128_scaled(sa, 2 * ea - 110);
            const double xb = eb == kNoExp ? 0.0 : u128_scaled(sb, 2 * eb - 110);
            v = __dmul_rn(xa, xb);
        }
        if (lane == 0) w[r] = acc ? __dadd_rn(w[r], v) : v;   // shared weight of several pairs: one rounding per pair
    }
}

// alpha = 2 on complex128 rows: SSM (one window over both sets) or PSM (one per set, multiplied)
__global__ void __launch_bounds__(kThreads) weights_squares_c128(const double2 *__restrict__ phi, int64_t ld_phi,
                                                                 int n_phi, const double2 *__restrict__ psi,
                                                                 int64_t ld_psi, int n_psi, int64_t n_r, int psm,
                                                                 double *__restrict__ w, int acc)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    auto squares = [&](const double2 *row, int n, int E, U128 &s) {
        for_components(row, n, lane, [&](unsigned long long u) { add_square(s, u, E); });
    };
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n_r; r += nw) {
        const double2 *a = phi + r * ld_phi, *b = psi + r * ld_psi;
        const int ea = row_exp(a, n_phi, lane), eb = row_exp(b, n_psi, lane);
        double v;
        if (!psm) {
            const int E = max(ea, eb);
            U128 s{0ull, 0ull};
            if (E != kNoExp) {
                squares(a, n_phi, E, s);
                squares(b, n_psi, E, s);
            }
            s = warp_sum(s);
            v = E == kNoExp ? 0.0 : u128_scaled(s, 2 * E - 110);
        } else {
            U128 sa{0ull, 0ull}, sb{0ull, 0ull};
            if (ea != kNoExp) squares(a, n_phi, ea, sa);
            if (eb != kNoExp) squares(b, n_psi, eb, sb);
            sa = warp_sum(sa);
            sb = warp_sum(sb);
            const double xa = ea == kNoExp ? 0.0 : u128_scaled(sa, 2 * ea - 110);
            const double xb = eb == kNoExp ? 0.0 : u128_scaled(sb, 2 * eb - 110);
            v = __dmul_rn(xa, xb);
        }
        if (lane == 0) w[r] = acc ? __dadd_rn(w[r], v) : v;
    }
}

// |z|^alpha in FP64 for alpha != 2: m = re*re + im*im with each operation rounded (for complex64
// input the products are exact, so one fused multiply-add gives the same bits)
template <int AK>  // 1, 3, 4: sqrt/product forms; 0: pow
__device__ __forceinline__ double modulus_pow(double re, double im, bool exact_products, double half_alpha)
{
    const double m = exact_products ? __fma_rn(re, re, __dmul_rn(im, im))
                                    : __dadd_rn(__dmul_rn(re, re), __dmul_rn(im, im));
    if (AK == 1) return __dsqrt_rn(m);
    if (AK == 3) return __dmul_rn(m, __dsqrt_rn(m));
    if (AK == 4) return __dmul_rn(m, m);
    return pow(m, half_alpha);
}

template <typename T, int AK, typename F>
__device__ __forceinline__ void for_terms(const T *row, int n, int lane, double half_alpha, F &&fn)
{
    for (int i = lane; i < n; i += 32) {
        const double2 z = cload(row, i);
        fn(modulus_pow<AK>(z.x, z.y, sizeof(T) == 8, half_alpha));
    }
}

// floor(t 2^s) of a non-negative double as a 128-bit integer (t 2^s < 2^127)
__device__ __forceinline__ void add_fixed(U128 &a, double t, int s)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(t);
    const int b = (int)((u >> 52) & 0x7FF);
    const unsigned long long f = u & 0xFFFFFFFFFFFFFull;
    if (!b && !f) return;
    const unsigned long long m = b ? (f | (1ull << 52)) : f;
    add_shifted128(a, m, 0ull, (b ? b - 1075 : -1074) + s);
}

// alpha != 2: the FP64 terms summed exactly over both sets (the terms are formed twice: once for
// the window, once for the sum; this path serves the weight-function study)
template <typename T, int AK>
__global__ void __launch_bounds__(kThreads) weights_terms(const T *__restrict__ phi, int64_t ld_phi, int n_phi,
                                                          const T *__restrict__ psi, int64_t ld_psi, int n_psi,
                                                          int64_t n_r, double half_alpha, double *__restrict__ w,
                                                          int acc)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n_r; r += nw) {
        const T *a = phi + r * ld_phi, *b = psi + r * ld_psi;
        int e = kNoExp;
        auto mx = [&](double t) {
            if (t != 0.0) e = max(e, exp_of((unsigned long long)__double_as_longlong(t)));
        };
        for_terms<T, AK>(a, n_phi, lane, half_alpha, mx);
        for_terms<T, AK>(b, n_psi, lane, half_alpha, mx);
        const int E = __reduce_max_sync(0xffffffffu, e);
        U128 s{0ull, 0ull};
        if (E != kNoExp) {
            auto add = [&](double t) { add_fixed(s, t, 110 - E); };
            for_terms<T, AK>(a, n_phi, lane, half_alpha, add);
            for_terms<T, AK>(b, n_psi, lane, half_alpha, add);
        }
        s = warp_sum(s);
        const double v = E == kNoExp ? 0.0 : u128_scaled(s, E - 110);
        if (lane == 0) w[r] = acc ? __dadd_rn(w[r], v) : v;
    }
}

unsigned grid_rows(int64_t n_r)
{
    // 4 blocks of 8 warps per SM: enough loads in flight, and the rows between a warp's two passes
    // (about 32 warps x 152 SMs rows) stay in L2 for the second read
    const int64_t g = (n_r + 7) / 8;
    return (unsigned)(g < 152 * 4 ? (g < 1 ? 1 : g) : 152 * 4);
}

template <typename T>
isdf_status launch_weights(const void *phi, int64_t ld_phi, int n_phi, const void *psi, int64_t ld_psi,
                           int n_psi, int64_t n_r, int psm, double alpha, double *w, int acc, cudaStream_t st)
{
    const unsigned grid = grid_rows(n_r);
    const T *a = static_cast<const T *>(phi);
    const T *b = static_cast<const T *>(psi);
    const double ha = 0.5 * alpha;
    if (psm || alpha == 2.0) {
        if constexpr (sizeof(T) == 8)
            weights_squares_c64<<<grid, kThreads, 0, st>>>(a, ld_phi, n_phi, b, ld_psi, n_psi, n_r, psm, w, acc);
        else
            weights_squares_c128<<<grid, kThreads, 0, st>>>(a, ld_phi, n_phi, b, ld_psi, n_psi, n_r, psm, w, acc);
    }
    else if (alpha == 1.0)
        weights_terms<T, 1><<<grid, kThreads, 0, st>>>(a, ld_phi, n_phi, b, ld_psi, n_psi, n_r, ha, w, acc);
    else if (alpha == 3.0)
        weights_terms<T, 3><<<grid, kThreads, 0, st>>>(a, ld_phi, n_phi, b, ld_psi, n_psi, n_r, ha, w, acc);
    else if (alpha == 4.0)
        weights_terms<T, 4><<<grid, kThreads, 0, st>>>(a, ld_phi, n_phi, b, ld_psi, n_psi, n_r, ha, w, acc);
    else
        weights_terms<T, 0><<<grid, kThreads, 0, st>>>(a, ld_phi, n_phi, b, ld_psi, n_psi, n_r, ha, w, acc);
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
