// Step 2: weighted Lloyd K-means on the real-space grid (Sec. 2.2,
// Eq. opt second form, Eq. r_k, Algorithm 1).
//
// Design (one CTA of 8 warps per 8 x 8 x 8 tile of the grid; each warp owns a
// 4 x 4 x 4 sub-cube, two points per lane):
//  * exact two-level pruning: the CTA bounds every centroid's squared
//    distance to its tile from below (LB) and above (UB) in FP32 with error
//    margins and keeps those with LB <= min UB (only they can be the nearest
//    centroid of a point in the tile); each warp prunes that list again
//    against its own sub-cube;
//  * FP32 screen: each point evaluates its warp's candidates in FP32 in
//    tile-local coordinates and keeps the two smallest values; when their gap
//    exceeds a rigorous bound E on |d_fp32 - d_exact| (+ FP64 rounding) the
//    FP32 winner is the FP64 winner. Otherwise the point re-evaluates the close
//    candidates with the FP64 formula ((dx*dx + dy*dy) + dz*dz) and takes the
//    smallest (distance, mu) pair - exactly the brute-force FP64 decision. The
//    bound and the gap test are evaluated in FP32 with upward margins (a test
//    that errs sends a point to the FP64 path, never past it), and the grid
//    coordinates RN(i h) of a tile come from a per-CTA table: GB300 issues
//    FP64 at about 2 operations per clock per SM, so the pass keeps FP64 for
//    the decisions and the products w*x of the exact sums;
//  * exact update: each FP64 product w*x enters as the 128-bit integer
//    floor(w*x*2^s); sums are integer (associative, so the result does not
//    depend on thread or block order): per warp by shuffles for each distinct
//    winner, then per CTA in shared memory, then in global memory, with the
//    carry of the low word detected by the adding thread; the update kernel
//    rounds each sum to FP64 and divides once.
#include <mutex>

#include "common.cuh"

namespace {

constexpr int TX = 8, TY = 8, TZ = 8;    // CTA tile (smaller tiles repeat the per-tile centroid scan)
constexpr int kThreads = 256;            // 8 warps x (4 x 4 x 4 sub-cube, 2 points per lane)
constexpr int kWarpCap = 256;            // per-warp candidate list capacity (else the CTA list is used)
constexpr int kSlots = 256;              // per-CTA shared accumulators (first candidates)
constexpr int kMaxMu = 8192;

struct KmCtl {
    unsigned long long wmax_bits;
    unsigned long long ties;
    unsigned long long refined;
    unsigned int moved[2];     // update t sets moved[t & 1] when any centroid changed
    int error;
    int converged;
    int n_iter;
    int pad;
};

struct KmArgs {
    const double *w;
    int nx, ny, nz;
    double hx, hy, hz;
    double tie_floor;     // hmin^2
    int n_mu;
    int s_base;           // 126 - bits(N_r) - e(max(L, 1))
    int ntx, nty, ntz;    // tiles per axis
    double *cent;         // n_mu x 3
    float4 *c32;          // n_mu: FP32 copies of the centroids for the conservative tile scan
    float scan_err;       // bound on the FP32 error of a tile-local centroid coordinate in the scan
    double lmax;          // max(Lx, Ly, Lz)
    int want_obj;         // objective requested: FP64 distance of every winner
    unsigned long long *acc;  // n_mu x 8: (w, wx, wy, wz) x (lo, hi)
    int32_t *labels;
    double *dist;
    double *jpart;
    unsigned long long *best;
    unsigned long long *idx_u;
    KmCtl *ctl;
    int early_stop;
};

struct U128 {
    unsigned long long lo, hi;
};

// floor(v * 2^s) for finite v >= 0 and 0 <= s, as an exact 128-bit integer
__device__ __forceinline__ U128 fixed_of(double v, int s)
{
    U128 r{0ull, 0ull};
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);   // +-0 gives m = 0 below
    const int e = (int)((b >> 52) & 0x7ff);
    unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    int sh;
    if (e == 0) {
        sh = s - 1074;
    } else {
        m |= 1ull << 52;
        sh = e - 1075 + s;
    }
    if (sh >= 0) {
        if (sh == 0) {
            r.lo = m;
        } else if (sh < 64) {
            r.lo = m << sh;
            r.hi = m >> (64 - sh);
        } else if (sh < 128) {
            r.hi = m << (sh - 64);
        }
    } else if (sh > -64) {
        r.lo = m >> (-sh);
    }
    return r;
}

__device__ __forceinline__ void atomic_add_u128(unsigned long long *p, U128 v)
{
    if ((v.lo | v.hi) == 0ull) return;
    const unsigned long long old = atomicAdd(p, v.lo);
    const unsigned long long h = v.hi + ((old + v.lo < old) ? 1ull : 0ull);
    if (h) atomicAdd(p + 1, h);
}

// round-to-nearest-even conversion of an unsigned 128-bit integer
__device__ __forceinline__ double u128_to_double(unsigned long long lo, unsigned long long hi)
{
    if (hi == 0ull) return __ull2double_rn(lo);
    const int n = __clzll((long long)hi);
    unsigned long long top = n ? ((hi << n) | (lo >> (64 - n))) : hi;
    const unsigned long long rest = lo << n;
    if (rest) top |= 1ull;
    return ldexp(__ull2double_rn(top), 64 - n);
}

__device__ __forceinline__ double dist2_fp64(double x, double y, double z, double cx, double cy, double cz)
{
    const double dx = __dsub_rn(x, cx), dy = __dsub_rn(y, cy), dz = __dsub_rn(z, cz);
    double d = __dmul_rn(dx, dx);
    d = __dadd_rn(d, __dmul_rn(dy, dy));
    d = __dadd_rn(d, __dmul_rn(dz, dz));
    return d;
}

__device__ __forceinline__ int fixed_scale(const KmArgs &a)
{
    const double wmax = __longlong_as_double((long long)a.ctl->wmax_bits);
    int e = 0;
    if (wmax > 0.0) frexp(wmax, &e);
    return a.s_base - e;
}

// deterministic block sum (fixed shuffle pattern, fixed warp order)
__device__ double block_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_down_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s = __dadd_rn(s, red[i]);
    return s;  // valid in thread 0
}

__global__ void km_init(KmArgs a, const int64_t *__restrict__ init_idx, int64_t n_r)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        a.ctl->wmax_bits = 0ull;
        a.ctl->ties = 0ull;
        a.ctl->refined = 0ull;
        a.ctl->moved[0] = 0u;
        a.ctl->moved[1] = 0u;
        a.ctl->error = 0;
        a.ctl->converged = 0;
        a.ctl->n_iter = 0;
    }
    if (i < a.n_mu) {
        int64_t r = init_idx[i];
        if (r < 0 || r >= n_r) {
            atomicExch(&a.ctl->error, 2);
            r = 0;
        }
        const int64_t ix = r / ((int64_t)a.ny * a.nz), iy = (r / a.nz) % a.ny, iz = r % a.nz;
        a.cent[3 * i + 0] = __dmul_rn((double)ix, a.hx);
        a.cent[3 * i + 1] = __dmul_rn((double)iy, a.hy);
        a.cent[3 * i + 2] = __dmul_rn((double)iz, a.hz);
        a.c32[i] = make_float4((float)a.cent[3 * i], (float)a.cent[3 * i + 1], (float)a.cent[3 * i + 2], 0.f);
#pragma unroll
        for (int k = 0; k < 8; ++k) a.acc[8 * i + k] = 0ull;
        a.best[i] = ~0ull;
        a.idx_u[i] = ~0ull;
    }
    for (int64_t r = i; r < n_r; r += (int64_t)gridDim.x * blockDim.x) a.labels[r] = -1;
}

__global__ void km_wmax(KmArgs a, int64_t n_r)
{
    unsigned long long m = 0ull;
    int bad = 0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_r; r += (int64_t)gridDim.x * blockDim.x) {
        const double v = a.w[r];
        if (!(v >= 0.0) || isinf(v)) bad = 1;
        else if (v > 0.0) m = max(m, (unsigned long long)__double_as_longlong(v));
    }
    for (int o = 16; o > 0; o >>= 1) {
        m = max(m, __shfl_down_sync(0xffffffffu, m, o));
        bad |= __shfl_down_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (m) atomicMax(&a.ctl->wmax_bits, m);
        if (bad) atomicExch(&a.ctl->error, 1);
    }
}

__global__ void km_check_scale(KmArgs a)
{
    if (threadIdx.x == 0 && fixed_scale(a) < 0) atomicExch(&a.ctl->error, 1);
}

__device__ __forceinline__ U128 shfl_down_u128(U128 v, int o)
{
    U128 r;
    r.lo = __shfl_down_sync(0xffffffffu, v.lo, o);
    r.hi = __shfl_down_sync(0xffffffffu, v.hi, o);
    return r;
}

__device__ __forceinline__ U128 add_u128(U128 a, U128 b)
{
    U128 r;
    r.lo = a.lo + b.lo;
    r.hi = a.hi + b.hi + (r.lo < a.lo ? 1ull : 0ull);
    return r;
}

// Sum the (w, wx, wy, wz) integers of the lanes that share a winner, one
// distinct winner at a time, and add each sum once (lane 0) to its slot.
__device__ __forceinline__ void warp_accumulate(int key, const U128 (&v)[4], unsigned long long (*slot)[8],
                                                unsigned long long *acc, const float4 *cand, int lane)
{
    unsigned pending = __ballot_sync(0xffffffffu, key >= 0);
    while (pending) {
        const int leader = __ffs(pending) - 1;
        const int k = __shfl_sync(0xffffffffu, key, leader);
        const bool mine = (key == k);
        pending &= ~__ballot_sync(0xffffffffu, mine);
        U128 s[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) s[q] = mine ? v[q] : U128{0ull, 0ull};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < 4; ++q) s[q] = add_u128(s[q], shfl_down_u128(s[q], o));
        if (lane == 0) {
            unsigned long long *dst = (k < kSlots) ? &slot[k][0] : &acc[8 * (int64_t)__float_as_int(cand[k].w)];
#pragma unroll
            for (int q = 0; q < 4; ++q) atomic_add_u128(dst + 2 * q, s[q]);
        }
    }
}

// NW = 8: an 8 x 8 x 8 tile per CTA (warps = its eight 4 x 4 x 4 sub-cubes); NW = 4: a 4 x 8 x 8 half
// tile (the four sub-cubes of one x half), which doubles the CTAs on grids with few tiles per SM
template <bool FINAL, int NW>
__global__ void __launch_bounds__(32 * NW, 1) km_assign(KmArgs a, int t)
{
    constexpr int NT = 32 * NW, TXE = NW == 8 ? TX : TX / 2;
    if (a.ctl->error) return;
    if (!FINAL && a.ctl->converged) return;
    if (!FINAL && a.early_stop && t >= 2 && a.ctl->moved[(t - 1) & 1] == 0u) {
        // update t-1 left every centroid bit-identical, so this and every later pass would
        // repeat the labels and sums of pass t-1: the loop has converged. The labels first
        // repeated at pass t-1 (labels repeat, so the sums and then the centroids repeat one
        // update later), which is the count reported; objective entries and near-tie counts
        // of passes 0 .. t-1 are complete. (Points of zero weight can change cluster without
        // moving a centroid; then the count is one below the first pass whose labels repeat.)
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.ctl->n_iter = t - 1;
            a.ctl->converged = 1;
        }
        return;
    }

    extern __shared__ float4 cand[];  // n_mu entries: (qx, qy, qz, mu bits), tile-local FP32 coordinates
    __shared__ unsigned long long slot[kSlots][8];
    __shared__ unsigned short wlist[NW][kWarpCap];
    __shared__ int wcount[NW];
    __shared__ unsigned int n_cand;
    __shared__ float minub_sh[NW];
    __shared__ double red[NW];
    __shared__ unsigned long long redu[NW];
    __shared__ unsigned long long redu2[NW];

    // grid coordinates of the tile (xs[i] = RN((ix0 + i) hx), ...) and its FP32 extents, formed once per CTA:
    // the FP64 pipe (about 2 operations per clock per SM) is the scarce unit of this kernel
    __shared__ double xs[TXE], ys[TY], zs[TZ];
    __shared__ float hdr32[11];  // hx, hy, hz, Px, Py, Pz (tile extents), ox, oy, oz (origin), L, hmin^2 in FP32
    __shared__ int s_fix_sh;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int b = blockIdx.x;
    const int tz = b % a.ntz, ty = (b / a.ntz) % a.nty, tx = b / (a.ntz * a.nty);
    const int ix0 = tx * TXE, iy0 = ty * TY, iz0 = tz * TZ;
    const int ex = min(TXE, a.nx - ix0), ey = min(TY, a.ny - iy0), ez = min(TZ, a.nz - iz0);
    if (tid < TXE) xs[tid] = __dmul_rn((double)(ix0 + tid), a.hx);
    else if (tid < TXE + TY) ys[tid - TXE] = __dmul_rn((double)(iy0 + tid - TXE), a.hy);
    else if (tid < TXE + TY + TZ) zs[tid - TXE - TY] = __dmul_rn((double)(iz0 + tid - TXE - TY), a.hz);
    else if (tid == 32) {
        hdr32[0] = (float)a.hx;
        hdr32[1] = (float)a.hy;
        hdr32[2] = (float)a.hz;
        hdr32[3] = (float)((ex - 1) * a.hx);
        hdr32[4] = (float)((ey - 1) * a.hy);
        hdr32[5] = (float)((ez - 1) * a.hz);
        hdr32[6] = (float)__dmul_rn((double)ix0, a.hx);   // = (float)xs[0], ...
        hdr32[7] = (float)__dmul_rn((double)iy0, a.hy);
        hdr32[8] = (float)__dmul_rn((double)iz0, a.hz);
        hdr32[9] = (float)a.lmax;
        hdr32[10] = (float)a.tie_floor;
        n_cand = 0u;
        if (!FINAL) s_fix_sh = fixed_scale(a);
    }
    __syncthreads();
    const double ox = xs[0], oy = ys[0], oz = zs[0];
    const float hx = hdr32[0], hy = hdr32[1], hz = hdr32[2];
    const float Px = hdr32[3], Py = hdr32[4], Pz = hdr32[5];

    // ---- tile scan (FP32, conservative): min over centroids of the largest squared distance to the tile
    const float ox32 = hdr32[6], oy32 = hdr32[7], oz32 = hdr32[8];
    const float dq = a.scan_err;
    float mub = INFINITY;
    for (int m = tid; m < a.n_mu; m += NT) {
        const float4 c = a.c32[m];
        const float qx = c.x - ox32, qy = c.y - oy32, qz = c.z - oz32;
        const float ux = fmaxf(fabsf(qx), fabsf(Px - qx));
        const float uy = fmaxf(fabsf(qy), fabsf(Py - qy));
        const float uz = fmaxf(fabsf(qz), fabsf(Pz - qz));
        mub = fminf(mub, ux * ux + uy * uy + uz * uz);
    }
    for (int o = 16; o > 0; o >>= 1) mub = fminf(mub, __shfl_xor_sync(0xffffffffu, mub, o));
    if (lane == 0) minub_sh[warp] = mub;
    __syncthreads();
    float minub = minub_sh[0];
    for (int i = 1; i < NW; ++i) minub = fminf(minub, minub_sh[i]);
    const float sminub = sqrtf(minub);
    // keep every centroid whose smallest squared distance to the tile can reach min UB: each
    // coordinate carries an error <= dq, so LB and UB move by <= dq (2 sqrt(3) sqrt(.) + 3 dq)
    for (int m = tid; m < a.n_mu; m += NT) {
        const float4 c = a.c32[m];
        const float qx = c.x - ox32, qy = c.y - oy32, qz = c.z - oz32;
        const float lx = fmaxf(0.f, fmaxf(-qx, qx - Px));
        const float ly = fmaxf(0.f, fmaxf(-qy, qy - Py));
        const float lz = fmaxf(0.f, fmaxf(-qz, qz - Pz));
        const float lb = lx * lx + ly * ly + lz * lz;
        const float margin = dq * (3.5f * (sqrtf(lb) + sminub) + 6.f * dq) + 1e-6f * (lb + minub) + 1e-30f;
        if (lb <= minub + margin) {
            const unsigned j = atomicAdd(&n_cand, 1u);
            // accurate tile-local coordinates of the kept centroids (one FP64 subtraction each)
            cand[j] = make_float4((float)__dsub_rn(a.cent[3 * m + 0], ox), (float)__dsub_rn(a.cent[3 * m + 1], oy),
                                  (float)__dsub_rn(a.cent[3 * m + 2], oz), __int_as_float(m));
        }
    }
    __syncthreads();
    const int nc = (int)n_cand;
    const int ns = min(nc, kSlots);
    if (!FINAL)
        for (int i = tid; i < ns * 8; i += NT) slot[i >> 3][i & 7] = 0ull;

    // ---- this warp's 4 x 4 x 4 sub-cube and its candidate list
    const int sx = (warp >> 2) & 1, sy = (warp >> 1) & 1, sz = warp & 1;
    const int bx = 4 * sx, by = 4 * sy, bz = 4 * sz;
    const int wex = min(4, ex - bx), wey = min(4, ey - by), wez = min(4, ez - bz);
    const bool wvalid = wex > 0 && wey > 0 && wez > 0;
    const float Sx0 = bx * hx, Sy0 = by * hy, Sz0 = bz * hz;
    const float Sx1 = Sx0 + (wex - 1) * hx, Sy1 = Sy0 + (wey - 1) * hy, Sz1 = Sz0 + (wez - 1) * hz;
    float wub = INFINITY;
    for (int j = lane; j < nc; j += 32) {
        const float4 q = cand[j];
        const float ux = fmaxf(fabsf(q.x - Sx0), fabsf(Sx1 - q.x));
        const float uy = fmaxf(fabsf(q.y - Sy0), fabsf(Sy1 - q.y));
        const float uz = fmaxf(fabsf(q.z - Sz0), fabsf(Sz1 - q.z));
        wub = fminf(wub, ux * ux + uy * uy + uz * uz);
    }
    for (int o = 16; o > 0; o >>= 1) wub = fminf(wub, __shfl_xor_sync(0xffffffffu, wub, o));
    // tile-local coordinates are accurate to ~1e-7 relative; the margin covers them and the float sums
    const float Tmx = fmaxf(Px, fmaxf(Py, Pz));
    const float wcut = wub * 1.0001f + 4e-6f * (Tmx * Tmx + wub) + 1e-30f;
    int wn = 0;
    float wq = 0.f;
    for (int base = 0; base < nc; base += 32) {
        const int j = base + lane;
        bool keep = false;
        if (j < nc) {
            const float4 q = cand[j];
            const float lx = fmaxf(0.f, fmaxf(Sx0 - q.x, q.x - Sx1));
            const float ly = fmaxf(0.f, fmaxf(Sy0 - q.y, q.y - Sy1));
            const float lz = fmaxf(0.f, fmaxf(Sz0 - q.z, q.z - Sz1));
            keep = (lx * lx + ly * ly + lz * lz) * 0.9999f <= wcut;
            if (keep) wq = fmaxf(wq, fmaxf(fabsf(q.x), fmaxf(fabsf(q.y), fabsf(q.z))));
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        const int pos = wn + __popc(bal & ((1u << lane) - 1u));
        if (keep && pos < kWarpCap) wlist[warp][pos] = (unsigned short)j;
        wn += __popc(bal);
    }
    for (int o = 16; o > 0; o >>= 1) wq = fmaxf(wq, __shfl_xor_sync(0xffffffffu, wq, o));
    const bool use_w = wn <= kWarpCap;          // overflow: scan the whole tile list instead
    const int cnt = use_w ? wn : nc;
    if (!use_w) wq = 0.f;
    if (!use_w)
        for (int j = lane; j < nc; j += 32) {
            const float4 q = cand[j];
            wq = fmaxf(wq, fmaxf(fabsf(q.x), fmaxf(fabsf(q.y), fabsf(q.z))));
        }
    for (int o = 16; o > 0; o >>= 1) wq = fmaxf(wq, __shfl_xor_sync(0xffffffffu, wq, o));

    // rigorous bound on |d_fp32 - d_exact| (+ FP64 rounding) for this warp: the point coordinates
    // (integer offset x FP32 spacing) carry <= 2.01 u32 |p|, the candidates <= 1.0001 u32 |q|,
    // their difference one more rounding, then three FP32 products and two FP32 additions
    // It is evaluated in FP32: every quantity is positive, so each operation adds at most a relative
    // 2^-24 (a fused multiply-add one rounding); the factor 1 + 2^-16 covers the dozen roundings, and the
    // formula's 1 % slack the rounding of its decimal constants and of L.
    constexpr float u32 = 5.9604644775390625e-8f;   // 2^-24
    constexpr float up = 1.f + 1.52587890625e-5f;   // 1 + 2^-16
    const float Pm = Tmx, Qm = wq;
    const float Tm = (Pm + Qm) * (1.f + 4.f * u32);
    const float del = 1.01f * u32 * (2.01f * Pm + 1.0001f * Qm + (Pm + Qm)) + 8e-16f * hdr32[9];
    const float E = 1.01f * (3.f * del * (2.f * Tm + del) + 9.001f * u32 * Tm * Tm + 1.6e-15f * 3.f * Tm * Tm) * up;

    // ---- the two points of this lane
    const int lx2 = lane >> 4, ly = (lane >> 2) & 3, lz = lane & 3;
    float px[2], py[2], pz[2], d1[2], d2[2];
    int j1[2];
    bool valid[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int dxl = lx2 + 2 * h;
        valid[h] = wvalid && dxl < wex && ly < wey && lz < wez;
        px[h] = (float)(bx + dxl) * hx;
        py[h] = (float)(by + ly) * hy;
        pz[h] = (float)(bz + lz) * hz;
        d1[h] = INFINITY;
        d2[h] = INFINITY;
        j1[h] = 0;
    }
    __syncthreads();   // slots cleared
    for (int i = 0; i < cnt; ++i) {
        const int j = use_w ? (int)wlist[warp][i] : i;
        const float4 q = cand[j];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float dx = px[h] - q.x, dy = py[h] - q.y, dz = pz[h] - q.z;
            const float d = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            if (d < d1[h]) {
                d2[h] = d1[h];
                d1[h] = d;
                j1[h] = j;
            } else if (d < d2[h]) {
                d2[h] = d;
            }
        }
    }

    double jv = 0.0;
    unsigned long long my_ties = 0, my_ref = 0;
    const int s_fix = FINAL ? 0 : s_fix_sh;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        int key = -1;
        U128 v[4] = {{0ull, 0ull}, {0ull, 0ull}, {0ull, 0ull}, {0ull, 0ull}};
        if (valid[h]) {
            const int ix = ix0 + bx + lx2 + 2 * h, iy = iy0 + by + ly, iz = iz0 + bz + lz;
            const int64_t r = ((int64_t)ix * a.ny + iy) * a.nz + iz;
            const double x = xs[bx + lx2 + 2 * h], y = ys[by + ly], z = zs[bz + lz];   // RN(ix hx), ...
            // the FP32 winner is the FP64 winner when the runner-up is further than the gap; the test is
            // conservative in FP32 (gap rounded up by 1 + 2^-16, the difference scaled down by 1 - 2^-22)
            const float gap = (2.f * E + 2.0e-12f * fmaxf(d1[h] + E, hdr32[10]) + 1.0e-14f * (d1[h] + E)) * up;
            int win_j = j1[h], win_mu = __float_as_int(cand[j1[h]].w);
            double win_d = 0.0;
            if ((d2[h] - d1[h]) * (1.f - 2.384185791015625e-7f) > gap) {
                if (FINAL || a.want_obj)
                    win_d = dist2_fp64(x, y, z, a.cent[3 * win_mu], a.cent[3 * win_mu + 1], a.cent[3 * win_mu + 2]);
            } else {
                // FP64 decision over the candidates that can still win
                my_ref += 1;
                double b1 = INFINITY, b2 = INFINITY;
                int bm = 0x7fffffff, bj = 0;
                const double lim = (double)d1[h] + (double)gap;
                for (int i = 0; i < cnt; ++i) {
                    const int j = use_w ? (int)wlist[warp][i] : i;
                    const float4 q = cand[j];
                    const float dx = px[h] - q.x, dy = py[h] - q.y, dz = pz[h] - q.z;
                    const float d = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                    if ((double)d > lim) continue;
                    const int m = __float_as_int(q.w);
                    const double e = dist2_fp64(x, y, z, a.cent[3 * m], a.cent[3 * m + 1], a.cent[3 * m + 2]);
                    if (e < b1 || (e == b1 && m < bm)) {
                        b2 = b1;
                        b1 = e;
                        bm = m;
                        bj = j;
                    } else if (e < b2) {
                        b2 = e;
                    }
                }
                win_j = bj;
                win_mu = bm;
                win_d = b1;
                if (a.n_mu > 1 && __dsub_rn(b2, b1) <= 1e-12 * fmax(b1, a.tie_floor)) my_ties += 1;
            }
            const double wr = a.w[r];
            if (FINAL || a.want_obj) jv = __dadd_rn(jv, __dmul_rn(wr, win_d));
            if (!FINAL) {
                key = win_j;
                v[0] = fixed_of(wr, s_fix);
                v[1] = fixed_of(__dmul_rn(wr, x), s_fix);
                v[2] = fixed_of(__dmul_rn(wr, y), s_fix);
                v[3] = fixed_of(__dmul_rn(wr, z), s_fix);
            } else {
                a.labels[r] = win_mu;
                a.dist[r] = win_d;
                atomicMin(&a.best[win_mu], (unsigned long long)__double_as_longlong(win_d));
            }
        }
        if (!FINAL) warp_accumulate(key, v, slot, a.acc, cand, lane);
    }
    // the objective partial (fixed shuffle pattern and warp order: deterministic) and the two
    // counts, reduced together with one barrier, which also completes the shared slots
    const bool want_j = FINAL || a.want_obj;
    for (int o = 16; o > 0; o >>= 1) {
        if (want_j) jv = __dadd_rn(jv, __shfl_down_sync(0xffffffffu, jv, o));
        my_ties += __shfl_down_sync(0xffffffffu, my_ties, o);
        my_ref += __shfl_down_sync(0xffffffffu, my_ref, o);
    }
    if (lane == 0) {
        red[warp] = jv;
        redu[warp] = my_ties;
        redu2[warp] = my_ref;
    }
    __syncthreads();
    if (tid == 0) {
        double jt = 0.0;
        unsigned long long tt = 0ull, rr = 0ull;
        for (int i = 0; i < NW; ++i) {
            jt = __dadd_rn(jt, red[i]);
            tt += redu[i];
            rr += redu2[i];
        }
        if (want_j) a.jpart[b] = jt;
        if (tt) atomicAdd(&a.ctl->ties, tt);
        if (rr) atomicAdd(&a.ctl->refined, rr);
    }
    if (!FINAL) {
        for (int j = tid; j < ns; j += NT) {
            unsigned long long *src = &slot[j][0];
            if ((src[0] | src[1]) == 0ull) continue;
            const int m = __float_as_int(cand[j].w);
            unsigned long long *dst = &a.acc[8 * (int64_t)m];
#pragma unroll
            for (int k = 0; k < 4; ++k) atomic_add_u128(dst + 2 * k, U128{src[2 * k], src[2 * k + 1]});
        }
    }
}

// deterministic sum of the per-tile objective partials (one CTA)
__device__ double sum_partials(const double *p, int n, double *red)
{
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v = __dadd_rn(v, p[i]);
    return block_sum(v, red);
}

__global__ void km_update(KmArgs a, int t, int n_tiles, double *objective)
{
    __shared__ double red[32];
    if (a.ctl->error || a.ctl->converged) return;
    if (blockIdx.x == 0) {
        if (objective) {
            const double J = sum_partials(a.jpart, n_tiles, red);
            if (threadIdx.x == 0) objective[t] = J;
        }
        if (threadIdx.x == 0) {
            a.ctl->moved[(t + 1) & 1] = 0u;   // read by pass t (done), next written by update t + 1
            a.ctl->n_iter = t + 1;
        }
    }
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= a.n_mu) return;
    unsigned long long *q = &a.acc[8 * (int64_t)m];
    if ((q[0] | q[1]) != 0ull) {
        const double sw = u128_to_double(q[0], q[1]);
        const double cx = __ddiv_rn(u128_to_double(q[2], q[3]), sw);
        const double cy = __ddiv_rn(u128_to_double(q[4], q[5]), sw);
        const double cz = __ddiv_rn(u128_to_double(q[6], q[7]), sw);
        if (a.early_stop && (__double_as_longlong(cx) != __double_as_longlong(a.cent[3 * m]) ||
                             __double_as_longlong(cy) != __double_as_longlong(a.cent[3 * m + 1]) ||
                             __double_as_longlong(cz) != __double_as_longlong(a.cent[3 * m + 2])))
            atomicOr(&a.ctl->moved[t & 1], 1u);
        a.cent[3 * m + 0] = cx;
        a.cent[3 * m + 1] = cy;
        a.cent[3 * m + 2] = cz;
        a.c32[m] = make_float4((float)a.cent[3 * m], (float)a.cent[3 * m + 1], (float)a.cent[3 * m + 2], 0.f);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) q[k] = 0ull;
}

__global__ void km_snap(KmArgs a, int64_t n_r)
{
    if (a.ctl->error) return;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_r; r += (int64_t)gridDim.x * blockDim.x) {
        const int m = a.labels[r];
        if (m < 0) continue;
        if ((unsigned long long)__double_as_longlong(a.dist[r]) == a.best[m]) atomicMin(&a.idx_u[m], (unsigned long long)r);
    }
}

__global__ void km_finish(KmArgs a, int max_iter, int n_tiles, int64_t *idx, double *centroids, double *objective,
                          int64_t *stats)
{
    __shared__ double red[32];
    __shared__ int empty_sh;
    if (threadIdx.x == 0) empty_sh = 0;
    __syncthreads();
    const int err = a.ctl->error;
    const double J = sum_partials(a.jpart, n_tiles, red);
    int empty = 0;
    for (int m = threadIdx.x; m < a.n_mu; m += blockDim.x) {
        const unsigned long long u = a.idx_u[m];
        const bool e = err || u == ~0ull;
        idx[m] = e ? -1 : (int64_t)u;
        empty += e ? 1 : 0;
        if (centroids) {
            centroids[3 * m + 0] = a.cent[3 * m + 0];
            centroids[3 * m + 1] = a.cent[3 * m + 1];
            centroids[3 * m + 2] = a.cent[3 * m + 2];
        }
    }
    atomicAdd(&empty_sh, empty);
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nit = a.ctl->converged ? a.ctl->n_iter : max_iter;
        if (objective) {
            objective[max_iter] = J;
            for (int p = nit + 1; p < max_iter; ++p) objective[p] = objective[nit];
        }
        if (stats) {
            stats[0] = nit;
            stats[1] = (int64_t)a.ctl->ties;
            stats[2] = err == 2 ? -2 : (err ? -1 : empty_sh);
            stats[3] = (int64_t)a.ctl->refined;
        }
    }
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

struct WsLayout {
    size_t cent, c32, acc, labels, dist, jpart, best, idx_u, ctl, total;
};

WsLayout ws_layout(int64_t n_r, int n_mu, int n_tiles)
{
    WsLayout L;
    size_t o = 0;
    L.cent = o; o = align256(o + sizeof(double) * 3 * n_mu);
    L.c32 = o; o = align256(o + sizeof(float4) * n_mu);
    L.acc = o; o = align256(o + sizeof(unsigned long long) * 8 * n_mu);
    L.labels = o; o = align256(o + sizeof(int32_t) * n_r);
    L.dist = o; o = align256(o + sizeof(double) * n_r);
    L.jpart = o; o = align256(o + sizeof(double) * n_tiles);
    L.best = o; o = align256(o + sizeof(unsigned long long) * n_mu);
    L.idx_u = o; o = align256(o + sizeof(unsigned long long) * n_mu);
    L.ctl = o; o = align256(o + sizeof(KmCtl));
    L.total = o;
    return L;
}

int bits_of(uint64_t v)
{
    int b = 0;
    while (v) {
        ++b;
        v >>= 1;
    }
    return b;
}

// the dynamic shared-memory limit of the assign kernels, set once per device
// (so that later calls issue only stream-ordered work and can be captured)
isdf_status set_kernel_attributes()
{
    static std::mutex lock;
    static bool done[64] = {};
    int dev = 0;
    ISDF_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return ISDF_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> guard(lock);
    if (done[dev]) return ISDF_OK;
    ISDF_CUDA_TRY(cudaFuncSetAttribute(km_assign<false, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(float4) * kMaxMu)));
    ISDF_CUDA_TRY(cudaFuncSetAttribute(km_assign<true, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(float4) * kMaxMu)));
    ISDF_CUDA_TRY(cudaFuncSetAttribute(km_assign<false, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(float4) * kMaxMu)));
    ISDF_CUDA_TRY(cudaFuncSetAttribute(km_assign<true, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(float4) * kMaxMu)));
    done[dev] = true;
    return ISDF_OK;
}

// CTA tiles of the assignment: 8 x 8 x 8, or 4 x 8 x 8 halves when the grid has fewer than two full
// tiles per SM of the 152 (the halves' own candidate scans cost less than the idle SMs)
struct TilePlan {
    int half, ntx, nty, ntz, n_tiles;
};

TilePlan tile_plan(int nx, int ny, int nz)
{
    TilePlan p;
    p.nty = (ny + TY - 1) / TY;
    p.ntz = (nz + TZ - 1) / TZ;
    const int full = ((nx + TX - 1) / TX) * p.nty * p.ntz;
    p.half = full < 2 * 152 ? 1 : 0;
    const int tx = p.half ? TX / 2 : TX;
    p.ntx = (nx + tx - 1) / tx;
    p.n_tiles = p.ntx * p.nty * p.ntz;
    return p;
}

}  // namespace

extern "C" isdf_status isdf_kmeans_workspace(int32_t nx, int32_t ny, int32_t nz, int32_t n_mu, size_t *ws_bytes)
{
    if (nx < 1 || ny < 1 || nz < 1 || n_mu < 1 || !ws_bytes) return ISDF_ERR_INVALID_ARG;
    const int64_t n_r = (int64_t)nx * ny * nz;
    *ws_bytes = ws_layout(n_r, n_mu, tile_plan(nx, ny, nz).n_tiles).total;
    return ISDF_OK;
}

extern "C" isdf_status isdf_kmeans(const double *w, int32_t nx, int32_t ny, int32_t nz, const double *cell,
                                   int32_t n_mu, const int64_t *init_idx, int32_t max_iter, int32_t flags,
                                   int64_t *idx, double *centroids, double *objective, int32_t *labels,
                                   int64_t *stats, void *ws, size_t ws_bytes, void *stream)
{
    if (nx < 1 || ny < 1 || nz < 1 || !cell || !w || !init_idx || !idx) return ISDF_ERR_INVALID_ARG;
    const int64_t n_r = (int64_t)nx * ny * nz;
    if (n_r >= ((int64_t)1 << 31)) return ISDF_ERR_UNSUPPORTED;
    if (n_mu < 1 || n_mu > n_r || max_iter < 0 || (flags & ~ISDF_KMEANS_EARLY_STOP)) return ISDF_ERR_INVALID_ARG;
    if (n_mu > kMaxMu) return ISDF_ERR_UNSUPPORTED;
    for (int k = 0; k < 3; ++k)
        if (!(cell[k] > 0.0) || cell[k] > 1e300) return ISDF_ERR_INVALID_ARG;
    const TilePlan tp = tile_plan(nx, ny, nz);
    const int ntx = tp.ntx, nty = tp.nty, ntz = tp.ntz;
    const int n_tiles = tp.n_tiles;
    const WsLayout L = ws_layout(n_r, n_mu, n_tiles);
    if (!ws || ws_bytes < L.total || !aligned(ws, 256)) return ISDF_ERR_WORKSPACE;
    char *base = static_cast<char *>(ws);

    KmArgs a;
    a.w = w;
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.hx = cell[0] / nx;
    a.hy = cell[1] / ny;
    a.hz = cell[2] / nz;
    double hmin = a.hx < a.hy ? a.hx : a.hy;
    hmin = hmin < a.hz ? hmin : a.hz;
    a.tie_floor = hmin * hmin;
    a.n_mu = n_mu;
    double lmax = 1.0;
    for (int k = 0; k < 3; ++k) lmax = cell[k] > lmax ? cell[k] : lmax;
    int el = 0;
    frexp(lmax, &el);
    a.s_base = 126 - (bits_of((uint64_t)n_r) + el);
    a.ntx = ntx;
    a.nty = nty;
    a.ntz = ntz;
    a.cent = reinterpret_cast<double *>(base + L.cent);
    a.c32 = reinterpret_cast<float4 *>(base + L.c32);
    a.acc = reinterpret_cast<unsigned long long *>(base + L.acc);
    a.labels = labels ? labels : reinterpret_cast<int32_t *>(base + L.labels);
    a.dist = reinterpret_cast<double *>(base + L.dist);
    a.jpart = reinterpret_cast<double *>(base + L.jpart);
    a.best = reinterpret_cast<unsigned long long *>(base + L.best);
    a.idx_u = reinterpret_cast<unsigned long long *>(base + L.idx_u);
    a.ctl = reinterpret_cast<KmCtl *>(base + L.ctl);
    a.early_stop = (flags & ISDF_KMEANS_EARLY_STOP) ? 1 : 0;
    a.want_obj = objective ? 1 : 0;
    a.lmax = lmax;
    // |float(c) - c| + |float(o) - o| + rounding of their difference, for |c|, |o| <= L
    a.scan_err = (float)(4.0 * 5.9604644775390625e-8 * lmax * 1.01);

    cudaStream_t st = as_stream(stream);
    const size_t smem = sizeof(float4) * (size_t)n_mu;
    ISDF_TRY(set_kernel_attributes());
    const int64_t nmax = n_r > n_mu ? n_r : n_mu;
    const unsigned ginit = (unsigned)((nmax + 255) / 256 < 4096 ? (nmax + 255) / 256 : 4096);
    km_init<<<ginit, 256, 0, st>>>(a, init_idx, n_r); isdf_note_launch();
    km_wmax<<<(unsigned)((n_r + 255) / 256 < 1024 ? (n_r + 255) / 256 : 1024), 256, 0, st>>>(a, n_r); isdf_note_launch();
    km_check_scale<<<1, 32, 0, st>>>(a); isdf_note_launch();
    ISDF_LAUNCH_CHECK();
    // small blocks spread the FP64 divisions of the update over many SMs
    const unsigned gmu = (unsigned)((n_mu + 63) / 64);
    for (int t = 0; t < max_iter; ++t) {
        if (tp.half) km_assign<false, 4><<<n_tiles, 128, smem, st>>>(a, t);
        else km_assign<false, 8><<<n_tiles, kThreads, smem, st>>>(a, t);
        isdf_note_launch();
        km_update<<<gmu, 64, 0, st>>>(a, t, n_tiles, objective); isdf_note_launch();
    }
    if (tp.half) km_assign<true, 4><<<n_tiles, 128, smem, st>>>(a, max_iter);
    else km_assign<true, 8><<<n_tiles, kThreads, smem, st>>>(a, max_iter);
    isdf_note_launch();
    km_snap<<<(unsigned)((n_r + 255) / 256 < 4096 ? (n_r + 255) / 256 : 4096), 256, 0, st>>>(a, n_r); isdf_note_launch();
    km_finish<<<1, 256, 0, st>>>(a, max_iter, n_tiles, idx, centroids, objective, stats); isdf_note_launch();
    ISDF_LAUNCH_CHECK();
    return ISDF_OK;
}

extern "C" isdf_status isdf_kmeans_status(const int64_t *stats, void *stream)
{
    if (!stats) return ISDF_ERR_INVALID_ARG;
    ISDF_CUDA_TRY(cudaStreamSynchronize(as_stream(stream)));
    int64_t h[4] = {0, 0, 0, 0};
    ISDF_CUDA_TRY(cudaMemcpy(h, stats, sizeof(h), cudaMemcpyDeviceToHost));
    if (h[2] == -2) return ISDF_ERR_INVALID_ARG;
    if (h[2] < 0) return ISDF_ERR_NONFINITE;
    return h[2] > 0 ? ISDF_ERR_EMPTY_CLUSTER : ISDF_OK;
}
