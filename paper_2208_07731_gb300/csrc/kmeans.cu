// Step 2: weighted Lloyd K-means on the real-space grid (Sec. 2.2,
// Eq. opt second form, Eq. r_k, Algorithm 1).
//
// Design (one CTA per 4 x 8 x 8 sub-box of the grid, one thread per point):
//  * exact pruning: the CTA bounds every centroid's squared distance to its
//    box from below (LB) and above (UB); only centroids with LB <= min UB can
//    be the nearest one of any point in the box (margins cover rounding);
//  * FP32 screen: each point evaluates its candidates in FP32 in box-local
//    coordinates and keeps the two smallest values; when their gap exceeds a
//    rigorous bound E on |d_fp32 - d_exact| (+ FP64 rounding) the FP32 winner
//    is the FP64 winner. Otherwise the point re-evaluates the close candidates
//    with the FP64 formula ((dx*dx + dy*dy) + dz*dz) and takes the smallest
//    (distance, mu) pair - exactly the brute-force FP64 decision;
//  * exact update: each FP64 product w*x enters as the 128-bit integer
//    floor(w*x*2^s); sums are integer (associative, so the result does not
//    depend on thread or block order), first per CTA in shared memory, then in
//    global memory, with the carry of the low word detected by the adding
//    thread; the update kernel rounds each sum to FP64 and divides once.
#include "common.cuh"

namespace {

constexpr int TX = 4, TY = 8, TZ = 8;
constexpr int kThreads = TX * TY * TZ;   // 256
constexpr int kSlots = 256;              // per-CTA shared accumulators (first candidates)
constexpr int kMaxMu = 8192;

struct KmCtl {
    unsigned long long wmax_bits;
    unsigned long long ties;
    unsigned long long refined;
    unsigned int changed[2];
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
    if (v == 0.0) return r;
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
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

__device__ unsigned long long block_sum_u64(unsigned long long v, unsigned long long *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    unsigned long long s = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;
}

__global__ void km_init(KmArgs a, const int64_t *__restrict__ init_idx, int64_t n_r)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        a.ctl->wmax_bits = 0ull;
        a.ctl->ties = 0ull;
        a.ctl->refined = 0ull;
        a.ctl->changed[0] = 0u;
        a.ctl->changed[1] = 0u;
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

template <bool FINAL>
__global__ void __launch_bounds__(kThreads) km_assign(KmArgs a, int t)
{
    if (a.ctl->error) return;
    if (!FINAL && a.ctl->converged) return;

    extern __shared__ float4 cand[];  // n_mu entries: (qx, qy, qz, mu bits)
    __shared__ unsigned long long slot[kSlots][8];
    __shared__ unsigned int n_cand;
    __shared__ unsigned int qmax_bits;
    __shared__ float minub_sh[kThreads / 32];
    __shared__ double red[kThreads / 32];
    __shared__ unsigned long long redu[kThreads / 32];

    const int tid = threadIdx.x;
    const int b = blockIdx.x;
    const int tz = b % a.ntz, ty = (b / a.ntz) % a.nty, tx = b / (a.ntz * a.nty);
    const int ix0 = tx * TX, iy0 = ty * TY, iz0 = tz * TZ;
    const int ex = min(TX, a.nx - ix0), ey = min(TY, a.ny - iy0), ez = min(TZ, a.nz - iz0);
    const double ox = __dmul_rn((double)ix0, a.hx), oy = __dmul_rn((double)iy0, a.hy), oz = __dmul_rn((double)iz0, a.hz);
    const float Px = (float)((ex - 1) * a.hx), Py = (float)((ey - 1) * a.hy), Pz = (float)((ez - 1) * a.hz);

    if (tid == 0) {
        n_cand = 0u;
        qmax_bits = 0u;
    }
    // pass 1: min over centroids of the largest squared distance to the box
    float mub = INFINITY;
    for (int m = tid; m < a.n_mu; m += kThreads) {
        const float qx = (float)__dsub_rn(a.cent[3 * m + 0], ox);
        const float qy = (float)__dsub_rn(a.cent[3 * m + 1], oy);
        const float qz = (float)__dsub_rn(a.cent[3 * m + 2], oz);
        const float ux = fmaxf(fabsf(qx), fabsf(Px - qx));
        const float uy = fmaxf(fabsf(qy), fabsf(Py - qy));
        const float uz = fmaxf(fabsf(qz), fabsf(Pz - qz));
        mub = fminf(mub, ux * ux + uy * uy + uz * uz);
    }
    for (int o = 16; o > 0; o >>= 1) mub = fminf(mub, __shfl_xor_sync(0xffffffffu, mub, o));
    if ((tid & 31) == 0) minub_sh[tid >> 5] = mub;
    __syncthreads();
    float minub = minub_sh[0];
    for (int i = 1; i < kThreads / 32; ++i) minub = fminf(minub, minub_sh[i]);
    // generous margins: rounding of q and of the float sums is ~1e-7 relative
    const float cut = minub * 1.0001f + 1e-6f * (Px * Px + Py * Py + Pz * Pz) + 1e-30f;

    // pass 2: keep centroids whose smallest squared distance to the box can win
    for (int m = tid; m < a.n_mu; m += kThreads) {
        const float qx = (float)__dsub_rn(a.cent[3 * m + 0], ox);
        const float qy = (float)__dsub_rn(a.cent[3 * m + 1], oy);
        const float qz = (float)__dsub_rn(a.cent[3 * m + 2], oz);
        const float lx = fmaxf(0.f, fmaxf(-qx, qx - Px));
        const float ly = fmaxf(0.f, fmaxf(-qy, qy - Py));
        const float lz = fmaxf(0.f, fmaxf(-qz, qz - Pz));
        const float lb = (lx * lx + ly * ly + lz * lz) * 0.9999f;
        if (lb <= cut) {
            const unsigned j = atomicAdd(&n_cand, 1u);
            cand[j] = make_float4(qx, qy, qz, __int_as_float(m));
            const float qm = fmaxf(fabsf(qx), fmaxf(fabsf(qy), fabsf(qz)));
            atomicMax(&qmax_bits, __float_as_uint(qm));
        }
    }
    __syncthreads();
    const int nc = (int)n_cand;
    const int ns = min(nc, kSlots);
    if (!FINAL)
        for (int i = tid; i < ns * 8; i += kThreads) slot[i >> 3][i & 7] = 0ull;

    // rigorous bound on |d_fp32 - d_exact| (+ FP64 rounding) for this box
    const float Pmax = fmaxf(Px, fmaxf(Py, Pz));
    const float Qmax = __uint_as_float(qmax_bits);
    const double u32 = 5.9604644775390625e-8;  // 2^-24
    const double Tm = ((double)Pmax + (double)Qmax) * (1.0 + 4.0 * u32);
    const double del = 2.0003 * u32 * ((double)Pmax + (double)Qmax);
    const double E = 1.01 * (3.0 * del * (2.0 * Tm + del) + 9.001 * u32 * Tm * Tm + 1.6e-15 * 3.0 * Tm * Tm);

    // this thread's point
    const int lz = tid % TZ, ly = (tid / TZ) % TY, lx = tid / (TZ * TY);
    const bool valid = lx < ex && ly < ey && lz < ez;
    const int ix = ix0 + lx, iy = iy0 + ly, iz = iz0 + lz;
    const int64_t r = ((int64_t)ix * a.ny + iy) * a.nz + iz;
    double jv = 0.0;
    unsigned long long my_ties = 0, my_ref = 0;
    unsigned int my_changed = 0;
    __syncthreads();
    if (valid && nc > 0) {
        const double x = __dmul_rn((double)ix, a.hx), y = __dmul_rn((double)iy, a.hy), z = __dmul_rn((double)iz, a.hz);
        const float px = (float)__dsub_rn(x, ox), py = (float)__dsub_rn(y, oy), pz = (float)__dsub_rn(z, oz);
        float d1 = INFINITY, d2 = INFINITY;
        int j1 = 0;
        for (int j = 0; j < nc; ++j) {
            const float4 q = cand[j];
            const float dx = px - q.x, dy = py - q.y, dz = pz - q.z;
            const float d = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            if (d < d1) {
                d2 = d1;
                d1 = d;
                j1 = j;
            } else if (d < d2) {
                d2 = d;
            }
        }
        const double dd1 = (double)d1;
        const double gap = 2.0 * E + 2.0e-12 * fmax(dd1 + E, a.tie_floor) + 1.0e-14 * (dd1 + E);
        int win_j = j1, win_mu = __float_as_int(cand[j1].w);
        double win_d;
        if ((double)d2 - dd1 > gap) {
            win_d = dist2_fp64(x, y, z, a.cent[3 * win_mu], a.cent[3 * win_mu + 1], a.cent[3 * win_mu + 2]);
        } else {
            // FP64 decision over the candidates that can still win
            my_ref = 1;
            double b1 = INFINITY, b2 = INFINITY;
            int bm = 0x7fffffff, bj = 0;
            const double lim = dd1 + gap;
            for (int j = 0; j < nc; ++j) {
                const float4 q = cand[j];
                const float dx = px - q.x, dy = py - q.y, dz = pz - q.z;
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
            if (a.n_mu > 1 && __dsub_rn(b2, b1) <= 1e-12 * fmax(b1, a.tie_floor)) my_ties = 1;
        }
        const double wr = a.w[r];
        jv = __dmul_rn(wr, win_d);
        if (!FINAL) {
            my_changed = (a.labels[r] != win_mu) ? 1u : 0u;
            a.labels[r] = win_mu;
            const int s = fixed_scale(a);
            unsigned long long *dst = (win_j < kSlots) ? &slot[win_j][0] : &a.acc[8 * (int64_t)win_mu];
            atomic_add_u128(dst + 0, fixed_of(wr, s));
            atomic_add_u128(dst + 2, fixed_of(__dmul_rn(wr, x), s));
            atomic_add_u128(dst + 4, fixed_of(__dmul_rn(wr, y), s));
            atomic_add_u128(dst + 6, fixed_of(__dmul_rn(wr, z), s));
        } else {
            a.labels[r] = win_mu;
            a.dist[r] = win_d;
            atomicMin(&a.best[win_mu], (unsigned long long)__double_as_longlong(win_d));
        }
    }
    const double jt = block_sum(jv, red);
    if (tid == 0) a.jpart[b] = jt;
    const unsigned long long tt = block_sum_u64(my_ties, redu);
    if (tid == 0 && tt) atomicAdd(&a.ctl->ties, tt);
    const unsigned long long rr = block_sum_u64(my_ref, redu);
    if (tid == 0 && rr) atomicAdd(&a.ctl->refined, rr);
    if (!FINAL) {
        const unsigned long long cc = block_sum_u64(my_changed, redu);
        if (tid == 0 && cc) atomicAdd(&a.ctl->changed[t & 1], (unsigned int)cc);
        __syncthreads();
        for (int j = tid; j < ns; j += kThreads) {
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
    const unsigned int changed = a.ctl->changed[t & 1];
    if (blockIdx.x == 0) {
        const double J = sum_partials(a.jpart, n_tiles, red);
        if (threadIdx.x == 0) {
            if (objective) objective[t] = J;
            a.ctl->changed[(t + 1) & 1] = 0u;
        }
    }
    if (a.early_stop && t > 0 && changed == 0u) {
        // labels repeated: the sums equal the previous ones, so the centroids
        // would not move; later passes are skipped
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.ctl->converged = 1;
            a.ctl->n_iter = t;
        }
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl->n_iter = t + 1;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= a.n_mu) return;
    unsigned long long *q = &a.acc[8 * (int64_t)m];
    if ((q[0] | q[1]) != 0ull) {
        const double sw = u128_to_double(q[0], q[1]);
        a.cent[3 * m + 0] = __ddiv_rn(u128_to_double(q[2], q[3]), sw);
        a.cent[3 * m + 1] = __ddiv_rn(u128_to_double(q[4], q[5]), sw);
        a.cent[3 * m + 2] = __ddiv_rn(u128_to_double(q[6], q[7]), sw);
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
            stats[2] = err ? -1 : empty_sh;
            stats[3] = (int64_t)a.ctl->refined;
        }
    }
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

struct WsLayout {
    size_t cent, acc, labels, dist, jpart, best, idx_u, ctl, total;
};

WsLayout ws_layout(int64_t n_r, int n_mu, int n_tiles)
{
    WsLayout L;
    size_t o = 0;
    L.cent = o; o = align256(o + sizeof(double) * 3 * n_mu);
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

}  // namespace

extern "C" isdf_status isdf_kmeans_workspace(int32_t nx, int32_t ny, int32_t nz, int32_t n_mu, size_t *ws_bytes)
{
    if (nx < 1 || ny < 1 || nz < 1 || n_mu < 1 || !ws_bytes) return ISDF_ERR_INVALID_ARG;
    const int64_t n_r = (int64_t)nx * ny * nz;
    const int n_tiles = ((nx + TX - 1) / TX) * ((ny + TY - 1) / TY) * ((nz + TZ - 1) / TZ);
    *ws_bytes = ws_layout(n_r, n_mu, n_tiles).total;
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
    const int ntx = (nx + TX - 1) / TX, nty = (ny + TY - 1) / TY, ntz = (nz + TZ - 1) / TZ;
    const int n_tiles = ntx * nty * ntz;
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
    a.acc = reinterpret_cast<unsigned long long *>(base + L.acc);
    a.labels = labels ? labels : reinterpret_cast<int32_t *>(base + L.labels);
    a.dist = reinterpret_cast<double *>(base + L.dist);
    a.jpart = reinterpret_cast<double *>(base + L.jpart);
    a.best = reinterpret_cast<unsigned long long *>(base + L.best);
    a.idx_u = reinterpret_cast<unsigned long long *>(base + L.idx_u);
    a.ctl = reinterpret_cast<KmCtl *>(base + L.ctl);
    a.early_stop = (flags & ISDF_KMEANS_EARLY_STOP) ? 1 : 0;

    cudaStream_t st = as_stream(stream);
    const size_t smem = sizeof(float4) * (size_t)n_mu;
    ISDF_CUDA_TRY(cudaFuncSetAttribute(km_assign<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(float4) * kMaxMu)));
    ISDF_CUDA_TRY(cudaFuncSetAttribute(km_assign<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(float4) * kMaxMu)));
    const int64_t nmax = n_r > n_mu ? n_r : n_mu;
    const unsigned ginit = (unsigned)((nmax + 255) / 256 < 4096 ? (nmax + 255) / 256 : 4096);
    km_init<<<ginit, 256, 0, st>>>(a, init_idx, n_r); isdf_note_launch();
    km_wmax<<<(unsigned)((n_r + 255) / 256 < 1024 ? (n_r + 255) / 256 : 1024), 256, 0, st>>>(a, n_r); isdf_note_launch();
    km_check_scale<<<1, 32, 0, st>>>(a); isdf_note_launch();
    ISDF_LAUNCH_CHECK();
    // small blocks spread the FP64 divisions of the update over many SMs
    const unsigned gmu = (unsigned)((n_mu + 63) / 64);
    for (int t = 0; t < max_iter; ++t) {
        km_assign<false><<<n_tiles, kThreads, smem, st>>>(a, t); isdf_note_launch();
        km_update<<<gmu, 64, 0, st>>>(a, t, n_tiles, objective); isdf_note_launch();
    }
    km_assign<true><<<n_tiles, kThreads, smem, st>>>(a, max_iter); isdf_note_launch();
    km_snap<<<(unsigned)((n_r + 255) / 256 < 4096 ? (n_r + 255) / 256 : 4096), 256, 0, st>>>(a, n_r); isdf_note_launch();
    km_finish<<<1, 256, 0, st>>>(a, max_iter, n_tiles, idx, centroids, objective, stats); isdf_note_launch();
    ISDF_LAUNCH_CHECK();
    return ISDF_OK;
}
