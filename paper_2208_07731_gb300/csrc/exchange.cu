// ISDF exchange application (Sec. 2.3): the projected exchange integrals
// V_mu = v * zeta_mu of Eq. V_mu for every interpolation vector, solved in
// reciprocal space on the periodic FFT grid, and the application of Eq. v2,
//     (V_X psi_j)(r) = -sum_mu V_mu(r) sum_i phi_i(r) phi_i*(r_mu) psi_j(r_mu)
//                    = -[(V o (Phi Phi_mu^H)) Psi_mu](r, j).
//
// The 3-D FFTs run over all N_mu columns of the N_r x N_mu matrix at once:
// every kernel launch transforms lines along one grid axis, one CTA per
// (line, tile of TM adjacent columns), so each grid point contributes one
// contiguous 256-byte chunk (TM complex numbers) to a coalesced load. The
// line is transformed in shared memory by a Stockham autosort FFT (radices
// 4, 2, 3 and 5; the published formulation for GPUs that writes every stage
// in natural order). Five passes over the data: forward x, forward y, then
// forward z, multiplication by the kernel's Fourier coefficients (with the
// 1/N_r of the inverse) and inverse z fused in one pass, inverse y, inverse x.
// The products of the application run on the tcgen05 tensor cores: in
// ISDF_MIXED mode as split-FP16 products with FP32 accumulation, the Hadamard
// product with V fused into the first product's epilogue (mixed.cu); in
// ISDF_FP64 mode (or for sizes the split kernels do not take) by exact
// integer slicing with FP64-grade results (ozaki.cuh), V o (Phi Phi_mu^H)
// formed between them.
#include <math.h>

#include "common.cuh"
#include "mixed.cuh"
#include "ozaki.cuh"
#include "zgemm.cuh"

namespace {

constexpr int FFT_THREADS = 256;
constexpr int FFT_NMAX = 256;       // longest axis
constexpr int FFT_MAXSTAGE = 12;

struct Radices {
    int count;
    int r[FFT_MAXSTAGE];
};

struct KernelParams {
    int kind;           // ISDF_KERNEL_COULOMB or ISDF_KERNEL_ERFC
    double omega;
    double scale;       // 1 / N_r
    double gfac[3];     // 2 pi / L_a
    double q[3];
    int n[3];
};

template <typename T> struct Real;
template <> struct Real<double2> { typedef double type; };
template <> struct Real<float2> { typedef float type; };

template <typename T> __device__ __forceinline__ T cadd(T a, T b) { a.x += b.x; a.y += b.y; return a; }
template <typename T> __device__ __forceinline__ T csub(T a, T b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename T> __device__ __forceinline__ T cmul_t(T a, T b)
{
    T c;
    c.x = a.x * b.x - a.y * b.y;
    c.y = a.x * b.y + a.y * b.x;
    return c;
}
// multiply by -i (forward) or +i (inverse)
template <typename T> __device__ __forceinline__ T rot(T a, bool inv)
{
    T c;
    if (inv) { c.x = -a.y; c.y = a.x; }
    else     { c.x = a.y;  c.y = -a.x; }
    return c;
}

// one Stockham stage of radix R over TM columns: input index j + r n/R, output
// (j / Ns) Ns R + j % Ns + r Ns, twiddle exp(-+2 pi i r (j % Ns) / (Ns R))
// (NC, NSC > 0: the length and Ns as compile-time constants, so that every index division is by a constant)
template <typename T, int TM, int R, int NC = 0, int NSC = 0>
__device__ __forceinline__ void fft_stage(const T *__restrict__ in, T *__restrict__ out, const T *tw, int n_rt,
                                          int Ns_rt, bool inv)
{
    typedef typename Real<T>::type RT;
    const int n = NC > 0 ? NC : n_rt;
    const int Ns = NC > 0 ? NSC : Ns_rt;
    const int nb = n / R;
    const int step = n / (Ns * R);
    for (int it = threadIdx.x; it < nb * TM; it += FFT_THREADS) {
        const int c = it % TM, j = it / TM;
        const int k = j % Ns;
        T a[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            a[r] = in[(j + r * nb) * TM + c];
            if (r > 0 && k > 0) {
                T w = tw[r * k * step];
                if (inv) w.y = -w.y;
                a[r] = cmul_t(a[r], w);
            }
        }
        T b[R];
        if (R == 2) {
            b[0] = cadd(a[0], a[1]);
            b[1] = csub(a[0], a[1]);
        } else if (R == 4) {
            const T t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
            const T t2 = cadd(a[1], a[3]), t3 = rot(csub(a[1], a[3]), inv);
            b[0] = cadd(t0, t2);
            b[2] = csub(t0, t2);
            b[1] = cadd(t1, t3);
            b[3] = csub(t1, t3);
        } else if (R == 3) {
            const RT s = (RT)0.86602540378443864676;   // sin(2 pi / 3)
            const T t = cadd(a[1], a[2]);
            T m;
            m.x = a[0].x - (RT)0.5 * t.x;
            m.y = a[0].y - (RT)0.5 * t.y;
            T d = rot(csub(a[1], a[2]), inv);
            d.x *= s;
            d.y *= s;
            b[0] = cadd(a[0], t);
            b[1] = cadd(m, d);
            b[2] = csub(m, d);
        } else {
            // generic odd radix: b_s = sum_r a_r w^(r s), w^t = tw[t n / R]
#pragma unroll
            for (int s2 = 0; s2 < R; ++s2) {
                T acc = a[0];
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    T w = tw[((r * s2) % R) * nb];
                    if (inv) w.y = -w.y;
                    acc = cadd(acc, cmul_t(a[r], w));
                }
                b[s2] = acc;
            }
        }
        const int base = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) out[(base + r * Ns) * TM + c] = b[r];
    }
}

// all stages of one direction; returns the buffer holding the result
template <typename T, int TM>
__device__ T *fft_line(T *b0, T *b1, const T *tw, int n, const Radices &rd, bool inv)
{
    T *in = b0, *out = b1;
    int Ns = 1;
    for (int s = 0; s < rd.count; ++s) {
        const int R = rd.r[s];
        if (R == 4) fft_stage<T, TM, 4>(in, out, tw, n, Ns, inv);
        else if (R == 2) fft_stage<T, TM, 2>(in, out, tw, n, Ns, inv);
        else if (R == 3) fft_stage<T, TM, 3>(in, out, tw, n, Ns, inv);
        else fft_stage<T, TM, 5>(in, out, tw, n, Ns, inv);
        __syncthreads();
        Ns *= R;
        T *t = in;
        in = out;
        out = t;
    }
    return in;
}

// radix sequence of a length (4s first, then 2, 3, 5), usable in constant expressions
struct RadPlan {
    int count;
    int r[FFT_MAXSTAGE];
};
constexpr RadPlan rad_plan(int n)
{
    RadPlan p{0, {}};
    while (n % 4 == 0 && p.count < FFT_MAXSTAGE) { p.r[p.count++] = 4; n /= 4; }
    while (n % 2 == 0 && p.count < FFT_MAXSTAGE) { p.r[p.count++] = 2; n /= 2; }
    while (n % 3 == 0 && p.count < FFT_MAXSTAGE) { p.r[p.count++] = 3; n /= 3; }
    while (n % 5 == 0 && p.count < FFT_MAXSTAGE) { p.r[p.count++] = 5; n /= 5; }
    return p;
}

// all stages for a compile-time length NC, from stage S with Ns = NS; returns the result buffer
template <typename T, int TM, int NC, int S, int NS>
__device__ __forceinline__ T *fft_line_ct(T *in, T *out, const T *tw, bool inv)
{
    constexpr RadPlan P = rad_plan(NC);
    if constexpr (S == P.count) {
        return in;
    } else {
        constexpr int R = P.r[S];
        fft_stage<T, TM, R, NC, NS>(in, out, tw, NC, NS, inv);
        __syncthreads();
        return fft_line_ct<T, TM, NC, S + 1, NS * R>(out, in, tw, inv);
    }
}

// signed FFT frequency of index k on an axis of n points (the Nyquist index n/2 reads as -n/2)
__device__ __forceinline__ int freq(int k, int n) { return k <= (n - 1) / 2 ? k : k - n; }

// Fourier coefficient of the interaction at G + q, times 1/N_r
__device__ double kernel_value(const KernelParams &kp, int kx, int ky, int kz)
{
    const double gx = kp.gfac[0] * freq(kx, kp.n[0]) + kp.q[0];
    const double gy = kp.gfac[1] * freq(ky, kp.n[1]) + kp.q[1];
    const double gz = kp.gfac[2] * freq(kz, kp.n[2]) + kp.q[2];
    const double g2 = gx * gx + gy * gy + gz * gz;
    const double four_pi = 12.566370614359172954;
    double v;
    if (kp.kind == ISDF_KERNEL_COULOMB)
        v = g2 > 0.0 ? four_pi / g2 : 0.0;
    else
        v = g2 > 0.0 ? -four_pi * expm1(-g2 / (4.0 * kp.omega * kp.omega)) / g2
                     : 3.14159265358979323846 / (kp.omega * kp.omega);
    return v * kp.scale;
}

// One launch: lines along one axis (points p at rows base + p * pstride, base =
// (l / d) S1 + (l % d) S2) x tiles of TM columns. FUSED (the last axis): forward
// FFT, multiplication by the kernel, inverse FFT.
// NC > 0: the axis length as a compile-time constant (n is then ignored).
template <typename T, int TM, bool FUSED, int NC>
__global__ void __launch_bounds__(FFT_THREADS) fft_lines(const T *in, int64_t ld_in, T *out, int64_t ld_out, int ncol,
                                                         int n_arg, int64_t pstride, int64_t lines, int64_t d,
                                                         int64_t S1, int64_t S2, const T *tw_g, Radices rd,
                                                         int inverse, KernelParams kp)
{
    const int n = NC > 0 ? NC : n_arg;
    typedef typename Real<T>::type RT;
    extern __shared__ __align__(16) unsigned char fft_smem[];
    T *b0 = reinterpret_cast<T *>(fft_smem);
    T *b1 = b0 + n * TM;
    T *tw = b1 + n * TM;
    RT *kv = reinterpret_cast<RT *>(tw + n);
    const int64_t l = (int64_t)blockIdx.z * 32768 + blockIdx.y;
    if (l >= lines) return;
    const int col0 = blockIdx.x * TM;
    const int64_t base = (l / d) * S1 + (l % d) * S2;
    for (int t = threadIdx.x; t < n; t += FFT_THREADS) tw[t] = tw_g[t];
    if (FUSED) {
        // the line is (kx, ky) = (l / n_y, l % n_y) of the z pass
        const int kx = (int)(l / kp.n[1]), ky = (int)(l % kp.n[1]);
        for (int t = threadIdx.x; t < n; t += FFT_THREADS) kv[t] = (RT)kernel_value(kp, kx, ky, t);
    }
    for (int it = threadIdx.x; it < n * TM; it += FFT_THREADS) {
        const int c = it % TM, p = it / TM;
        T x;
        x.x = 0;
        x.y = 0;
        if (col0 + c < ncol) x = in[(base + p * pstride) * ld_in + col0 + c];
        b0[it] = x;
    }
    __syncthreads();
    T *res;
    if constexpr (NC > 0) res = fft_line_ct<T, TM, NC, 0, 1>(b0, b1, tw, FUSED ? false : inverse != 0);
    else res = fft_line<T, TM>(b0, b1, tw, n, rd, FUSED ? false : inverse != 0);
    if (FUSED) {
        for (int it = threadIdx.x; it < n * TM; it += FFT_THREADS) {
            const RT s = kv[it / TM];
            res[it].x *= s;
            res[it].y *= s;
        }
        __syncthreads();
        T *other = res == b0 ? b1 : b0;
        if constexpr (NC > 0) res = fft_line_ct<T, TM, NC, 0, 1>(res, other, tw, true);
        else res = fft_line<T, TM>(res, other, tw, n, rd, true);
    }
    for (int it = threadIdx.x; it < n * TM; it += FFT_THREADS) {
        const int c = it % TM, p = it / TM;
        if (col0 + c < ncol) out[(base + p * pstride) * ld_out + col0 + c] = res[it];
    }
}

// twiddle table exp(-2 pi i t / n), t < n
template <typename T>
__global__ void twiddles(T *tw, int n)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    double s, c;
    sincospi(-2.0 * t / n, &s, &c);
    tw[t].x = c;
    tw[t].y = s;
}

// rows idx[mu] of an n_r x n matrix, widened to complex128; bad indices give zero rows and a flag
template <typename T>
__global__ void gather_rows(const T *x, int64_t ld, int n, int64_t n_r, const int64_t *idx, int n_mu, double2 *out,
                            int *err)
{
    const int64_t tot = (int64_t)n_mu * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int mu = (int)(e / n), i = (int)(e % n);
        const int64_t r = idx[mu];
        if (r < 0 || r >= n_r) {
            out[e] = make_double2(0.0, 0.0);
            if (i == 0) atomicExch(err, 1);
        } else {
            out[e] = cload(x, r * ld + i);
        }
    }
}

// G <- G o V over a block of rows (G: rows x n_mu, leading dimension n_mu)
template <typename T>
__global__ void hadamard_v(double2 *G, const T *V, int64_t ldv, int rows, int n_mu)
{
    const int64_t tot = (int64_t)rows * n_mu;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / n_mu;
        const int mu = (int)(e % n_mu);
        G[e] = cmul(G[e], cload(V, r * ldv + mu));
    }
}

unsigned grid_for(int64_t tot)
{
    const int64_t b = (tot + 255) / 256;
    return (unsigned)(b < 16384 ? (b > 0 ? b : 1) : 16384);
}

bool factor(int n, Radices *rd)
{
    rd->count = 0;
    int m = n;
    while (m % 4 == 0 && rd->count < FFT_MAXSTAGE) { rd->r[rd->count++] = 4; m /= 4; }
    while (m % 2 == 0 && rd->count < FFT_MAXSTAGE) { rd->r[rd->count++] = 2; m /= 2; }
    while (m % 3 == 0 && rd->count < FFT_MAXSTAGE) { rd->r[rd->count++] = 3; m /= 3; }
    while (m % 5 == 0 && rd->count < FFT_MAXSTAGE) { rd->r[rd->count++] = 5; m /= 5; }
    return m == 1;
}

template <typename T> constexpr int tile_cols() { return 256 / (int)sizeof(T); }   // 256 bytes per grid point

template <typename T>
size_t fft_smem_bytes(int n)
{
    return (size_t)(2 * tile_cols<T>() + 1) * n * sizeof(T) + (size_t)n * sizeof(typename Real<T>::type);
}

}  // namespace

struct isdf_exchange {
    int n[3];
    int64_t n_r;
    double cell[3];
    int n_mu, n_phi, n_psi, orb_dtype, mode, kind;
    double omega, q[3];
    int64_t max_rows;
    Radices rd[3];
    void *tw[3];                // twiddle tables (complex128 in ISDF_FP64 mode, complex64 in ISDF_MIXED)
    double2 *phi_mu, *psi_mu;   // gathered rows, complex128
    double2 *blkG;              // max_rows x n_mu
    OzWork oz;
    MixedExchange *mixed;       // split-FP16 tensor-core products (ISDF_MIXED), or NULL
    int *flags;                 // [0]: Ozaki bounded-wait error, [1]: bad interpolation index
};

namespace {

// one pass: the kernel specialised for the axis length when it is one of the common grid sizes
template <typename T, bool FUSED, int NC>
isdf_status launch_pass(dim3 grid, size_t smem, cudaStream_t st, const T *src, int64_t lds, T *dst, int64_t ldd,
                        int ncol, int n, int64_t pstride, int64_t lines, int64_t d, int64_t S1, int64_t S2,
                        const T *tw, const Radices &rd, int inverse, const KernelParams &kp)
{
    constexpr int TM = tile_cols<T>();
    static bool attr_set[64] = {false};
    int dev = 0;
    ISDF_CUDA_TRY(cudaGetDevice(&dev));
    if (dev >= 64 || !attr_set[dev]) {
        ISDF_CUDA_TRY(cudaFuncSetAttribute(fft_lines<T, TM, FUSED, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)fft_smem_bytes<T>(FFT_NMAX)));
        // the whole unified L1/shared array as shared memory: several line tiles resident per SM
        ISDF_CUDA_TRY(cudaFuncSetAttribute(fft_lines<T, TM, FUSED, NC>,
                                           cudaFuncAttributePreferredSharedMemoryCarveout,
                                           (int)cudaSharedmemCarveoutMaxShared));
        if (dev < 64) attr_set[dev] = true;
    }
    fft_lines<T, TM, FUSED, NC><<<grid, FFT_THREADS, smem, st>>>(src, lds, dst, ldd, ncol, n, pstride, lines, d, S1, S2,
                                                                tw, rd, inverse, kp);
    isdf_note_launch();
    ISDF_LAUNCH_CHECK();
    return ISDF_OK;
}

template <typename T, bool FUSED>
isdf_status dispatch_pass(dim3 grid, size_t smem, cudaStream_t st, const T *src, int64_t lds, T *dst, int64_t ldd,
                          int ncol, int n, int64_t pstride, int64_t lines, int64_t d, int64_t S1, int64_t S2,
                          const T *tw, const Radices &rd, int inverse, const KernelParams &kp)
{
#define FFT_CASE(NV)                                                                                            \
    case NV:                                                                                                    \
        return launch_pass<T, FUSED, NV>(grid, smem, st, src, lds, dst, ldd, ncol, n, pstride, lines, d, S1, S2, \
                                         tw, rd, inverse, kp);
    switch (n) {
        FFT_CASE(24)
        FFT_CASE(48)
        FFT_CASE(64)
        FFT_CASE(72)
        FFT_CASE(96)
        FFT_CASE(128)
        default:
            return launch_pass<T, FUSED, 0>(grid, smem, st, src, lds, dst, ldd, ncol, n, pstride, lines, d, S1, S2, tw,
                                            rd, inverse, kp);
    }
#undef FFT_CASE
}

template <typename T>
isdf_status potential(isdf_exchange *ex, const T *theta, int64_t ldt, T *v, int64_t ldv, cudaStream_t st)
{
    constexpr int TM = tile_cols<T>();
    const int nx = ex->n[0], ny = ex->n[1], nz = ex->n[2];
    KernelParams kp;
    kp.kind = ex->kind;
    kp.omega = ex->omega;
    kp.scale = 1.0 / (double)ex->n_r;
    for (int a = 0; a < 3; ++a) {
        kp.gfac[a] = 6.283185307179586477 / ex->cell[a];
        kp.q[a] = ex->q[a];
        kp.n[a] = ex->n[a];
    }
    const unsigned tiles = (unsigned)((ex->n_mu + TM - 1) / TM);
    // axis a: pstride, lines, d, S1, S2
    struct Pass {
        int axis;
        int64_t pstride, lines, d, S1, S2;
        int inverse;
        bool fused;
    };
    const int64_t yz = (int64_t)ny * nz;
    const Pass passes[5] = {
        {0, yz, yz, yz, 0, 1, 0, false},                  // x: lines (iy, iz), base = iy nz + iz
        {1, nz, (int64_t)nx * nz, nz, yz, 1, 0, false},   // y: lines (ix, iz), base = ix ny nz + iz
        {2, 1, (int64_t)nx * ny, 1, nz, 0, 0, true},      // z: lines (ix, iy), base = (ix ny + iy) nz
        {1, nz, (int64_t)nx * nz, nz, yz, 1, 1, false},
        {0, yz, yz, yz, 0, 1, 1, false},
    };
    for (int s = 0; s < 5; ++s) {
        const Pass &P = passes[s];
        const int n = ex->n[P.axis];
        const dim3 grid(tiles, (unsigned)(P.lines < 32768 ? P.lines : 32768), (unsigned)((P.lines + 32767) / 32768));
        const size_t smem = fft_smem_bytes<T>(n);
        const T *src = s == 0 ? theta : v;
        const int64_t lds = s == 0 ? ldt : ldv;
        const T *tw = static_cast<const T *>(ex->tw[P.axis]);
        if (P.fused)
            ISDF_TRY((dispatch_pass<T, true>(grid, smem, st, src, lds, v, ldv, ex->n_mu, n, P.pstride, P.lines, P.d, P.S1,
                                             P.S2, tw, ex->rd[P.axis], 0, kp)));
        else
            ISDF_TRY((dispatch_pass<T, false>(grid, smem, st, src, lds, v, ldv, ex->n_mu, n, P.pstride, P.lines, P.d,
                                              P.S1, P.S2, tw, ex->rd[P.axis], P.inverse, kp)));
    }
    return ISDF_OK;
}

template <typename T>
isdf_status alloc(T **p, size_t count)
{
    *p = nullptr;
    ISDF_CUDA_TRY(cudaMalloc((void **)p, sizeof(T) * (count ? count : 1)));
    return ISDF_OK;
}

ZOperand opnd(const void *p, int64_t s0, int64_t s1, int conj, int type)
{
    ZOperand o;
    o.p = p;
    o.s0 = s0;
    o.s1 = s1;
    o.conj = conj;
    o.type = type;
    return o;
}

ZGemm product(int M, int N, int K, ZOperand A, ZOperand B, void *C, int64_t ldc, double alpha)
{
    ZGemm g = {};
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
    g.beta = 0;
    g.splits = 1;
    g.tile = 64;
    g.batch = 1;
    return g;
}

void release(isdf_exchange *ex)
{
    if (!ex) return;
    for (int a = 0; a < 3; ++a) cudaFree(ex->tw[a]);
    cudaFree(ex->phi_mu);
    cudaFree(ex->psi_mu);
    cudaFree(ex->blkG);
    cudaFree(ex->oz.sa);
    cudaFree(ex->oz.sb);
    cudaFree(ex->oz.ma);
    cudaFree(ex->oz.mb);
    cudaFree(ex->flags);
    mixed_exchange_release(ex->mixed);
    delete ex;
}

}  // namespace

extern "C" isdf_status isdf_exchange_create(isdf_exchange **out, int32_t nx, int32_t ny, int32_t nz,
                                            const double *cell, int32_t n_mu, int32_t n_phi, int32_t n_psi,
                                            int32_t orb_dtype, int32_t mode, int32_t kernel, double omega,
                                            const double *q, int64_t max_rows, void *stream)
{
    if (!out || !cell) return ISDF_ERR_INVALID_ARG;
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || n_mu < 1 || n_phi < 1 || n_psi < 1 || max_rows < 1)
        return ISDF_ERR_INVALID_ARG;
    if (orb_dtype != ISDF_C128 && orb_dtype != ISDF_C64) return ISDF_ERR_INVALID_ARG;
    if (mode != ISDF_FP64 && mode != ISDF_MIXED) return ISDF_ERR_INVALID_ARG;
    if (kernel != ISDF_KERNEL_COULOMB && kernel != ISDF_KERNEL_ERFC) return ISDF_ERR_INVALID_ARG;
    if (kernel == ISDF_KERNEL_ERFC && !(omega > 0.0)) return ISDF_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (!(cell[a] > 0.0)) return ISDF_ERR_INVALID_ARG;
    const int64_t n_r = (int64_t)nx * ny * nz;
    if (n_mu > n_r) return ISDF_ERR_INVALID_ARG;
    if (nx > FFT_NMAX || ny > FFT_NMAX || nz > FFT_NMAX || n_mu > 8192 || n_phi > 4096 || n_psi > 4096)
        return ISDF_ERR_UNSUPPORTED;
    isdf_exchange *ex = new isdf_exchange();
    ex->n[0] = nx;
    ex->n[1] = ny;
    ex->n[2] = nz;
    ex->n_r = n_r;
    for (int a = 0; a < 3; ++a) {
        ex->cell[a] = cell[a];
        ex->q[a] = q ? q[a] : 0.0;
        if (!factor(ex->n[a], &ex->rd[a])) {
            delete ex;
            return ISDF_ERR_UNSUPPORTED;   // axis lengths are products of 2, 3 and 5
        }
    }
    ex->n_mu = n_mu;
    ex->n_phi = n_phi;
    ex->n_psi = n_psi;
    ex->orb_dtype = orb_dtype;
    ex->mode = mode;
    ex->kind = kernel;
    ex->omega = omega;
    ex->max_rows = max_rows < n_r ? max_rows : n_r;
    cudaStream_t st = as_stream(stream);
#define EX_TRY(expr)                      \
    do {                                  \
        isdf_status s_ = (expr);          \
        if (s_ != ISDF_OK) {              \
            release(ex);                  \
            return s_;                    \
        }                                 \
    } while (0)
    for (int a = 0; a < 3; ++a) {
        const int n = ex->n[a];
        if (mode == ISDF_FP64) {
            double2 *t;
            EX_TRY(alloc(&t, n));
            ex->tw[a] = t;
            twiddles<double2><<<(n + 127) / 128, 128, 0, st>>>(t, n);
        } else {
            float2 *t;
            EX_TRY(alloc(&t, n));
            ex->tw[a] = t;
            twiddles<float2><<<(n + 127) / 128, 128, 0, st>>>(t, n);
        }
        isdf_note_launch();
        if (cudaGetLastError() != cudaSuccess) {
            release(ex);
            return ISDF_ERR_CUDA;
        }
    }
    EX_TRY(alloc(&ex->phi_mu, (size_t)n_mu * n_phi));
    EX_TRY(alloc(&ex->psi_mu, (size_t)n_mu * n_psi));
    if (mode == ISDF_MIXED && mixed_exchange_supported(n_phi, n_psi, n_mu)) {
        EX_TRY(mixed_exchange_create(&ex->mixed, n_r, n_phi, n_psi, n_mu, ex->max_rows));
    } else {
        EX_TRY(alloc(&ex->blkG, (size_t)ex->max_rows * n_mu));
        size_t ha1, hb1, ra1, rb1, ha2, hb2, ra2, rb2;
        oz_sizes((int)ex->max_rows, n_mu, n_phi, 1, &ha1, &hb1, &ra1, &rb1);
        oz_sizes((int)ex->max_rows, n_psi, n_mu, 1, &ha2, &hb2, &ra2, &rb2);
        ex->oz.cap_a = ha1 > ha2 ? ha1 : ha2;
        ex->oz.cap_b = hb1 > hb2 ? hb1 : hb2;
        ex->oz.cap_ma = ra1 > ra2 ? ra1 : ra2;
        ex->oz.cap_mb = rb1 > rb2 ? rb1 : rb2;
        EX_TRY(alloc(&ex->oz.sa, ex->oz.cap_a));
        EX_TRY(alloc(&ex->oz.sb, ex->oz.cap_b));
        EX_TRY(alloc(&ex->oz.ma, ex->oz.cap_ma));
        EX_TRY(alloc(&ex->oz.mb, ex->oz.cap_mb));
    }
    ex->oz.gsum = nullptr;
    ex->oz.cap_g = 0;
    EX_TRY(alloc(&ex->flags, 2));
    if (cudaMemsetAsync(ex->flags, 0, 2 * sizeof(int), st) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        release(ex);
        return ISDF_ERR_CUDA;
    }
#undef EX_TRY
    *out = ex;
    return ISDF_OK;
}

extern "C" isdf_status isdf_exchange_potential(isdf_exchange *ex, const void *theta, int64_t ld_theta, void *v,
                                               int64_t ld_v, void *stream)
{
    if (!ex || !theta || !v || ld_theta < ex->n_mu || ld_v < ex->n_mu) return ISDF_ERR_INVALID_ARG;
    const size_t el = ex->mode == ISDF_FP64 ? 16 : 8;
    if (!aligned(theta, el) || !aligned(v, el)) return ISDF_ERR_INVALID_ARG;
    cudaStream_t st = as_stream(stream);
    if (ex->mode == ISDF_FP64)
        return potential<double2>(ex, static_cast<const double2 *>(theta), ld_theta, static_cast<double2 *>(v), ld_v,
                                  st);
    return potential<float2>(ex, static_cast<const float2 *>(theta), ld_theta, static_cast<float2 *>(v), ld_v, st);
}

extern "C" isdf_status isdf_exchange_apply(isdf_exchange *ex, const void *phi, int64_t ld_phi, const void *psi,
                                           int64_t ld_psi, const int64_t *idx, const void *v, int64_t ld_v,
                                           int64_t row_begin, int64_t row_count, void *out, int64_t ld_out,
                                           void *stream)
{
    if (!ex || !phi || !psi || !idx || !v || !out) return ISDF_ERR_INVALID_ARG;
    if (ld_phi < ex->n_phi || ld_psi < ex->n_psi || ld_v < ex->n_mu || ld_out < ex->n_psi) return ISDF_ERR_INVALID_ARG;
    if (row_begin < 0 || row_count < 0 || row_begin + row_count > ex->n_r) return ISDF_ERR_INVALID_ARG;
    const size_t oel = ex->orb_dtype == ISDF_C128 ? 16 : 8, vel = ex->mode == ISDF_FP64 ? 16 : 8;
    if (!aligned(phi, oel) || !aligned(psi, oel) || !aligned(v, vel) || !aligned(out, 16) || !aligned(idx, 8))
        return ISDF_ERR_INVALID_ARG;
    if (row_count == 0) return ISDF_OK;
    cudaStream_t st = as_stream(stream);
    const int nm = ex->n_mu, ot = ex->orb_dtype == ISDF_C128 ? ZG_C128 : ZG_C64;
    if (ex->orb_dtype == ISDF_C128) {
        gather_rows<double2><<<grid_for((int64_t)nm * ex->n_phi), 256, 0, st>>>(
            static_cast<const double2 *>(phi), ld_phi, ex->n_phi, ex->n_r, idx, nm, ex->phi_mu, ex->flags + 1);
        gather_rows<double2><<<grid_for((int64_t)nm * ex->n_psi), 256, 0, st>>>(
            static_cast<const double2 *>(psi), ld_psi, ex->n_psi, ex->n_r, idx, nm, ex->psi_mu, ex->flags + 1);
    } else {
        gather_rows<float2><<<grid_for((int64_t)nm * ex->n_phi), 256, 0, st>>>(
            static_cast<const float2 *>(phi), ld_phi, ex->n_phi, ex->n_r, idx, nm, ex->phi_mu, ex->flags + 1);
        gather_rows<float2><<<grid_for((int64_t)nm * ex->n_psi), 256, 0, st>>>(
            static_cast<const float2 *>(psi), ld_psi, ex->n_psi, ex->n_r, idx, nm, ex->psi_mu, ex->flags + 1);
    }
    isdf_note_launch();
    isdf_note_launch();
    ISDF_LAUNCH_CHECK();
    if (ex->mixed)
        return mixed_exchange_apply(ex->mixed, phi, ld_phi, ex->orb_dtype, ex->phi_mu, ex->psi_mu,
                                    static_cast<const float2 *>(v), ld_v, row_begin, row_count,
                                    static_cast<double2 *>(out), ld_out, st);
    for (int64_t r0 = row_begin; r0 < row_begin + row_count; r0 += ex->max_rows) {
        const int rows = (int)((row_begin + row_count - r0) < ex->max_rows ? (row_begin + row_count - r0)
                                                                            : ex->max_rows);
        // G = Phi_b Phi_mu^H
        const void *pb = static_cast<const char *>(phi) + r0 * ld_phi * oel;
        ZGemm g1 = product(rows, nm, ex->n_phi, opnd(pb, ld_phi, 1, 0, ot), opnd(ex->phi_mu, 1, ex->n_phi, 1, ZG_C128),
                           ex->blkG, nm, 1.0);
        ISDF_TRY(oz_zgemm(g1, ex->oz, ex->flags, st));
        // G <- V_b o G
        if (ex->mode == ISDF_FP64)
            hadamard_v<double2><<<grid_for((int64_t)rows * nm), 256, 0, st>>>(
                ex->blkG, static_cast<const double2 *>(v) + r0 * ld_v, ld_v, rows, nm);
        else
            hadamard_v<float2><<<grid_for((int64_t)rows * nm), 256, 0, st>>>(
                ex->blkG, static_cast<const float2 *>(v) + r0 * ld_v, ld_v, rows, nm);
        isdf_note_launch();
        ISDF_LAUNCH_CHECK();
        // out_b = -G Psi_mu
        double2 *ob = static_cast<double2 *>(out) + (r0 - row_begin) * ld_out;
        ZGemm g2 = product(rows, ex->n_psi, nm, opnd(ex->blkG, nm, 1, 0, ZG_C128),
                           opnd(ex->psi_mu, ex->n_psi, 1, 0, ZG_C128), ob, ld_out, -1.0);
        ISDF_TRY(oz_zgemm(g2, ex->oz, ex->flags, st));
    }
    return ISDF_OK;
}

extern "C" isdf_status isdf_exchange_status(isdf_exchange *ex)
{
    if (!ex) return ISDF_ERR_INVALID_ARG;
    int h[2] = {0, 0};
    ISDF_CUDA_TRY(cudaMemcpy(h, ex->flags, sizeof(h), cudaMemcpyDeviceToHost));
    if (h[0]) return h[0] == 2 ? ISDF_ERR_NONFINITE : ISDF_ERR_TIMEOUT;
    if (h[1]) return ISDF_ERR_INVALID_ARG;
    if (ex->mixed) return (isdf_status)mixed_exchange_error(ex->mixed);
    return ISDF_OK;
}

extern "C" void isdf_exchange_destroy(isdf_exchange *ex)
{
    if (!ex) return;
    cudaDeviceSynchronize();
    release(ex);
}
