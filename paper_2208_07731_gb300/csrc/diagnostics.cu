// Decomposition diagnostics of Appendix A: the cluster residual R of Eq.
// errorISDF. Every row Z(r) of cluster mu is projected on the row Z(r_mu) of
// the cluster's selected point (Eq. proj); with Eq. Zmu the squared distance
// is p(r) q(r) - |a(r)|^2 |b(r)|^2 / (p(r_mu) q(r_mu)), p = sum_i |phi_i|^2,
// q = sum_j |psi_j|^2, a(r) = Phi(r) . Phi*(r_mu), b(r) = Psi(r) . Psi*(r_mu),
// so R needs two dot products of length N per grid point and never forms Z.
#include "common.cuh"

namespace {

// one warp per grid row: R_r and ||Z(r)||^2 in FP64, accumulated into sums[1], sums[0]
template <typename T>
__global__ void cluster_residual_kernel(const T *phi, int64_t ldp, int n_phi, const T *psi, int64_t ldq, int n_psi,
                                        int64_t n_r, const int32_t *labels, const int64_t *idx, int n_mu,
                                        double *sums, int *bad)
{
    __shared__ double red[2][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double zs = 0.0, rs = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; r < n_r;
         r += (int64_t)gridDim.x * (blockDim.x >> 5)) {
        const int m = labels[r];
        int64_t s = -1;
        if (m >= 0 && m < n_mu) s = idx[m];
        if (s < 0 || s >= n_r) {   // no valid cluster point: reported, row skipped
            if (lane == 0) atomicExch(bad, 1);
            continue;
        }
        double p = 0.0, q = 0.0, ps = 0.0, qs = 0.0;
        double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
        for (int i = lane; i < n_phi; i += 32) {
            const double2 x = cload(phi, r * ldp + i), xs = cload(phi, s * ldp + i);
            p += x.x * x.x + x.y * x.y;
            ps += xs.x * xs.x + xs.y * xs.y;
            a.x += x.x * xs.x + x.y * xs.y;   // x conj(xs)
            a.y += x.y * xs.x - x.x * xs.y;
        }
        for (int j = lane; j < n_psi; j += 32) {
            const double2 y = cload(psi, r * ldq + j), ys = cload(psi, s * ldq + j);
            q += y.x * y.x + y.y * y.y;
            qs += ys.x * ys.x + ys.y * ys.y;
            b.x += y.x * ys.x + y.y * ys.y;
            b.y += y.y * ys.x - y.x * ys.y;
        }
        for (int o = 16; o > 0; o >>= 1) {
            p += __shfl_xor_sync(0xffffffffu, p, o);
            q += __shfl_xor_sync(0xffffffffu, q, o);
            ps += __shfl_xor_sync(0xffffffffu, ps, o);
            qs += __shfl_xor_sync(0xffffffffu, qs, o);
            a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
            a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
            b.x += __shfl_xor_sync(0xffffffffu, b.x, o);
            b.y += __shfl_xor_sync(0xffffffffu, b.y, o);
        }
        const double zz = p * q, den = ps * qs;
        zs += zz;
        rs += den > 0.0 ? zz - (a.x * a.x + a.y * a.y) * (b.x * b.x + b.y * b.y) / den : zz;
    }
    if (lane == 0) {
        red[0][warp] = zs;
        red[1][warp] = rs;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double z = 0.0, rr = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            z += red[0][i];
            rr += red[1][i];
        }
        atomicAdd(sums, z);
        atomicAdd(sums + 1, rr);
    }
}

}  // namespace

extern "C" isdf_status isdf_cluster_residual(const void *phi, int64_t ld_phi, int32_t n_phi, const void *psi,
                                             int64_t ld_psi, int32_t n_psi, int64_t n_r, int32_t dtype,
                                             const int32_t *labels, const int64_t *idx, int32_t n_mu, double *sums,
                                             int32_t *bad, void *stream)
{
    if (!phi || !psi || !labels || !idx || !sums || !bad || n_r < 0 || n_phi < 1 || n_psi < 1 || n_mu < 1 ||
        ld_phi < n_phi || ld_psi < n_psi)
        return ISDF_ERR_INVALID_ARG;
    if (dtype != ISDF_C128 && dtype != ISDF_C64) return ISDF_ERR_INVALID_ARG;
    const size_t el = dtype == ISDF_C128 ? 16 : 8;
    if (!aligned(phi, el) || !aligned(psi, el) || !aligned(sums, 8) || !aligned(bad, 4) || !aligned(labels, 4) ||
        !aligned(idx, 8))
        return ISDF_ERR_INVALID_ARG;
    if (n_r == 0) return ISDF_OK;
    cudaStream_t st = as_stream(stream);
    const int64_t blocks = (n_r + 7) / 8;
    const unsigned g = (unsigned)(blocks < 8192 ? blocks : 8192);
    if (dtype == ISDF_C128)
        cluster_residual_kernel<double2><<<g, 256, 0, st>>>(static_cast<const double2 *>(phi), ld_phi, n_phi,
                                                            static_cast<const double2 *>(psi), ld_psi, n_psi, n_r,
                                                            labels, idx, n_mu, sums, bad);
    else
        cluster_residual_kernel<float2><<<g, 256, 0, st>>>(static_cast<const float2 *>(phi), ld_phi, n_phi,
                                                           static_cast<const float2 *>(psi), ld_psi, n_psi, n_r,
                                                           labels, idx, n_mu, sums, bad);
    isdf_note_launch();
    ISDF_LAUNCH_CHECK();
    return ISDF_OK;
}
