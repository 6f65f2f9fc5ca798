/*
 * isdf.h - C ABI of the GB300 (sm_103a) complex-valued K-means ISDF library.
 *
 * The library computes the interpolative separable density fitting (ISDF)
 * decomposition of the transposed Khatri-Rao product
 *     Z(r)_{ij} = phi_i(r) conj(psi_j(r)),   Z ~= Theta C,        (Sec. 2.1, Eqs. decomposition, decomMatrix)
 * in three steps:
 *   1. the K-means weight w(r) from the orbitals            (Sec. 2.2, Eqs. weight function, weight function 2)
 *   2. weighted Lloyd K-means on the real-space grid, which  (Sec. 2.2, Eq. opt (second form), Eq. r_k, Algorithm 1)
 *      selects N_mu interpolation points idx
 *   3. the interpolation vectors Theta = Y M^-1 with        (Sec. 2.1, Eq. theta, Eqs. phipsi, muRownuCol,
 *      Y = Z C^H = (Phi Phi_mu^H) o conj(Psi Psi_mu^H) and    muRownuColden; Sec. 2.4 for M as rows of Z C^H)
 *      M = C C^H = (Phi_mu Phi_mu^H) o conj(Psi_mu Psi_mu^H)
 * plus the adjoint of step 3 at fixed idx.
 *
 * Conventions shared by every entry point:
 *  - Orbitals Phi (N_r x N_phi) and Psi (N_r x N_psi) are row-major
 *    interleaved complex (re, im) with a leading dimension ld >= N counted in
 *    complex elements; row r of Phi starts at phi + r*ld.
 *  - The real-space grid is nx*ny*nz points, linear index
 *    r = (ix*ny + iy)*nz + iz, coordinates x_r = (ix*Lx/nx, iy*Ly/ny, iz*Lz/nz).
 *  - Every pointer argument is a DEVICE pointer owned by the caller unless
 *    its comment says "host". The library never frees caller memory.
 *  - Every call is asynchronous and stream-ordered on `stream` (a
 *    cudaStream_t; NULL is the legacy default stream). Results are valid once
 *    the stream has reached them.
 *  - Every call returns an isdf_status; arguments are validated on the host
 *    before anything is launched, so an argument error launches nothing.
 *    Failures found on the device (a non-positive Cholesky pivot, a
 *    non-finite input) are recorded in a device status word and read with
 *    isdf_plan_status (which synchronises the stream).
 */
#ifndef ISDF_H
#define ISDF_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define ISDF_API __attribute__((visibility("default")))
#else
#define ISDF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ISDF_OK = 0,
    ISDF_ERR_INVALID_ARG = 1,   /* bad size, pointer, enum or alignment; nothing was launched */
    ISDF_ERR_CUDA = 2,          /* a CUDA runtime call failed (launch, allocation, copy) */
    ISDF_ERR_NOT_HPD = 3,       /* M = C C^H is not Hermitian positive definite; detail = failing pivot */
    ISDF_ERR_EMPTY_CLUSTER = 4, /* K-means left a cluster without weight; its idx is -1 */
    ISDF_ERR_NONFINITE = 5,     /* a NaN or infinity was found on the device */
    ISDF_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up */
    ISDF_ERR_WORKSPACE = 7,     /* workspace missing or smaller than the queried size */
    ISDF_ERR_UNSUPPORTED = 8    /* valid request outside this build's limits (e.g. sizes) */
} isdf_status;

typedef enum { ISDF_C128 = 0, ISDF_C64 = 1 } isdf_dtype;   /* interleaved complex double / float */
typedef enum { ISDF_W_SSM = 0, ISDF_W_PSM = 1 } isdf_wkind;
#define ISDF_W_ACCUMULATE 0x100   /* kind flag: w(r) += the pair's weight (one FP64 rounding), for a weight
                                     shared by several orbital pairs, e.g. k-points or spin channels */

/* Precision of the Theta fit.
 *  ISDF_FP64:  every step in FP64; Theta is complex128.
 *  ISDF_MIXED: the two Gram GEMMs (with the Hadamard conjugate product fused)
 *              and the application of M^-1 run on the tcgen05 tensor cores as
 *              three FP16 products of a power-of-two-scaled hi+lo split with
 *              FP32 accumulation; M, its Cholesky factor and M^-1 stay FP64.
 *              Theta is complex64.
 * In both modes the large FP64 products of the plan update (M, the upper
 * levels of the triangular inverse, M^-1 = L^-H L^-1) run on the tensor cores
 * as exact integer-sliced products accumulated in FP64 (the Ozaki scheme),
 * whose error is that of an FP64 GEMM; OR-ing ISDF_PLAN_FP64_SIMT into the
 * mode keeps them on the FP64 pipe. */
typedef enum { ISDF_FP64 = 0, ISDF_MIXED = 1 } isdf_mode;
#define ISDF_PLAN_FP64_SIMT 0x100   /* mode flag: plan-update products on the FP64 pipe only */

/* isdf_kmeans flags */
#define ISDF_KMEANS_EARLY_STOP 1   /* stop once the labels repeat (identical result, fewer passes); detected as
                                      an update that leaves every centroid bit-identical, one pass later */

/* ---------------------------------------------------------------------------
 * Step 1: weight function (Sec. 2.2).
 *   kind ISDF_W_SSM (Eq. weight function 2): w(r) = sum_i |phi_i(r)|^alpha + sum_j |psi_j(r)|^alpha
 *       alpha = 2 is SSM (the paper's choice); 1, 3, 4 are SM, SCM, SQM.
 *   kind ISDF_W_PSM (Eq. weight function):   w(r) = (sum_i |phi_i(r)|^2)(sum_j |psi_j(r)|^2)
 *       (alpha is ignored).
 * Each sum is the exact sum of its terms, rounded once to FP64 (so it does not
 * depend on summation order): for alpha = 2 the terms are the exact squares of
 * the real components x = Re z, Im z, truncated 2^-110 below 2^(2E) with E the
 * largest floor(log2|x|) of the sum's components (the result is the correctly
 * rounded sum unless it lies within ~2^-96 of a rounding boundary); for
 * alpha != 2 the terms are |z|^alpha formed in FP64 (m = re*re + im*im, each
 * operation rounded; sqrt and products for alpha = 1, 3, 4, pow otherwise),
 * truncated 2^-110 below the largest term. PSM rounds each of its two sums
 * and multiplies once. Results in FP64's subnormal range are rounded twice.
 * phi, psi: dtype (ISDF_C128 or ISDF_C64) arrays of n_r rows; ld >= n.
 * w: n_r doubles (output; with ISDF_W_ACCUMULATE OR-ed into kind, w(r) is
 * replaced by fl(w(r) + the pair's weight), so B calls in order b = 0..B-1
 * after one plain call give the shared weight sum_b w_b(r) summed left to
 * right). Requires n_r >= 0, n_phi, n_psi >= 1, alpha > 0, 16-byte aligned
 * phi, psi and 8-byte aligned w.
 * ------------------------------------------------------------------------- */
ISDF_API isdf_status isdf_weights(const void *phi, int64_t ld_phi, int32_t n_phi,
                         const void *psi, int64_t ld_psi, int32_t n_psi,
                         int64_t n_r, int32_t dtype, int32_t kind, double alpha,
                         double *w, void *stream);

/* ---------------------------------------------------------------------------
 * Step 2: weighted Lloyd K-means on the grid (Sec. 2.2, Eq. opt second form,
 * Eq. r_k, Algorithm 1).
 *   c_0 = x[init_idx]; for t < max_iter: a_t(r) = argmin_mu |x_r - c_mu|^2
 *   (FP64 distance ((dx*dx + dy*dy) + dz*dz), ties to the lowest mu), then
 *   c_{t+1,mu} = sum w x / sum w over a_t = mu. The sums are exact: each FP64
 *   product w*x enters as the 128-bit integer floor(w*x*2^s) with
 *   s = 126 - (bits(N_r) + e(max w) + e(max(Lx,Ly,Lz,1))) (e() the frexp
 *   exponent), and each integer sum is rounded to FP64 before one IEEE
 *   division; an empty (zero-weight) cluster keeps its centroid. Finally
 *   idx_mu = the member of cluster mu nearest to c_mu (ties to the lowest r)
 *   under the last assignment, or -1 for an empty cluster.
 *   The result is bit-identical to a plain FP64 brute-force evaluation of
 *   these formulas; the device prunes centroids per tile with exact distance
 *   bounds and screens in FP32 with a rigorous error bound before deciding in
 *   FP64.
 * w:          n_r = nx*ny*nz weights (>= 0, finite).
 * cell:       HOST array of 3 doubles (Lx, Ly, Lz), each > 0.
 * init_idx:   n_mu grid indices (int64, in [0, n_r)).
 * max_iter:   number of Lloyd updates T >= 0.
 * flags:      0 or ISDF_KMEANS_EARLY_STOP.
 * idx:        out, n_mu int64.
 * centroids:  out, n_mu x 3 doubles (final centroids), or NULL.
 * objective:  out, max_iter + 1 doubles J_t = sum_r w(r)|x_r - c_{a_t(r)}|^2, or NULL.
 * labels:     out, n_r int32 final assignment, or NULL.
 * stats:      out, 4 int64: {Lloyd updates done, near ties, empty clusters,
 *             points decided in FP64 after the FP32 screen}, or NULL. A near
 *             tie is a point whose two smallest distances d1 <= d2 satisfy
 *             d2 - d1 <= 1e-12 max(d1, hmin^2); they are counted over every
 *             assignment pass and are resolved exactly by the lowest-mu rule.
 * ws, ws_bytes: device workspace of at least isdf_kmeans_workspace() bytes,
 *             256-byte aligned. Its contents need no initialisation.
 * Limits: 1 <= n_mu <= min(n_r, 8192), n_r < 2^31. Weights with
 * n_r * max(w) * max(L, 1) >= 2^126 are rejected on the device
 * (ISDF_ERR_NONFINITE recorded in stats[2] = -1); an init_idx entry outside
 * [0, n_r) gives stats[2] = -2. isdf_kmeans_status turns stats into a status.
 * ------------------------------------------------------------------------- */
ISDF_API isdf_status isdf_kmeans_workspace(int32_t nx, int32_t ny, int32_t nz, int32_t n_mu, size_t *ws_bytes);

/* The outcome of an isdf_kmeans call as a status code. stats is that call's
 * device stats array (4 int64); the call synchronises `stream` (the stream the
 * K-means ran on) and reads stats[2]:
 *   0  -> ISDF_OK;
 *   >0 -> ISDF_ERR_EMPTY_CLUSTER (that many clusters had no member after the
 *         last assignment: their idx entries are -1, Algorithm 1 leaves the
 *         case open);
 *   -1 -> ISDF_ERR_NONFINITE (a weight negative, infinite or NaN, or too large
 *         for the 128-bit fixed-point sums: every idx is -1);
 *   -2 -> ISDF_ERR_INVALID_ARG (an init_idx entry outside [0, n_r): every idx
 *         is -1). */
ISDF_API isdf_status isdf_kmeans_status(const int64_t *stats, void *stream);
ISDF_API isdf_status isdf_kmeans(const double *w, int32_t nx, int32_t ny, int32_t nz, const double *cell,
                        int32_t n_mu, const int64_t *init_idx, int32_t max_iter, int32_t flags,
                        int64_t *idx, double *centroids, double *objective, int32_t *labels,
                        int64_t *stats, void *ws, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------------------
 * K-means without allocation (no counterpart in the paper: an interface for
 * callers that cannot allocate device memory).
 * Callers inside another framework whose allocator already owns the device
 * memory, or loops that must not allocate mid-step, cannot call cudaMalloc for
 * the workspace isdf_kmeans needs. isdf_kmeans_noalloc takes the same
 * arguments as isdf_kmeans without ws/ws_bytes and computes the same result,
 * with its workspace in a fixed array of ISDF_KMEANS_NOALLOC_SCRATCH_BYTES
 * (32 MiB) of device memory that the library holds on every GPU that loads it
 * until the process exits. It calls no cudaMalloc, cudaFree or other
 * allocating routine. Inputs and outputs are still the caller's device buffers.
 *  - Problems whose isdf_kmeans_workspace() exceeds the array size return
 *    ISDF_ERR_UNSUPPORTED before anything is launched (32 MiB covers a
 *    128^3 grid with 4096 points).
 *  - The first call in a CUDA context looks up the array's device address in
 *    that context (cudaGetSymbolAddress, with the context current) and keeps
 *    it; a later call under a different current context on the same device
 *    (after cudaDeviceReset, or a driver-API caller's own context) looks it up
 *    again. Make the first call of each context before any stream capture on
 *    the device. The lookup is not repeated for a context that is destroyed
 *    and re-created at the same handle value. Arguments are checked like
 *    isdf_kmeans's (ISDF_ERR_INVALID_ARG) before the size check.
 *  - Every call, on every stream, uses the same array, and the array keeps the
 *    last call's contents (each call re-initialises what it reads). Calls that
 *    overlap on the GPU (different streams, or different host threads without
 *    ordering) race on the array and give wrong results: order them.
 * ------------------------------------------------------------------------- */
#define ISDF_KMEANS_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
ISDF_API isdf_status isdf_kmeans_noalloc(const double *w, int32_t nx, int32_t ny, int32_t nz, const double *cell,
                                         int32_t n_mu, const int64_t *init_idx, int32_t max_iter, int32_t flags,
                                         int64_t *idx, double *centroids, double *objective, int32_t *labels,
                                         int64_t *stats, void *stream);

/* ---------------------------------------------------------------------------
 * Step 3: the interpolation-vector fit (Sec. 2.1, Eq. theta with the
 * Hermitian adjoint for complex orbitals; Eqs. muRownuCol, muRownuColden).
 *
 * isdf_plan_create gathers Phi_mu = Phi[idx], Psi_mu = Psi[idx] (Eq. Cmu),
 * forms M = (Phi_mu Phi_mu^H) o conj(Psi_mu Psi_mu^H) in FP64, factors
 * M = L L^H (blocked Cholesky, FP64) and forms M^-1 = L^-H L^-1 in FP64.
 * The plan keeps phi/psi pointers: the orbitals must stay alive and unchanged
 * while the plan is used, with one exception: in ISDF_MIXED mode
 * isdf_fit_theta and isdf_fit_theta_host read only the FP16 operand copies
 * that isdf_plan_create / isdf_plan_update made, so once the create or update
 * has completed on its stream the orbitals may be overwritten (for instance
 * with the next decomposition's orbitals) until the next isdf_plan_update or
 * adjoint call, which read them again. idx must hold n_mu distinct indices in [0, n_r)
 * (duplicates make M singular: ISDF_ERR_NOT_HPD). max_rows bounds the rows
 * of one internal block (the plan holds two blocks of max_rows x n_mu
 * complex128 scratch); larger requests are processed in several blocks.
 * The plan allocates its own device memory (cudaMalloc) and frees it in
 * isdf_plan_destroy.
 * mode: ISDF_FP64 or ISDF_MIXED, optionally OR ISDF_PLAN_FP64_SIMT.
 * Limits: 1 <= n_mu <= 8192; n_phi, n_psi <= 4096; in ISDF_MIXED mode
 * n_mu % 64 == 0 and n_phi, n_psi % 32 == 0.
 * ------------------------------------------------------------------------- */
typedef struct isdf_plan isdf_plan;

ISDF_API isdf_status isdf_plan_create(isdf_plan **plan, const void *phi, int64_t ld_phi, const void *psi, int64_t ld_psi,
                             int64_t n_r, int32_t n_phi, int32_t n_psi, int32_t dtype,
                             const int64_t *idx, int32_t n_mu, int32_t mode, int64_t max_rows, void *stream);

/* Theta rows [row_begin, row_begin + row_count): Theta_b = Y_b M^-1 with
 * Y_b = (Phi_b Phi_mu^H) o conj(Psi_b Psi_mu^H).
 * theta: row_count x n_mu, row-major with leading dimension ld_theta >= n_mu,
 * complex128 in ISDF_FP64 mode and complex64 in ISDF_MIXED mode. */
ISDF_API isdf_status isdf_fit_theta(isdf_plan *plan, int64_t row_begin, int64_t row_count,
                           void *theta, int64_t ld_theta, void *stream);

/* The same Theta rows written to host memory. The rows are fitted block by
 * block (max_rows rows each) into one of three device staging blocks owned by
 * the plan (allocated on the first call, freed by isdf_plan_destroy); each
 * block is copied to theta_host, in two halves on two copy streams of the
 * plan, while the next block is fitted. theta_host: row_count x n_mu, row-major with leading
 * dimension ld_theta_host >= n_mu, complex128 (ISDF_FP64) / complex64
 * (ISDF_MIXED), and the whole range must be page-locked host memory
 * (cudaHostAlloc, cudaMallocHost or cudaHostRegister); pageable or device
 * memory is refused with ISDF_ERR_INVALID_ARG before any work is enqueued.
 * Ordered on stream: work enqueued on stream after the call runs after the
 * last copy has landed (synchronise stream before reading theta_host), also
 * when the call returns an error after enqueueing part of the work. The
 * caller must not write theta_host until then. */
ISDF_API isdf_status isdf_fit_theta_host(isdf_plan *plan, int64_t row_begin, int64_t row_count,
                                         void *theta_host, int64_t ld_theta_host, void *stream);

/* Adjoint of Theta(Phi, Psi) at fixed idx, for one block of rows.
 * Given dL/dTheta = G (convention G = dL/dRe Theta + i dL/dIm Theta) on the
 * rows of the block, or, when grad_theta is NULL, the exchange-like surrogate
 *   L = dV sum_r sum_{mu,nu} Re[conj(Theta_{r,mu}) K_{mu,nu} Theta_{r,nu}]
 * whose G = 2 dV Theta conj(K) is formed in the kernel (K: n_mu x n_mu
 * complex128 Hermitian, row-major), this call
 *   - recomputes Theta_b (never stored),
 *   - adds Abar_b Phi_mu into grad_phi rows and Bbar_b Psi_mu into grad_psi
 *     rows of the block, with Ybar = G M^-1, Abar = Ybar o B, Bbar = conj(Ybar) o A,
 *   - accumulates Mbar -= Theta_b^H Ybar, Phibar_mu += Abar^H Phi_b and
 *     Psibar_mu += Bbar^H Psi_b inside the plan,
 *   - adds the block's surrogate loss to *loss (device double) if loss != NULL.
 * grad_theta: row_count x n_mu (ld_grad), complex128 (FP64) / complex64 (MIXED).
 * grad_phi, grad_psi: n_r x n complex128 (ld_gphi, ld_gpsi), accumulated (+=).
 * Call isdf_fit_theta_backward_finalize once after all blocks: it adds the
 * M-dependent terms (Mbar o B_mu and conj(Mbar) o A_mu, through
 * (Abar_mu + Abar_mu^H) Phi_mu) and scatter-adds Phibar_mu, Psibar_mu into the
 * idx rows of grad_phi, grad_psi, then clears the plan's accumulators. */
ISDF_API isdf_status isdf_fit_theta_backward(isdf_plan *plan, int64_t row_begin, int64_t row_count,
                                    const void *grad_theta, int64_t ld_grad, const void *K, double dV,
                                    void *grad_phi, int64_t ld_gphi, void *grad_psi, int64_t ld_gpsi,
                                    double *loss, void *stream);
ISDF_API isdf_status isdf_fit_theta_backward_finalize(isdf_plan *plan, void *grad_phi, int64_t ld_gphi,
                                             void *grad_psi, int64_t ld_gpsi, void *stream);

/* Recomputes the plan for new interpolation points idx (n_mu distinct
 * indices) and the current contents of the orbitals it was created with:
 * gather, M, Cholesky factor and M^-1 (and, in ISDF_MIXED mode, the split
 * tensor-core operands), reusing the plan's memory. This is the per-step call
 * of an MD loop where the orbitals and the K-means points change but the
 * sizes do not. */
ISDF_API isdf_status isdf_plan_update(isdf_plan *plan, const int64_t *idx, void *stream);

/* ---------------------------------------------------------------------------
 * Batched decompositions: B orbital pairs on one grid (k-points or spin
 * channels of complex Bloch orbitals, Sec. 2.1) sharing one set of
 * interpolation points, e.g. from one isdf_kmeans on the shared weight
 * (isdf_weights with ISDF_W_ACCUMULATE). Each pair gets its own plan (as
 * isdf_plan_create, all with the same sizes, dtype, mode and max_rows);
 * isdf_batch_update and isdf_batch_fit_theta run the pairs' plan updates /
 * fits on one internal stream per pair, ordered after the work already on
 * `stream` and before anything later on it (event fork and join, so the
 * batch can be captured into a CUDA graph from `stream`). The pairs' results
 * are bit-identical to B separate plans run one after another.
 * phi, psi, ld_phi, ld_psi, theta: HOST arrays of count entries (device
 * pointers / leading dimensions); idx: device int64[n_mu]. Each plan keeps
 * its phi/psi pointers (they must stay valid and unchanged).
 * isdf_batch_plan returns pair i's plan (owned by the batch) for the other
 * plan entry points; isdf_batch_status reports the first failing pair's
 * isdf_plan_status (which = its index, or -1) and synchronises.
 * ------------------------------------------------------------------------- */
typedef struct isdf_batch isdf_batch;

ISDF_API isdf_status isdf_batch_create(isdf_batch **batch, int32_t count, const void *const *phi,
                                       const int64_t *ld_phi, const void *const *psi, const int64_t *ld_psi,
                                       int64_t n_r, int32_t n_phi, int32_t n_psi, int32_t dtype, const int64_t *idx,
                                       int32_t n_mu, int32_t mode, int64_t max_rows, void *stream);
ISDF_API isdf_status isdf_batch_update(isdf_batch *batch, const int64_t *idx, void *stream);
ISDF_API isdf_status isdf_batch_fit_theta(isdf_batch *batch, int64_t row_begin, int64_t row_count,
                                          void *const *theta, int64_t ld_theta, void *stream);
ISDF_API isdf_plan *isdf_batch_plan(isdf_batch *batch, int32_t i);
ISDF_API isdf_status isdf_batch_status(isdf_batch *batch, int32_t *which, int32_t *detail);
ISDF_API void isdf_batch_destroy(isdf_batch *batch);

/* ---------------------------------------------------------------------------
 * Decomposition diagnostics (Appendix A).
 *
 * isdf_fit_error: the least-squares residual of the ISDF fit over grid rows
 * [row_begin, row_begin + row_count), with Z(r) = [phi_i(r) conj(psi_j(r))]
 * and C = Z[idx]:  ||Z - Theta C||_F^2 = ||Z||_F^2 - Re tr(Theta^H Y), since
 * Theta C C^H = Z C^H = Y at the fitted Theta.  ||Z(r)||^2 =
 * (sum_i |phi_i(r)|^2)(sum_j |psi_j(r)|^2) (the factorisation of Eq. Zmu at
 * any r), so Z is never formed.
 * sums: device array of 2 doubles, ACCUMULATED into (the caller zeroes it):
 * sums[0] += ||Z_b||_F^2, sums[1] += Re tr(Theta_b^H Y_b).  The residual is
 * sums[0] - sums[1]; the relative error sqrt(1 - sums[1] / sums[0]).
 * ISDF_FP64 plans only (ISDF_ERR_UNSUPPORTED otherwise): in ISDF_MIXED mode
 * the difference would drown in the mixed products' rounding.  Uses the
 * plan's block scratch; ordered on stream like isdf_fit_theta.
 *
 * isdf_cluster_residual: R of Eq. errorISDF, the residual of projecting every
 * row Z(r) of cluster mu = labels[r] on the single row Z(idx[mu]) (Eq. proj).
 * With a = Phi(r) . conj(Phi(r_mu)), b = Psi(r) . conj(Psi(r_mu)),
 * p = |Phi(r)|^2, q = |Psi(r)|^2 (Eq. Zmu and the first lines of Eq. error2),
 * the row's term is p q - |a|^2 |b|^2 / (p(r_mu) q(r_mu)), or p q where Z(r_mu)
 * is zero.  phi, psi: device, row-major n_r x n_phi / n_r x n_psi with leading
 * dimensions ld_phi >= n_phi, ld_psi >= n_psi, complex128 (ISDF_C128) or
 * complex64 (ISDF_C64, widened to FP64).  labels: device int32[n_r] (the
 * labels isdf_kmeans writes), idx: device int64[n_mu].  sums: device double[2],
 * ACCUMULATED: sums[0] += ||Z||_F^2, sums[1] += R.  bad: device int32, set to 1
 * if a label lies outside [0, n_mu) or an index outside [0, n_r); those rows
 * are skipped.  Returns ISDF_ERR_INVALID_ARG for null or misaligned pointers
 * and bad sizes.
 * ------------------------------------------------------------------------- */
ISDF_API isdf_status isdf_fit_error(isdf_plan *plan, int64_t row_begin, int64_t row_count, double *sums,
                                    void *stream);

/* ---------------------------------------------------------------------------
 * ISDF exchange application (Sec. 2.3, Eq. v2 and Eq. V_mu).
 *
 * Step A, isdf_exchange_potential: V_mu(r) = int zeta_mu(r') v(r - r') dr' for
 * every column mu of Theta (the interpolation vectors), on the periodic grid
 * of the K-means (r = (ix*ny + iy)*nz + iz, orthorhombic cell of edges
 * cell[0..2]).  A column is read as the band-limited periodic function
 * sum_G c(G) exp(i G.r), c = (1/N_r) sum_r f(r) exp(-i G.r), and
 *     V = sum_G K(G + q) c(G) exp(i G.r),  G = 2 pi m / L,
 * m the signed frequency of the index (n/2 of an even axis reads as -n/2), with
 *     ISDF_KERNEL_COULOMB: K = 4 pi / |G+q|^2, zero where G + q = 0
 *                          (the interaction 1/|r - r'| of Eq. v);
 *     ISDF_KERNEL_ERFC:    K = 4 pi (1 - exp(-|G+q|^2 / (4 omega^2))) / |G+q|^2,
 *                          pi / omega^2 at zero (erfc(omega |r-r'|) / |r-r'|,
 *                          the short-range exchange of screened hybrids).
 * q (3 doubles, or NULL for zero) shifts the reciprocal vectors for pair
 * products with a Bloch phase exp(i q.r); the data are their periodic parts.
 * theta, v: n_r x n_mu row-major, leading dimensions >= n_mu, complex128 in
 * ISDF_FP64 mode (FP64 FFT) and complex64 in ISDF_MIXED mode (FP32 FFT).
 * v may equal theta (in place); otherwise theta is only read.
 * For the exchange, Theta must interpolate the pair products phi_i*(r) psi_j(r)
 * of Eq. v2: with isdf_plan_create that is the pair passed as (Psi, Phi).
 *
 * Step B, isdf_exchange_apply: rows [row_begin, row_begin + row_count) of
 *     out(r, j) = -sum_mu V_mu(r) sum_i phi_i(r) phi_i*(r_mu) psi_j(r_mu)
 *               = -[(V o (Phi Phi_mu^H)) Psi_mu](r, j),   r_mu = grid point idx[mu].
 * phi, psi: n_r x n_phi / n_r x n_psi (orb_dtype), idx: device int64[n_mu],
 * v: as written by step A, out: row_count x n_psi complex128 (device,
 * leading dimension ld_out >= n_psi, row 0 = grid row row_begin). Both
 * products run on the tcgen05 tensor cores, in blocks of max_rows rows: in
 * ISDF_MIXED mode, when n_phi, n_psi % 32 == 0 and n_mu % 64 == 0, as
 * split-FP16 x3 products with FP32 accumulation (relative error ~1e-6, the
 * Hadamard product with V fused into the first product); otherwise by exact
 * integer slicing with FP64-grade results.
 *
 * isdf_exchange_create sizes and allocates every buffer (cudaMalloc; about
 * max_rows * (n_mu * 16 + 28 * max(n_mu, n_phi) * 2) bytes for the sliced
 * products, n_r * n_phi * 8 + max_rows * n_mu * 8 for the split ones) and
 * computes the FFT twiddles; nothing is allocated later.  Axis lengths must be products of
 * 2, 3 and 5 and at most 256 (else ISDF_ERR_UNSUPPORTED); n_mu <= 8192,
 * n_phi, n_psi <= 4096.  isdf_exchange_status reports (synchronously) a bounded
 * device wait that gave up (ISDF_ERR_TIMEOUT) or an index of idx outside
 * [0, n_r) (ISDF_ERR_INVALID_ARG; those rows of Phi_mu, Psi_mu were zero),
 * or a non-finite operand bound in the split products (ISDF_ERR_NONFINITE).
 * ------------------------------------------------------------------------- */
/* ---------------------------------------------------------------------------
 * Interpolation points by QR with column pivoting (Sec. 2.1, Eq. QRCP): the
 * comparator of the K-means selection. Z^T (N_phi N_psi x N_r) is replaced by
 * the randomized sketch S^T with S = Z G, column k of G = a_k (x) conj(b_k):
 *     S(r, k) = (Phi A)(r, k) conj((Psi B)(r, k))      (FP64 products)
 * and idx receives the first n_mu pivots of S^T's column-pivoted QR, found by
 * greedy pivoted Gram-Schmidt in FP64 (at each step the grid point with the
 * largest residual norm; norms compared on their top 30 mantissa bits, ties
 * and near ties within ~1e-9 relative to the lowest grid index; residual norms
 * recomputed, not downdated), and rdiag the |R_kk| (non-increasing).
 * phi, psi: n_r x n_phi / n_r x n_psi (dtype, leading dims ld >= n);
 * A: n_phi x p, B: n_psi x p, complex128 row-major (the caller's random
 * numbers, e.g. complex Gaussian; p >= n_mu, a few more than n_mu);
 * idx: device int64[n_mu], rdiag: device double[n_mu].
 * Allocates n_r * p * 16 bytes (+ a row block when n_phi != n_psi) for the
 * sketch, frees it before returning, and synchronises the stream. Cost: one
 * pass over the sketch per point (FP64-bound). Limits: n_r < 2^22, p <= 8192.
 * Returns ISDF_ERR_NOT_HPD when every remaining column is exactly zero before
 * n_mu points are found (idx[k] = -1 from that step on); a numerically
 * rank-deficient sketch shows as tiny trailing rdiag instead.
 * ------------------------------------------------------------------------- */
ISDF_API isdf_status isdf_qrcp_points(const void *phi, int64_t ld_phi, int32_t n_phi, const void *psi,
                                      int64_t ld_psi, int32_t n_psi, int64_t n_r, int32_t dtype, const void *A,
                                      const void *B, int32_t p, int32_t n_mu, int64_t *idx, double *rdiag,
                                      void *stream);

typedef enum { ISDF_KERNEL_COULOMB = 0, ISDF_KERNEL_ERFC = 1 } isdf_kernel;
typedef struct isdf_exchange isdf_exchange;

ISDF_API isdf_status isdf_exchange_create(isdf_exchange **ex, int32_t nx, int32_t ny, int32_t nz, const double *cell,
                                          int32_t n_mu, int32_t n_phi, int32_t n_psi, int32_t orb_dtype,
                                          int32_t mode, int32_t kernel, double omega, const double *q,
                                          int64_t max_rows, void *stream);
ISDF_API isdf_status isdf_exchange_potential(isdf_exchange *ex, const void *theta, int64_t ld_theta, void *v,
                                             int64_t ld_v, void *stream);
ISDF_API isdf_status isdf_exchange_apply(isdf_exchange *ex, const void *phi, int64_t ld_phi, const void *psi,
                                         int64_t ld_psi, const int64_t *idx, const void *v, int64_t ld_v,
                                         int64_t row_begin, int64_t row_count, void *out, int64_t ld_out,
                                         void *stream);
ISDF_API isdf_status isdf_exchange_status(isdf_exchange *ex);
ISDF_API void isdf_exchange_destroy(isdf_exchange *ex);
ISDF_API isdf_status isdf_cluster_residual(const void *phi, int64_t ld_phi, int32_t n_phi, const void *psi,
                                           int64_t ld_psi, int32_t n_psi, int64_t n_r, int32_t dtype,
                                           const int32_t *labels, const int64_t *idx, int32_t n_mu, double *sums,
                                           int32_t *bad, void *stream);

/* Synchronises the plan's last stream and returns the first device-side
 * failure (ISDF_OK, ISDF_ERR_NOT_HPD with *detail = failing pivot index,
 * ISDF_ERR_NONFINITE, ISDF_ERR_TIMEOUT). detail may be NULL.
 * ISDF_ERR_NONFINITE is also what a NaN or infinity anywhere in the orbitals
 * gives: in ISDF_MIXED mode every row is scanned when the plan is created or
 * updated, in ISDF_FP64 mode every row of a block when it is fitted (the
 * tensor-core FP64 products cannot slice a non-finite entry); the affected
 * Theta rows are then not valid. With ISDF_PLAN_FP64_SIMT the FP64-pipe
 * products propagate a NaN into Theta instead. isdf_plan_update clears the
 * status. */
ISDF_API isdf_status isdf_plan_status(isdf_plan *plan, int32_t *detail);

/* Failure-path control, for tests of the bounded waits (Sec. 2.1 names no
 * such mechanism: it belongs to this implementation). Every wait of the
 * plan's tensor-core kernels (the split products of ISDF_MIXED, the
 * exact-slicing FP64 products) gives up after a budget of SM clock cycles,
 * about 0.1 s by default; the kernel then records ISDF_ERR_TIMEOUT, lets its
 * own copies and MMAs finish, frees its tensor memory and returns, and the
 * grid's remaining CTAs exit at once. For later launches of this plan:
 *   cycles > 0  replaces that budget for the pipeline waits (a wait may still
 *               succeed: one try of an mbarrier wait can itself suspend the
 *               thread for a while);
 *   cycles < 0  test hook: the MMA-issuing thread of each CTA first waits on
 *               a barrier that nothing signals, gives up after -cycles cycles
 *               and takes the timeout path, so the launch reliably reports
 *               ISDF_ERR_TIMEOUT (the other waits keep the default budget);
 *   cycles == 0 restores the default.
 * The waits that drain a kernel's own copies and MMAs before it exits always
 * keep the default budget. isdf_plan_update clears a recorded timeout.
 * Host-side setting only: nothing is launched. */
ISDF_API isdf_status isdf_plan_set_wait_budget(isdf_plan *plan, int64_t cycles);

/* Copies a plan-owned matrix into the caller's device buffer dst
 * (stream-ordered): which = 0 M, 1 L, 2 M^-1 (each n_mu x n_mu complex128,
 * row-major; L's strict upper triangle is zero), 3 Phi_mu, 4 Psi_mu
 * (n_mu x n complex128). */
ISDF_API isdf_status isdf_plan_copy_matrix(const isdf_plan *plan, int32_t which, void *dst, void *stream);

ISDF_API void isdf_plan_destroy(isdf_plan *plan);

/* Benchmark instrumentation.
 * isdf_plan_enable_timing(plan, capacity): when capacity > 0, the plan records
 * CUDA events on the launching stream around each launch of its Gram-Hadamard
 * kernel (kind 0) and its M^-1 application kernel (kind 1), and around the
 * stages of isdf_plan_create / isdf_plan_update: gather + M (2), Cholesky
 * factor (3), triangular inverse (4), M^-1 = L^-H L^-1 (5) and the tensor-core
 * operand preparation (6), for up to `capacity` records per kind; 0 switches
 * timing off. Kinds are 0..6.
 * isdf_plan_kernel_time(plan, kind, &ms, &launches, &rows): waits for those
 * events and returns the summed kernel time, the number of launches and the
 * grid rows they processed since the previous query, then resets the count.
 * isdf_kernel_launches(): number of kernels this library has launched in the
 * process so far (host-side counter). */
ISDF_API isdf_status isdf_plan_enable_timing(isdf_plan *plan, int32_t capacity);
ISDF_API isdf_status isdf_plan_kernel_time(isdf_plan *plan, int32_t kind, double *total_ms, int64_t *launches,
                                           int64_t *rows);
ISDF_API unsigned long long isdf_kernel_launches(void);

/* Human-readable name of a status code (static storage). */
ISDF_API const char *isdf_status_string(isdf_status s);

#ifdef __cplusplus
}
#endif

#endif /* ISDF_H */
