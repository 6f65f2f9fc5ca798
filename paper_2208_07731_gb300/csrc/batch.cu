// Batched decompositions: several orbital pairs on one grid (k-points or spin
// channels of complex Bloch orbitals, Sec. 2.1) that share the interpolation
// points of one K-means on their summed weight. Each pair keeps its own plan
// (its own M, Cholesky factor and M^-1); the batch issues the pairs' plan
// updates and fits on one stream per pair, forked from and joined back to the
// caller's stream with events, so the latency-bound FP64 chains and the small
// products of different pairs run side by side on the GPU's 152 SMs (and the
// whole batch captures into one CUDA graph).
#include <vector>

#include "common.cuh"

struct isdf_batch {
    int count;
    std::vector<isdf_plan *> plans;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork;
};

namespace {

void release(isdf_batch *b)
{
    for (isdf_plan *p : b->plans)
        if (p) isdf_plan_destroy(p);
    for (cudaStream_t s : b->streams)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->joins)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

// run f(i, stream_i) for every pair on its own stream, ordered after and before the caller's stream
template <typename F>
isdf_status fan_out(isdf_batch *b, cudaStream_t st, F f)
{
    ISDF_CUDA_TRY(cudaEventRecord(b->fork, st));
    isdf_status first = ISDF_OK;
    for (int i = 0; i < b->count; ++i) {
        ISDF_CUDA_TRY(cudaStreamWaitEvent(b->streams[i], b->fork, 0));
        const isdf_status s = f(i, b->streams[i]);
        if (s != ISDF_OK && first == ISDF_OK) first = s;
        ISDF_CUDA_TRY(cudaEventRecord(b->joins[i], b->streams[i]));
        ISDF_CUDA_TRY(cudaStreamWaitEvent(st, b->joins[i], 0));
    }
    return first;
}

}  // namespace

extern "C" isdf_status isdf_batch_create(isdf_batch **out, int32_t count, const void *const *phi,
                                         const int64_t *ld_phi, const void *const *psi, const int64_t *ld_psi,
                                         int64_t n_r, int32_t n_phi, int32_t n_psi, int32_t dtype,
                                         const int64_t *idx, int32_t n_mu, int32_t mode, int64_t max_rows,
                                         void *stream)
{
    if (!out || !phi || !psi || !ld_phi || !ld_psi || count < 1 || count > 1024) return ISDF_ERR_INVALID_ARG;
    *out = nullptr;
    for (int i = 0; i < count; ++i)
        if (!phi[i] || !psi[i]) return ISDF_ERR_INVALID_ARG;
    isdf_batch *b = new isdf_batch();
    b->count = count;
    b->plans.assign(count, nullptr);
    b->streams.assign(count, nullptr);
    b->joins.assign(count, nullptr);
    b->fork = nullptr;
    isdf_status s = ISDF_OK;
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) s = ISDF_ERR_CUDA;
    for (int i = 0; s == ISDF_OK && i < count; ++i) {
        if (cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->joins[i], cudaEventDisableTiming) != cudaSuccess) {
            s = ISDF_ERR_CUDA;
            break;
        }
        s = isdf_plan_create(&b->plans[i], phi[i], ld_phi[i], psi[i], ld_psi[i], n_r, n_phi, n_psi, dtype, idx, n_mu,
                             mode, max_rows, stream);
    }
    if (s != ISDF_OK) {
        cudaStreamSynchronize(as_stream(stream));
        release(b);
        return s;
    }
    *out = b;
    return ISDF_OK;
}

extern "C" isdf_status isdf_batch_update(isdf_batch *b, const int64_t *idx, void *stream)
{
    if (!b || !idx) return ISDF_ERR_INVALID_ARG;
    return fan_out(b, as_stream(stream), [&](int i, cudaStream_t s) { return isdf_plan_update(b->plans[i], idx, s); });
}

extern "C" isdf_status isdf_batch_fit_theta(isdf_batch *b, int64_t row_begin, int64_t row_count, void *const *theta,
                                            int64_t ld_theta, void *stream)
{
    if (!b || !theta) return ISDF_ERR_INVALID_ARG;
    for (int i = 0; i < b->count; ++i)
        if (!theta[i]) return ISDF_ERR_INVALID_ARG;
    return fan_out(b, as_stream(stream), [&](int i, cudaStream_t s) {
        return isdf_fit_theta(b->plans[i], row_begin, row_count, theta[i], ld_theta, s);
    });
}

extern "C" isdf_plan *isdf_batch_plan(isdf_batch *b, int32_t i)
{
    if (!b || i < 0 || i >= b->count) return nullptr;
    return b->plans[i];
}

extern "C" isdf_status isdf_batch_status(isdf_batch *b, int32_t *which, int32_t *detail)
{
    if (!b) return ISDF_ERR_INVALID_ARG;
    if (which) *which = -1;
    for (int i = 0; i < b->count; ++i) {
        int32_t d = 0;
        const isdf_status s = isdf_plan_status(b->plans[i], &d);
        if (s != ISDF_OK) {
            if (which) *which = i;
            if (detail) *detail = d;
            return s;
        }
    }
    return ISDF_OK;
}

extern "C" void isdf_batch_destroy(isdf_batch *b)
{
    if (!b) return;
    for (cudaStream_t s : b->streams)
        if (s) cudaStreamSynchronize(s);
    release(b);
}
