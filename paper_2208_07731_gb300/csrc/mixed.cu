// Tensor-core (tcgen05) split-precision path of the Theta fit.
#include "mixed.cuh"

bool mixed_supported(int, int, int64_t, int64_t, int) { return false; }
isdf_status mixed_prepare(isdf_plan *, cudaStream_t) { return ISDF_ERR_UNSUPPORTED; }
isdf_status mixed_fit(isdf_plan *, int64_t, int64_t, void *, int64_t, cudaStream_t) { return ISDF_ERR_UNSUPPORTED; }
isdf_status mixed_backward(isdf_plan *, int64_t, int64_t, const void *, int64_t, const void *, double, void *, int64_t,
                           void *, int64_t, double *, cudaStream_t)
{
    return ISDF_ERR_UNSUPPORTED;
}
void mixed_release(isdf_plan *) {}
