// K-means entry point that allocates nothing.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework whose allocator has already reserved the device memory (so a
// direct cudaMalloc fails or is forbidden by that framework), and
// molecular-dynamics or serving loops that must not allocate in the middle of
// a step. For them, isdf_kmeans_noalloc runs the same K-means as isdf_kmeans
// with its workspace in a fixed array of device memory that belongs to this
// library: every GPU that loads the library keeps the array until the process
// exits, and the library never allocates it, grows it or frees it.
//
// Host code cannot use the array's name as a device address (in host code it
// is a host-side stand-in), so the first call in each CUDA context, with that
// context current, asks the runtime for the array's device address and keeps
// it. The address belongs to the context that loaded the module: after
// cudaDeviceReset, or under another context on the same device (a driver-API
// caller's own context instead of the primary one), the array has a new
// address, so the cache is keyed on the current context and looked up again
// whenever the context differs.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"

namespace {

static __device__ __align__(256) unsigned char g_kmeans_scratch[ISDF_KMEANS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 256;
std::mutex g_lock;
struct ScratchEntry {
    CUcontext ctx;
    void *addr;
};
ScratchEntry g_entry[kMaxDevices] = {};

// cuCtxGetCurrent through the runtime's driver entry-point query (no link against libcuda)
CUresult current_context(CUcontext *ctx)
{
    static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p)
            return CUDA_ERROR_NOT_FOUND;
        fn = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
    }
    return fn(ctx);
}

// device address of g_kmeans_scratch in the current context (looked up once per context)
isdf_status scratch_address(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return ISDF_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return ISDF_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> guard(g_lock);
    CUcontext ctx = nullptr;
    if (current_context(&ctx) != CUDA_SUCCESS) return ISDF_ERR_CUDA;
    if (!ctx || !g_entry[dev].addr || g_entry[dev].ctx != ctx) {
        // with no context current yet, this runtime call makes the device's primary context
        // current, and the context is read again below
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_kmeans_scratch) != cudaSuccess || !p) return ISDF_ERR_CUDA;
        if (!ctx && (current_context(&ctx) != CUDA_SUCCESS || !ctx)) return ISDF_ERR_CUDA;
        g_entry[dev].ctx = ctx;
        g_entry[dev].addr = p;
    }
    *out = g_entry[dev].addr;
    return ISDF_OK;
}

}  // namespace

extern "C" isdf_status isdf_kmeans_noalloc(const double *w, int32_t nx, int32_t ny, int32_t nz, const double *cell,
                                           int32_t n_mu, const int64_t *init_idx, int32_t max_iter, int32_t flags,
                                           int64_t *idx, double *centroids, double *objective, int32_t *labels,
                                           int64_t *stats, void *stream)
{
    // the argument checks of isdf_kmeans first, so that an invalid call on a large grid is
    // reported as ISDF_ERR_INVALID_ARG rather than as too large for the scratch array
    if (nx < 1 || ny < 1 || nz < 1 || !cell || !w || !init_idx || !idx) return ISDF_ERR_INVALID_ARG;
    const int64_t n_r = (int64_t)nx * ny * nz;
    if (n_r >= ((int64_t)1 << 31)) return ISDF_ERR_UNSUPPORTED;
    if (n_mu < 1 || n_mu > n_r || max_iter < 0 || (flags & ~ISDF_KMEANS_EARLY_STOP)) return ISDF_ERR_INVALID_ARG;
    for (int k = 0; k < 3; ++k)
        if (!(cell[k] > 0.0) || cell[k] > 1e300) return ISDF_ERR_INVALID_ARG;
    size_t need = 0;
    isdf_status s = isdf_kmeans_workspace(nx, ny, nz, n_mu, &need);
    if (s != ISDF_OK) return s;
    if (need > (size_t)ISDF_KMEANS_NOALLOC_SCRATCH_BYTES) return ISDF_ERR_UNSUPPORTED;
    void *scratch = nullptr;
    s = scratch_address(&scratch);
    if (s != ISDF_OK) return s;
    // isdf_kmeans initialises every part of the workspace it reads (centroids,
    // 128-bit sums, labels, snap keys, counters) at the start of each call, so
    // the previous call's contents in the shared array do not leak into this one.
    return isdf_kmeans(w, nx, ny, nz, cell, n_mu, init_idx, max_iter, flags, idx, centroids, objective, labels,
                       stats, scratch, (size_t)ISDF_KMEANS_NOALLOC_SCRATCH_BYTES, stream);
}
