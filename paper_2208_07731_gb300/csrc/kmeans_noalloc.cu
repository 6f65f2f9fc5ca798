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
// is a host-side stand-in), so the first call on each device, with that device
// current, asks the runtime for the array's device address once and keeps it.
#include <mutex>

#include "common.cuh"

namespace {

static __device__ __align__(256) unsigned char g_kmeans_scratch[ISDF_KMEANS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 256;
std::mutex g_lock;
void *g_addr[kMaxDevices] = {};

// device address of g_kmeans_scratch on the current device (set up once per device)
isdf_status scratch_address(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return ISDF_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return ISDF_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_kmeans_scratch) != cudaSuccess || !p) return ISDF_ERR_CUDA;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return ISDF_OK;
}

}  // namespace

extern "C" isdf_status isdf_kmeans_noalloc(const double *w, int32_t nx, int32_t ny, int32_t nz, const double *cell,
                                           int32_t n_mu, const int64_t *init_idx, int32_t max_iter, int32_t flags,
                                           int64_t *idx, double *centroids, double *objective, int32_t *labels,
                                           int64_t *stats, void *stream)
{
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
