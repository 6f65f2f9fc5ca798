// Shared helpers of the CUDA library: status handling, complex arithmetic
// with explicit IEEE rounding, and the layout of the plan.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/isdf.h"

#define ISDF_CUDA_TRY(expr)                                   \
    do {                                                      \
        cudaError_t e_ = (expr);                              \
        if (e_ != cudaSuccess) return ISDF_ERR_CUDA;          \
    } while (0)

#define ISDF_LAUNCH_CHECK()                                   \
    do {                                                      \
        cudaError_t e_ = cudaGetLastError();                  \
        if (e_ != cudaSuccess) return ISDF_ERR_CUDA;          \
    } while (0)

#define ISDF_TRY(expr)                                        \
    do {                                                      \
        isdf_status s_ = (expr);                              \
        if (s_ != ISDF_OK) return s_;                         \
    } while (0)

// host-side count of the kernels this library has launched (for benchmarks)
void isdf_note_launch();

// Joins a forked stream back into the caller's stream on every return path.
// After `side` was made to wait on the caller's stream, arm() the guard; the
// normal path calls join() where the work is meant to merge. If the function
// returns early (an error after the fork), the destructor records `ev` on
// the side stream and makes the caller's stream wait on it, so no work of the
// side stream stays unjoined (a stream capture stays valid, and the caller's
// stream does not run ahead of kernels that still use the plan's buffers).
struct StreamJoin {
    cudaStream_t main = nullptr, side = nullptr;
    cudaEvent_t ev = nullptr;
    bool armed = false;
    void arm(cudaStream_t m, cudaStream_t s, cudaEvent_t e)
    {
        main = m;
        side = s;
        ev = e;
        armed = true;
    }
    cudaError_t join()
    {
        if (!armed) return cudaSuccess;
        armed = false;
        cudaError_t e = cudaEventRecord(ev, side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(main, ev, 0);
        return e;
    }
    ~StreamJoin() { join(); }
};

static inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

static inline bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Device status word of a plan: first failure wins.
struct DeviceStatus {
    int32_t code;    // isdf_status
    int32_t detail;  // e.g. the failing pivot
    int32_t ticket;  // arrival counter of the fused Cholesky step: its last CTA writes back and resets it
    int32_t pad;
};

__device__ __forceinline__ void set_status(DeviceStatus *st, int32_t code, int32_t detail)
{
    if (atomicCAS(&st->code, 0, code) == 0) st->detail = detail;
}

// ---- complex arithmetic on double2 (re, im) --------------------------------
// double -> float with integer operations only (the FP64 pipe is the scarce unit on
// GB300): the mantissa is rounded half-up at bit 29 (error <= 2^-24 relative), values
// below float's normal range become +-0, overflow becomes inf and a NaN stays a NaN.
__device__ __forceinline__ float d2f_int(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7FF) - 1023 + 127;
    unsigned int f;
    if (e == 0x7FF - 1023 + 127)
        f = 0x7F800000u | ((b & 0xFFFFFFFFFFFFFull) ? 0x400000u : 0u);
    else if (e <= 0)
        f = 0u;
    else if (e >= 255)
        f = 0x7F800000u;
    else {
        f = ((unsigned int)e << 23) | (unsigned int)((b >> 29) & 0x7FFFFFu);
        f += (unsigned int)((b >> 28) & 1u);   // carries into the exponent when the mantissa is full
        if (f > 0x7F800000u) f = 0x7F800000u;
    }
    return __uint_as_float(sign | f);
}

// float -> double by moving the bits (exact for normal floats; others take the conversion)
__device__ __forceinline__ double f2d_int(float f)
{
    const unsigned int u = __float_as_uint(f);
    const unsigned int e = (u >> 23) & 0xFFu;
    if (e == 0u || e == 0xFFu) return (double)f;
    const unsigned long long b = ((unsigned long long)(u >> 31) << 63) |
                                 ((unsigned long long)(e - 127u + 1023u) << 52) |
                                 ((unsigned long long)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)b);
}

__device__ __forceinline__ double2 cload(const double2 *p, int64_t i) { return p[i]; }
__device__ __forceinline__ double2 cload(const float2 *p, int64_t i)
{
    float2 v = p[i];
    return make_double2((double)v.x, (double)v.y);
}
__device__ __forceinline__ void cstore(double2 *p, int64_t i, double2 v) { p[i] = v; }
__device__ __forceinline__ void cstore(float2 *p, int64_t i, double2 v)
{
    p[i] = make_float2((float)v.x, (float)v.y);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__device__ __forceinline__ double2 cmulc(double2 a, double2 b)
{
    return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
