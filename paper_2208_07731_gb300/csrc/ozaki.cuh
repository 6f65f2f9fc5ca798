// FP64 complex GEMMs on the tcgen05 tensor cores by exact integer slicing
// (the Ozaki scheme). Used for the large FP64 products of the plan update
// (M^-1 = L^-H L^-1, the upper levels of the triangular inverse) when the
// tensor-core path is available.
#pragma once

#include <cuda_fp16.h>

#include "common.cuh"
#include "zgemm.cuh"

// Plan-owned scratch for the slices and the row scales.
struct OzWork {
    __half *sa, *sb;                 // slices of the A rows and of the rotated B rows
    size_t cap_a, cap_b;             // capacity in halves
    unsigned long long *ma, *mb;     // per-row max |x| (double bits)
    size_t cap_ma, cap_mb;           // capacity in rows
    int *gsum;                       // exact int32 group sums of a buffered product (or NULL)
    size_t cap_g;                    // capacity in ints
    long long wait_budget;           // cycle budget of the pipeline waits (0: the default; < 0: test hook)
};

// Halves and rows needed for an M x N x K product (batch products).
void oz_sizes(int M, int N, int K, int batch, size_t *halves_a, size_t *halves_b, size_t *rows_a, size_t *rows_b);

// True if g (single, complex128 operands and output) can run on the Ozaki path
// with the given scratch.
bool oz_fits(const ZGemm &g, const OzWork &w);

// C = alpha op(A) op(B) + beta C with the ZGemm conventions (strides, conj,
// lower_only, kmode, k_to_m_end, batch); the result carries an error of the
// order of an FP64 GEMM's (slices of 8 bits, 56 bits per operand, products of
// slice pairs with s + t <= 8). Device errors go to *err: 1 for a bounded wait
// that gave up, 2 for an infinite or NaN operand entry (first error wins).
isdf_status oz_zgemm(const ZGemm &g, const OzWork &w, int *err, cudaStream_t st);
