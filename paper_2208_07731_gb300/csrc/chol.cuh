#pragma once

#include "common.cuh"

struct isdf_plan;

// In place: L (n x n, row-major, holding a copy of M0 = M) becomes the
// Cholesky factor (strict upper triangle zeroed); Linv = L^-1 (lower);
// W = M^-1 = L^-H L^-1 (full Hermitian). tmp: n x n scratch. A pivot that is
// not above 1e-13 times M's original diagonal entry is recorded in *st
// (ISDF_ERR_NOT_HPD, detail = pivot index; ISDF_ERR_NONFINITE for NaN).
// part: split-K scratch of part_n complex128 elements (may be NULL).
// plan (may be NULL) supplies the look-ahead stream, event timings of the three
// stages (kinds 3, 4, 5) and, when plan->use_oz is set, the scratch of the
// tensor-core FP64 products used for M^-1 and the upper inverse levels.
isdf_status cholesky_inverse(const double2 *M0, double2 *L, double2 *Linv, double2 *W, double2 *tmp, int n,
                             double2 *part, size_t part_n, DeviceStatus *st, cudaStream_t stream,
                             isdf_plan *plan);
