// Tensor-core (tcgen05) split-precision path of the Theta fit (ISDF_MIXED).
#pragma once

#include "plan.cuh"

bool mixed_supported(int n, int n_mu, int64_t ld_phi, int64_t ld_psi, int dtype);
// scale bounds and FP16 splits of the orbitals (independent of the interpolation points)
isdf_status mixed_prepare_orbitals(isdf_plan *p, cudaStream_t st);
// after M^-1: its scale and the rotated B operands (needs mixed_prepare_orbitals first)
isdf_status mixed_prepare(isdf_plan *p, cudaStream_t st);
isdf_status mixed_fit(isdf_plan *p, int64_t row_begin, int64_t row_count, void *theta, int64_t ld_theta,
                      cudaStream_t st);
// adjoint of the Theta fit on the tensor cores for one range of rows (see isdf_fit_theta_backward)
isdf_status mixed_backward(isdf_plan *p, int64_t row_begin, int64_t row_count, const void *grad_theta,
                           int64_t ld_grad, const void *K, double dV, void *grad_phi, int64_t ld_gphi,
                           void *grad_psi, int64_t ld_gpsi, double *loss, cudaStream_t st);
// device-side failure of the tensor-core kernels (ISDF_ERR_TIMEOUT, ISDF_ERR_NONFINITE or 0); synchronous
isdf_status mixed_status(isdf_plan *p, int32_t *code);
void mixed_release(isdf_plan *p);
