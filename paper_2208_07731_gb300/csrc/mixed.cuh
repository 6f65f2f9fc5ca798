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

// Exchange application (Eq. v2) on the tensor cores: H = (Phi_b Phi_mu^H) o V_b with the
// Hadamard product in the first product's epilogue, then out_b = -H_b Psi_mu; split-FP16 x3
// products with FP32 accumulation, V complex64, output complex128.
struct MixedExchange;
bool mixed_exchange_supported(int n_phi, int n_psi, int n_mu);
isdf_status mixed_exchange_create(MixedExchange **out, int64_t n_r, int n_phi, int n_psi, int n_mu, int64_t max_rows);
isdf_status mixed_exchange_apply(MixedExchange *x, const void *phi, int64_t ld_phi, int orb_dtype,
                                 const double2 *phi_mu, const double2 *psi_mu, const float2 *V, int64_t ld_v,
                                 int64_t row_begin, int64_t row_count, double2 *out, int64_t ld_out, cudaStream_t st);
// device-side failure (ISDF_ERR_TIMEOUT, ISDF_ERR_NONFINITE or 0); synchronous
int mixed_exchange_error(MixedExchange *x);
void mixed_exchange_release(MixedExchange *x);
