"""CPU FP64 oracle for the complex-valued K-means ISDF (arXiv 2208.07731).

TEST INFRASTRUCTURE ONLY: a plain, slow, obviously correct restatement of the
paper's method that the CUDA path is checked against. Only the tests, the
smoke check and the CPU-baseline leg of the benchmark may import it; the
product path never does. It shares no code with the CUDA library and never
imports it.

Layout of the inputs (the same as the CUDA path's): Phi, Psi are N_r x N
row-major complex arrays (complex64 inputs are upcast exactly to complex128
here); the grid index is r = (ix*ny + iy)*nz + iz with x_r = h*(ix, iy, iz).

Every function is pinned by the CPU tests (tests/test_oracle_*.py) against
closed forms, brute force, explicit formation of Z, textbook least squares,
invariances and finite differences. No function is parity-unpinned.
"""
from .oracle import (  # noqa: F401
    load, weights, kmeans, kmeans_update, kmeans_assign, kmeans_snap, fixed_point_scale, gather, form_M, cholesky, gram_hadamard,
    theta_rows, fit_theta, surrogate_loss, surrogate_grad_theta, theta_backward,
    grid_coords, explicit_Z, isdf_error, cluster_residual,
    kernel_hat, poisson, exchange_apply, exchange_direct, qrcp_sketch, qrcp_points,
    shared_weights,
)
