// Generic strided complex FP64 GEMM used by the FP64 fit, the Cholesky
// factorisation, the triangular inverse and the adjoint.
#pragma once

#include "common.cuh"

enum { ZG_C128 = 0, ZG_C64 = 1 };
enum { ZG_K_ALL = 0, ZG_K_FROM_MAX_MN = 1, ZG_K_FROM_N0 = 2 };

// C(m, n) = alpha * sum_k opA(m, k) opB(k, n) + beta * C(m, n)            (single)
// C(m, n) = P1(m, n) * conj(P2(m, n)), P_i = sum_k opA_i(m, k) opB_i(k, n) (dual)
// opA(m, k) = [conj] A[m*sam + k*sak], opB(k, n) = [conj] B[k*sbk + n*sbn],
// all indices counted in complex elements. Batched (single) form: product b
// uses A1 + b*bsa, B1 + b*bsb, C + b*bsc.
struct ZOperand {
    const void *p;
    int64_t s0, s1;   // A: (m, k) strides; B: (k, n) strides
    int conj;
    int type;         // ZG_C128 or ZG_C64
};

struct ZGemm {
    int M, N, K;
    ZOperand A1, B1, A2, B2;  // A2, B2 only in dual mode
    int dual;
    void *C;
    int64_t scm, scn;
    int ctype;
    double alpha;
    int beta;                 // 0 or 1
    void *C1, *C2;            // dual mode: optional copies of P1, P2 (complex128, C's strides)
    int lower_only;           // skip tiles entirely above the diagonal
    int kmode;                // ZG_K_ALL, ZG_K_FROM_MAX_MN, ZG_K_FROM_N0
    int k_to_m_end;           // stop k at the tile's last row (A lower triangular)
    int splits;               // > 1: split-K into `partial`, then reduced
    double2 *partial;         // splits * M * N complex128
    int tile;                 // output tile edge: 64 (default) or 32
    int batch;                // > 1: independent products, operands offset by the strides below
    int64_t bsa, bsb, bsc;    // batch strides of A1, B1 and C (complex elements)
};

isdf_status zgemm(const ZGemm &g, cudaStream_t st);

// zgemm with the tile edge and split-K chosen from the problem shape so that
// small M x N products with deep K still fill the GPU (partial may be NULL).
isdf_status zgemm_auto(const ZGemm &g, double2 *partial, size_t partial_elems, cudaStream_t st);

// C = conj(C)^T in the strict upper triangle (completes a Hermitian matrix
// whose lower triangle was computed); n x n, row-major complex128, ld.
isdf_status hermitian_mirror(double2 *C, int n, int64_t ld, cudaStream_t st);
