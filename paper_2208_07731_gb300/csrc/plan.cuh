// The plan of one Theta fit: caller orbitals, gathered rows, M and its
// factors, block scratch and the adjoint accumulators.
#pragma once

#include "common.cuh"
#include "ozaki.cuh"

struct MixedBuffers;

#define ISDF_TIMER_KINDS 7
#define ISDF_HOST_STAGES 3   // device staging blocks of isdf_fit_theta_host

struct isdf_plan {
    const void *phi, *psi;
    int64_t ld_phi, ld_psi, n_r;
    int n_phi, n_psi, dtype, n_mu, mode;
    int64_t max_rows;
    cudaStream_t last_stream;
    DeviceStatus *status;
    int64_t *idx;
    double2 *phi_mu, *psi_mu;                 // n_mu x n (complex128)
    double2 *M, *Amu, *Bmu, *L, *Linv, *W;    // n_mu x n_mu
    double2 *tmp, *tmp2;                      // n_mu x n_mu scratch
    double2 *Mbar, *gphi_mu, *gpsi_mu;        // adjoint accumulators
    double2 *blkY, *blkT, *blkA, *blkB, *blkG;  // max_rows x n_mu block scratch
    double2 *partial;                         // split-K partials
    size_t partial_elems;
    MixedBuffers *mixed;                      // tensor-core path (ISDF_MIXED)
    int use_oz;                               // plan-update products on the tensor cores (exact slicing)
    OzWork oz;                                // their slice scratch
    int *oz_err;                              // device flag of those kernels: 1 a wait gave up, 2 non-finite input
    long long wait_budget;                    // cycle budget of the tensor-core kernels' waits (0: default)
    cudaStream_t side;                        // look-ahead stream of the Cholesky factorisation
    cudaEvent_t ev_fork, ev_join;             // its fork / join points
    cudaStream_t aux;                         // orbital operand preparation, concurrent with a8-a9
    cudaEvent_t ev_aux_fork, ev_aux_join;
    // isdf_fit_theta_host: device staging blocks (max_rows x n_mu each), their copy stream and events
    void *hstage[ISDF_HOST_STAGES];
    cudaStream_t hcopy, hcopy2;               // each block leaves in two halves, one per stream (copy engine)
    cudaEvent_t ev_hfit[ISDF_HOST_STAGES], ev_hcopied[ISDF_HOST_STAGES], ev_hhalf[ISDF_HOST_STAGES], ev_hjoin, ev_hjoin2;
    // optional event timing: kinds 0 Gram kernel, 1 M^-1 application kernel,
    // 2 gather + M, 3 Cholesky factor, 4 triangular inverse, 5 M^-1 = L^-H L^-1,
    // 6 tensor-core operand preparation
    int timing;
    int tcap;
    int tused[ISDF_TIMER_KINDS];
    cudaEvent_t *tev[ISDF_TIMER_KINDS];   // 2 * tcap events per kind: (start, stop) pairs
    int64_t *trows[ISDF_TIMER_KINDS];     // grid rows processed by each timed launch
};

// record a start event before a timed launch (no-op unless timing is enabled)
void timer_start(isdf_plan *p, int kind, cudaStream_t st);
// record the stop event after the launch of `rows` grid rows
void timer_stop(isdf_plan *p, int kind, cudaStream_t st, int64_t rows);
