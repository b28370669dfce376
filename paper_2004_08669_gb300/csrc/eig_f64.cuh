// eig_f64.cuh -- host entry points of the FP64 eigen-stage kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ctm_internal.cuh"

namespace ctm {

// Scratch of the small dense FP64 solvers (all device pointers).
struct EigWork {
    double* A0;     // npad x npad (Jacobi, two buffers)
    double* A1;
    double* S;      // npad x npad accumulated rotations
    double* diag;   // npad
    int* rank;      // npad
    double* gdots;  // 3 b
    double* gQ;     // 4 b
    int* gkind;     // b
};

int coop_grid_limit(const void* fn, int block, size_t smem);

// Eigenpairs of the symmetric n x n matrix H (FP64 cyclic Jacobi, round-robin
// parallel order), sorted by |theta| descending: theta (n), Sout (n x n, ldo).
cudaError_t jacobi_f64(cudaStream_t st, int n, const double* H, int ldh, EigWork& w, double* theta,
                       double* Sout, int ldo, int max_sweeps, DevCtl* ctl);

// G + shift_rel * trace(G) * I = L L^t, L lower in place (blocked, panel 32).
cudaError_t cholesky_f64(cudaStream_t st, int n, double* G, int ld, double shift_rel, DevCtl* ctl);

// X = L^{-1} for lower-triangular L.
void trinv_f64(cudaStream_t st, int n, const double* L, int ld, double* X, int ldx);

void resid_f64(cudaStream_t st, int N, int ncol, const double* T, const double* Z, int ld,
               const double* theta, double* res);
void decide(cudaStream_t st, int b, int L, int m, double tol, double tol_c, const double* theta,
            const double* res, DevCtl* ctl);
void next_block(cudaStream_t st, int N, int b, const double* T, const double* Z, int ld,
                const double* theta, double eps_theta, double* Vn);
void gauge_align(cudaStream_t st, int N, int b, double* Z, const double* V, int ld, const double* theta,
                 double tol_c, EigWork& w);
void randn_block(cudaStream_t st, int N, int b, double* V, int ld, uint64_t seed);
void identity_block(cudaStream_t st, int N, int b, double* V, int ld);

}  // namespace ctm
