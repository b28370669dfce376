// xi.cuh -- host entry points of the correlation-length kernels (xi.cu).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace ctm {

// Dynamic shared memory of the centre-vertex contraction for q spin states;
// *ta receives the tile of the first leg that one block handles.
size_t xi_w_smem(int q, int* ta);

// A2 = centre-vertex contraction of A1 (both (m q) x (m q), column-major):
// A2[(a + m t) + mq (s' + q g')] = sum_{s,u} W(s, t, s', u) A1[(a + m s) + mq (u + q g')],
// W(s, t, s', u) = E_st E_ts' E_s'u E_us.  cudaErrorInvalidValue if q is too
// large for the shared-memory slab.
cudaError_t xi_wcontract(cudaStream_t st, int m, int q, const double* A1, const double* E, double* A2);

// Blocks of the first pass of xi_dots (its partial buffer holds k of them per column).
int xi_dots_blocks(size_t n);

// out[j] = V[:, j] . w for j < k (V: n x k, leading dimension ldv), summed in
// a fixed order through part (k * xi_dots_blocks(n) doubles).
void xi_dots(cudaStream_t st, size_t n, int k, const double* V, size_t ldv, const double* w, double* part,
             double* out);

// w -= V[:, :k] c  (k <= 128; c on the device)
void xi_sub_multi(cudaStream_t st, size_t n, int k, const double* V, size_t ldv, const double* c, double* w);

// *beta_out = sqrt(dot[0]); vnext = w / *beta_out (zero if it is zero)
void xi_normalise(cudaStream_t st, size_t n, const double* w, const double* dot, double* vnext, double* beta_out);

// Tk (k x k, column-major) = tridiag(beta[0..k-2], alpha[0..k-1], beta[0..k-2])
void xi_tridiag(cudaStream_t st, int k, const double* alpha, const double* beta, double* Tk);

}  // namespace ctm
