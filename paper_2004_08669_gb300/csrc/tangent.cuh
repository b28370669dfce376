// tangent.cuh -- kernels of the forward-mode beta tangent of one CTMRG step
// (the derivative of the step of Algorithm 3 of arXiv:2004.08669).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

namespace ctm {

// out += d/dbeta of the blockwise vertex-weight contraction of X over its
// live x live q x q blocks (spin-fastest layout, leading dims ldx / ldo):
// each block M maps to E o (E (M o E_in) E), E = exp(beta v.v) (Eq. 1-2),
// whose beta-derivative has E_dot = (v.v) E = -Eh at each factor.  The inner
// factor E_in is E, or with inner_h the bond-impurity table Eh (its
// derivative -Eh^2 / E).  Requires q * q <= 1024.
cudaError_t wcontract_dbeta(cudaStream_t st, int q, int live, const double* X, int ldx, const double* E,
                            const double* Eh, double* out, int ldo, bool inner_h = false);

// out[i] = sum_t A[t, i] B[t, i] w[t % q] for the n columns (w NULL: 1).
void column_dots(cudaStream_t st, int N, int n, const double* A, int lda, const double* B, int ldb,
                 const double* wspin, int q, double* out);

// Zero the rows and columns t of the N x N matrix A whose block index t / q
// is >= live (the dead part of the renormalised leg).
void mask_live(cudaStream_t st, int N, int q, int live, double* A, int lda);

// The in-block coupling of the eigen tangent for the first n of bt Ritz
// pairs: with Hs = (H + H^t) / 2,
//   K[j + bt i] = Hs[j, i] / (theta_i - theta_j) (0 when |theta_i - theta_j|
//   <= tol |theta_0|, i.e. inside a cluster and on the diagonal),
//   lam_dot[i] = Hs[i, i].
void tangent_coupling(cudaStream_t st, int bt, int n, const double* H, int ldh, const double* theta, double tol,
                      double* K, double* lam_dot);

// One step of the deflated iteration, column i scaled by 1 / theta_i:
// Y <- (Rhs + T) / theta (T may be NULL: Y <- Rhs / theta).  part receives,
// per CTA, the largest |change| of Y and the largest |Y| (2 * kTanParts).
constexpr int kTanParts = 256;
void deflate_update(cudaStream_t st, int N, int n, const double* Rhs, const double* T, const double* theta,
                    double* Y, double* part);

// part[blk] = partial sums of x . y over kTanParts CTAs.
void dot_partial(cudaStream_t st, size_t n, const double* x, const double* y, double* part);

// y += x (n entries).
void add_inplace(cudaStream_t st, size_t n, const double* x, double* y);

// out = Rdot / k - R * c (the tangent of R / ||R|| with c = kdot / k^2).
void tangent_normalise(cudaStream_t st, size_t n, const double* R, const double* Rdot, double inv_k, double c,
                       double* out);

}  // namespace ctm
