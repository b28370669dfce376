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
    double* S1;     // npad x npad second buffer of S, or NULL (then one round per grid barrier)
    double* diag;   // npad
    int* rank;      // npad (also the Jacobi sweep tags)
    double* gdots;  // 3 b
    double* gQ;     // 4 b
    int* gkind;     // b
};

// Scratch of the warm-start Rayleigh-Ritz refinement (device, b x b each).
struct OaWork {
    double* X;
    double* W1;
    double* S;
    double* R;
    double* E;
    double* part;   // partial maxima (<= 608)
    int* clus;      // b flags: pair (i, i+1) is a strongly coupled doublet
    double* gpart;  // split-K partial sums, max_splits b^2
    int max_splits;
    // host-side record of the last call: 0 converged, 1 a strongly coupled
    // pair that is not a doublet, 2 a large rotation, 3 iteration cap,
    // 4 a multiplet of three or more
    int fail_reason = 0;
    int last_iter = 0;
    double last_max = 0.0;
};

int coop_grid_limit(const void* fn, int block, size_t smem);

// Scratch of the cluster-aware Rayleigh-Ritz refinement (rr_refine.cu):
// n x n double-float matrices (H, two X buffers, H X, X^t H X, X^t X, the
// update), the clusters' rotations (32 x n), Ritz values, cluster lists and
// the strongly coupled pairs.
struct RrcWork {
    float2 *Hd, *X0, *X1, *W, *S, *G, *F, *Qc;
    double* lam;
    int *root, *cid, *cpos, *clist, *coff, *edges;
    int edge_cap;
    int nmax;
};
size_t rrc_workspace_bytes(int n);
void rrc_carve(void* base, int n, RrcWork& w);
bool rrc_supported(int n);

// Eigenpairs of the warm Rayleigh-Ritz matrix H (n x n, FP64, nearly
// diagonal) by cluster-aware iterative refinement in double-float, one
// cooperative launch.  On success it writes the eigenvectors into ew.S
// (double-float, npad layout) and the Ritz values into ew.diag, exactly where
// the double-float Jacobi solver leaves them, and sets ctl->rrc_ok = 1;
// otherwise ctl->rrc_ok stays 0.  Launch jacobi_f64(..., df = true, skip =
// &ctl->rrc_ok) behind it: it solves only when the refinement gave up, and
// sorts in either case.  nhead: the leading columns (in the warm order, |Ritz
// value| descending) whose pairs must converge; pairs of two later columns
// (the oversampling's guard vectors) are left unrotated (0: all columns).
cudaError_t rr_cluster_refine(cudaStream_t st, int n, const double* H, int ldh, RrcWork& w, EigWork& ew,
                              DevCtl* ctl, int max_iter, int nhead = 0);

// Warm-start Rayleigh-Ritz by simultaneous Jacobi rotations (Ogita-Aishima
// refinement from X = I).  Returns iterations used, or -1 when it did not
// converge (largest rotation <= tol) in max_iter iterations: fall back to Jacobi.
// head: columns (in the warm order) whose Ritz pairs must converge; the rest
// are the oversampling tail, rotated with damped angles and not tested.
int rr_refine_f64(cudaStream_t st, int b, int head, const double* H, int ldh, OaWork& w, EigWork& ew,
                  double* theta, double* Sout, int ldo, double tol, int max_iter, DevCtl* ctl, DevCtl* hctl,
                  int* nlaunch);

// Eigenpairs of the symmetric n x n matrix H (FP64 cyclic Jacobi, round-robin
// parallel order), sorted by |theta| descending: theta (n), Sout (n x n, ldo).
// A pair is rotated while |a_pq| > max(rel_tol sqrt|a_pp a_qq|, floor_rel
// max_i |h_ii|) (rel_tol is at least the FP64 unit roundoff; floor_rel 0
// keeps the purely relative criterion).
// df: hold A and S as double-float pairs and compute on the FP32 pipe (about
// 48 significant bits; for the mixed-precision forms).
// skip (device, may be NULL): when *skip != 0 at run time the solve is left
// out (another solver already wrote w.S and w.diag) and only the sort runs.
// nhead > 0: only couplings with at least one index below nhead are driven
// below the threshold (a warm block's leading columns; the later ones are
// guard vectors whose mutual rotations do not matter); 0: all.
cudaError_t jacobi_f64(cudaStream_t st, int n, const double* H, int ldh, EigWork& w, double* theta,
                       double* Sout, int ldo, int max_sweeps, DevCtl* ctl, double rel_tol = 0.0,
                       double floor_rel = 0.0, bool df = false, const int* skip = nullptr, int nhead = 0);

// G + shift_rel * trace(G) * I = L L^t, L lower in place (blocked, panel 32).
// df: double-float arithmetic on the FP32 pipe (mixed-precision forms).
// skip (device, may be NULL): when *skip != 0 at run time the factorisation
// is left out (orth_check chose a Newton-Schulz correction).
cudaError_t cholesky_f64(cudaStream_t st, int n, double* G, int ld, double shift_rel, DevCtl* ctl, bool df = false,
                         const int* skip = nullptr);

// X = (3 I - (G + G^t)/2) / 2: the Newton-Schulz orthogonality correction
// of a block whose Gram matrix G is close to I.
void ns_coeff_f64(cudaStream_t st, int b, const double* G, int ldg, double* X, int ldx);

// X = L^{-1} for lower-triangular L (upper part of X zeroed); scratch:
// ceil(n / 32) * 1024 doubles.  skip as for cholesky_f64.  df: the
// substitution over the off-diagonal blocks in double-float on the FP32 pipe
// (the mixed-precision forms), else FP64.
void trinv_f64(cudaStream_t st, int n, const double* L, int ld, double* X, int ldx, double* scratch,
               const int* skip = nullptr, bool df = false);

// The defect max|G - I| of a Gram matrix; if it is at most thresh, sets
// ctl->orth_ns and writes X = (3I - G)/2 (a Newton-Schulz correction),
// otherwise clears ctl->orth_ns (pass it as skip to cholesky_f64/trinv_f64).
// slot: 0 for a block's first orthonormalisation pass, 1 for later ones
// (the defect histogram ctl->orth_hist)
void orth_check(cudaStream_t st, int b, const double* G, int ldg, double thresh, double* X, int ldx, DevCtl* ctl,
                int slot = 1);

void resid_f64(cudaStream_t st, int N, int ncol, const double* T, const double* Z, int ld,
               const double* theta, double* res);
void decide(cudaStream_t st, int b, int L, int m, double tol, double tol_c, const double* theta,
            const double* res, DevCtl* ctl);
void next_block(cudaStream_t st, int N, int b, const double* T, const double* Z, int ld,
                const double* theta, double eps_theta, double* Vn);

// The second of two power steps before one orthonormalisation, filtered:
// V <- (c Y / theta - V) / (c - 1), c = 2 theta^2 / theta_{b-1}^2 (the
// degree-2 Chebyshev polynomial on [-|theta_{b-1}|, |theta_{b-1}|]
// normalised at theta), from Y = C~ (C~ V / theta); in place in V.
// Three power steps before one orthonormalisation, filtered by the degree-3
// Chebyshev polynomial on [-|theta_{b-1}|, |theta_{b-1}|] normalised at theta:
// V <- (4u^3 Y/theta - 3u T)/(4u^3 - 3u), u = theta/|theta_{b-1}|, from
// T = C~ V / theta and Y = C~^3 V / theta^2 (V, T, Y distinct).
void cheb3_block(cudaStream_t st, int N, int b, const double* Y, const double* T, double* V, int ld,
                 const double* theta, double eps_theta);
void cheb2_block(cudaStream_t st, int N, int b, const double* Y, double* V, int ld, const double* theta,
                 double eps_theta);
void gauge_align(cudaStream_t st, int N, int b, double* Z, const double* V, int ld, const double* theta,
                 double tol_c, EigWork& w);
void randn_block(cudaStream_t st, int N, int b, double* V, int ld, uint64_t seed);
void identity_block(cudaStream_t st, int N, int b, double* V, int ld);

}  // namespace ctm
