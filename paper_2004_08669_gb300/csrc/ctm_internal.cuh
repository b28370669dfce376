// ctm_internal.cuh -- device-side helpers and kernel declarations shared by the
// translation units of libctm_gb300.so.
//
// Device layout: every (m q)-long combined index is spin-fastest,
// t = s + q * gamma, so that the live block of the extended corner (the rows
// with gamma < D) is its leading (q D) x (q D) block.  P is m x N column-major
// (P[alpha + m t]); C~ and all N x b blocks are column-major.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cuda/atomic>

namespace ctm {

constexpr int kThreads = 256;

// Device control block: flags and scalars written by kernels and read back by
// the host once per subspace iteration / step.
struct DevCtl {
    // eigen stage
    int meff_new;        // kept states after the multiplet rule
    int sub_converged;   // Ritz residuals below tol
    int jac_sweeps;      // sweeps of the last Jacobi
    int jac_status;      // 0 ok, 1 sweep cap, 2 barrier timeout
    int chol_status;     // 0 ok, 1 non-positive pivot, 2 barrier timeout
    int numeric_bad;     // NaN/Inf seen
    int pad0, pad1;
    double resid;        // max residual / |theta_0|
    double theta0;
    double theta_range;  // min |theta_i| / |theta_0| over the block's non-negligible Ritz values
    // step stage
    double kappa;
    double delta;
    double SE;
    double prev_kappa;
    int have_prev;
    int live;            // current live rows of P (D)
    int pad2, pad3;
    // barrier words (cooperative kernels)
    unsigned int bar_count;  // zeroed before every cooperative launch
    unsigned int bar_pad;
    int rot_count[64];   // rotations per Jacobi sweep
    // observables
    double obs_M_num, obs_u_num, obs_z4, obs_SE;
    // warm Rayleigh-Ritz refinement
    double oa_maxE;
    // cluster-aware refinement of the mixed-precision forms (rr_refine.cu)
    int rrc_ok;            // 1: the refinement produced the eigenpairs
    int rrc_iters;         // its iterations (couplings measured)
    int rrc_fail;          // 0 ok, 1 edge list full, 2 cluster too large, 3 iteration cap, 4 non-finite
    int rrc_done;          // converged at the last check (read by all blocks)
    int rrc_nedges;        // strongly coupled pairs found in the last check
    int rrc_ncl;           // clusters (> 1 member) of the last check
    int rrc_maxcl;         // largest cluster seen
    unsigned int rrc_maxc;  // bits of the largest relative coupling (non-negative float)
    unsigned int rrc_maxr;  // bits of the largest orthonormality defect
    int rrc_pad;
    // per iteration of the last refinement: largest coupling, largest
    // orthonormality defect, strongly coupled pairs, largest cluster
    float rrc_hist_c[16];
    float rrc_hist_r[16];
    int rrc_hist_ne[16];
    int rrc_hist_cl[16];
    // re-orthonormalisation: 1 when the block's defect max|G - I| was small
    // enough for a Newton-Schulz correction in place of a factorisation
    int orth_ns;
    float orth_defect;   // that defect (the last check)
    unsigned long long orth_max_bits;  // its running maximum (bits of a non-negative double)
    // checks so far by decade of the defect (bucket k: 10^-k <= d < 10^(1-k),
    // bucket 0: d >= 1, bucket 9: d < 1e-8), for the first pass and the others
    unsigned int orth_hist[2][10];
    // block 0's clock (ns) at the end of each phase of the last refinement's
    // first 16 iterations: after P1, P2, P3a, P3b, P3c, P3e, P4
    unsigned long long rrc_t0;
    unsigned int rrc_tph[16][8];
};

// FP32 -> FP64 by bit construction (the conversion instruction runs on the
// FP64 pipe, which is slow on this part); zero, subnormal and non-finite
// inputs take the instruction.
__device__ __forceinline__ double f2d_bits(float x) {
    const uint32_t u = __float_as_uint(x);
    const uint32_t ex = (u >> 23) & 0xFFu;
    if ((u << 1) == 0u) return __longlong_as_double((long long)((uint64_t)(u >> 31) << 63));
    if (ex == 0u || ex == 0xFFu) return (double)x;
    return __longlong_as_double((long long)(((uint64_t)(u >> 31) << 63) | ((uint64_t)(ex + 896u) << 52) |
                                            ((uint64_t)(u & 0x7FFFFFu) << 29)));
}

// v * 2^e by adding e to the exponent field; ldexp when the input or the
// result is zero, subnormal, non-finite or out of range.
__device__ __forceinline__ double scale_pow2(double v, int e) {
    const uint64_t b = (uint64_t)__double_as_longlong(v);
    const int ex = (int)((b >> 52) & 0x7FFu);
    if ((b << 1) == 0u) return v;
    const int ne = ex + e;
    if (ex == 0 || ex == 0x7FF || ne <= 0 || ne >= 0x7FF) return ldexp(v, e);
    return __longlong_as_double((long long)((b & ~(0x7FFull << 52)) | ((uint64_t)ne << 52)));
}

// Grid-wide barrier for cooperative launches on a monotonic arrival counter:
// the host zeroes *count before the launch, and a block's e-th barrier waits
// until e * gridDim.x arrivals are counted (one release-add per block, then
// acquire loads; no read-modify-write sits on the wait path).  Every wait is
// bounded: after 2^22 polls (about a second) the barrier records a timeout
// (2) in *err and returns false in every thread of the block, so a missing
// block can never hang the GPU.
__device__ __forceinline__ bool grid_sync(unsigned int* count, unsigned int& epoch, int* err) {
    __syncthreads();
    __shared__ int s_fail;
    ++epoch;
    if (threadIdx.x == 0) {
        s_fail = 0;
        const unsigned int target = epoch * gridDim.x;
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
        long polls = 0;
        unsigned int v;
        while (true) {
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
            if ((int)(v - target) >= 0) break;
            if (++polls > (1L << 22)) {
                atomicExch(err, 2);
                s_fail = 1;
                break;
            }
        }
        if (*(volatile int*)err == 2) s_fail = 1;
    }
    __syncthreads();
    return s_fail == 0;  // uniform across the block
}

// ---------------------------------------------------------------- kernels
// FP64 GEMM: C = alpha op(A) op(B) (+ beta C), column-major, optional per-k
// scaling of B (scaleK[k] * B(k, j)), split-K over blockIdx.z writing
// partial sums to C + z * splitStride (beta ignored when splits > 1).
// Returns the number of kernels launched (1, or 2 with split-K).  lowq > 0
// (no split-K): only the q x q blocks on or below the block diagonal of C are
// needed; tiles entirely above it are skipped (left unwritten).
int gemm_f64(cudaStream_t st, bool transA, bool transB, int M, int N, int K, double alpha,
             const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc,
             const double* scaleK, int splits, double* partial, int lowq = 0);

// Blockwise vertex-weight contraction, in place on an N x N matrix (spin-fastest
// index): every q x q block X_{gamma gamma'} becomes E o (E (X o E1) E), where
// E1 is E (plain weight) or E o h (bond impurity).  Blocks with gamma or
// gamma' >= *live are zero and skipped.  sym: X is symmetric and E1 = E, so
// only the blocks gamma >= gamma' are contracted and their transposes written
// (the result is then exactly symmetric).
void wcontract_f64(cudaStream_t st, int m, int q, double* X, int ldx, const double* E,
                   const double* E1, const int* live, bool sym = false);

// The same contraction with arithmetic 0 = FP64, 1 = FP32, 2 = double-float.
void wcontract_ar(cudaStream_t st, int arith, int m, int q, double* X, int ldx, const double* E, const double* E1,
                  const int* live, bool sym = false);

}  // namespace ctm
