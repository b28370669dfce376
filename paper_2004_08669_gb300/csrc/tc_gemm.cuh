// tc_gemm.cuh -- host entry points of the tcgen05 GEMM (tc_gemm.cu).
#pragma once

#include <cuda_runtime.h>

namespace ctm {

// Leading dimension (elements) of a K-major operand copy: K rounded up to 64.
int tc_ld(int K);

// Copy rows of a column-major FP64 matrix into a K-major operand (bf16 or
// fp32): dst[r * ldo + k] = src[k + lds * r] * (scale ? scale[k] : 1), zero
// for K <= k < ldo.
void to_operand(cudaStream_t st, bool bf16, int R, int K, const double* src, int lds, const double* scale,
                void* dst, int ldo);

// Launch shape of one GEMM: tile width bn (64, 128 or 256 columns of D per
// CTA) and the number of K slices (split-K; > 1 needs a partial buffer of
// slices * M * N doubles).
struct TcPlan {
    int bn;
    int splits;
};

// The untuned shape (bn 256 for N > 128, else 128; no split).
TcPlan tc_default_plan(int M, int N, int K, bool bf16);

// K slices a plan launches (its split count, lowered so that no slice is
// empty); *kchunk receives the K-tiles per slice.
int tc_plan_slices(const TcPlan& p, int K, bool bf16, int* kchunk);

// D (M x N, column-major FP64, ldd) = alpha * A . B^t + beta * D with A (M x K)
// and B (N x K) K-major operands of leading dimension lda, ldb (multiples of
// 64).  bf16: kind::f16 with bf16 operands; else kind::tf32 on fp32 storage.
// *err (device int) is set to 1 if a bounded wait gave up.  plan NULL: the
// default shape.  A split plan writes slices * M * N doubles of part
// (capacity part_cap doubles) and sums them in order; cudaErrorInvalidValue
// when they do not fit.  lowq > 0 (no split-K): only the q x q blocks on or
// below the block diagonal of D are needed; tiles entirely above it are
// skipped (left unwritten).
cudaError_t tc_gemm(cudaStream_t st, bool bf16, int M, int N, int K, double alpha, const void* A, int lda,
                    const void* B, int ldb, double beta, double* D, int ldd, int* err, const TcPlan* plan = nullptr,
                    double* part = nullptr, size_t part_cap = 0, int lowq = 0);

}  // namespace ctm
