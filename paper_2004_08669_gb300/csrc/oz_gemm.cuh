// oz_gemm.cuh -- host entry points of the FP64-emulating tensor-core GEMM.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace ctm {

// Bytes of the stacked digit planes of an operand with R rows of length K
// and s digits (A role: rows padded to 128; B role: to 64).
size_t oz_operand_bytes(int R, int K, int s, bool is_a);

// Split rows src(r, k) = src[k + lds r] (* scale[k]) into s bf16 digit planes
// and one exponent per row (rexp, R ints: the largest biased FP64 exponent of
// the row, 0 for a zero row; the row is scaled by 2^(rexp - 1022)).
void oz_split(cudaStream_t st, int R, int K, int s, const double* src, int lds, const double* scale, void* planes,
              bool is_a, int* rexp);

// Same with general strides: src(r, k) = src[r rs + k ks] (* scale[k]).
void oz_split_strided(cudaStream_t st, int R, int K, int s, const double* src, long rs, long ks,
                      const double* scale, void* planes, bool is_a, int* rexp);

// D (M x N, column-major FP64, ldd) = A . B^t from split operands (A: M rows,
// B: N rows, length K, s digits, 3 <= s <= 7).  *err (device) set on timeout.
// part (part_cap doubles, may be null): split-K partials, used when the
// output tiles alone cannot fill the GPU (splits_req = 0), or for the K
// slices requested (splits_req >= 1; slices are whole 512-wide exact chunks,
// cudaErrorInvalidValue if their partials do not fit part_cap).  lowq > 0
// (no split-K): only the q x q blocks on or below the block diagonal of D
// are needed; output tiles entirely above it are skipped (left unwritten).
cudaError_t oz_gemm(cudaStream_t st, int s, int M, int N, int K, const void* Aplanes, const int* eA,
                    const void* Bplanes, const int* eB, double* D, int ldd, int* err, double* part = nullptr,
                    size_t part_cap = 0, int splits_req = 0, int lowq = 0);

// K slices oz_gemm launches for a requested split count (whole exact chunks).
int oz_plan_slices(int K, int splits_req);

}  // namespace ctm
