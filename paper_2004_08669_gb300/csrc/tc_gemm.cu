// tc_gemm.cu -- tcgen05 tensor-core GEMM for the contractions of the CTMRG
// step in the reduced-precision forms (TF32 or BF16 operands, FP32
// accumulation in tensor memory, FP64 output).
//
//   D (M x N, column-major FP64) = alpha * A . B^t (+ beta * D)
//   A: M x K, B: N x K, both K-major (row r of the operand is contiguous in k),
//   stored as BF16 or FP32 with a leading dimension that is a multiple of 64.
//
// One CTA computes a 128 x BN tile (BN = 64, 128 or 256) over one slice of
// K (split-K: blockIdx.z; partial tiles go to an FP64 buffer that a second
// kernel sums in a fixed order).  Warp 0 (one lane)
// streams K-tiles of A and B into a 4-stage shared-memory ring with TMA
// (128-byte swizzle); warp 1 (one lane) issues tcgen05.mma into a TMEM
// accumulator and releases each stage with tcgen05.commit; then all four
// warps read their 32 TMEM lanes back with tcgen05.ld and write FP64.
// Every mbarrier wait is bounded: on timeout the kernel records an error,
// waits (bounded) for its own copies and MMAs, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "ctm_internal.cuh"
#include "tc_gemm.cuh"

namespace ctm {

namespace {

constexpr int kStages = 4;
constexpr int kBM = 128;
constexpr long kSpinLimit = 1L << 24;  // polls of one mbarrier before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait; returns false (and records the error) on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
    for (long i = 0; i < kSpinLimit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i > 32) __nanosleep(20);
    }
    atomicExch(err, 1);
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16u >> 4) << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

template <int KIND>  // 0: kind::f16 (bf16), 1: kind::tf32
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if (KIND == 0) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <int KIND, int BN>
__global__ void __launch_bounds__(128, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M, int N,
              int K, double alpha, double beta, double* __restrict__ D, int ldd, int kchunk,
              double* __restrict__ part, int* err, int lowq) {
    // K elements per 128-byte swizzle row: 64 (bf16) or 32 (fp32 / tf32)
    constexpr int KT = (KIND == 0) ? 64 : 32;
    constexpr int KMMA = (KIND == 0) ? 16 : 8;  // K per instruction (32 bytes)
    constexpr uint32_t A_BYTES = kBM * 128;
    constexpr uint32_t B_BYTES = BN * 128;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;
    uint8_t* sB = smem + kStages * A_BYTES;
    __shared__ __align__(8) uint64_t full_bar[kStages];
    __shared__ __align__(8) uint64_t empty_bar[kStages];
    __shared__ __align__(8) uint64_t accum_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
    // lower q x q block triangle only: a tile entirely above it exits at once
    // (uniformly, before any barrier or tensor-memory allocation)
    if (lowq > 0 && (min(m0 + kBM, M) - 1) / lowq < n0 / lowq) return;
    // this CTA's K-tiles: [kt0, kt0 + nk); the host makes every slice non-empty
    const int nk_all = (K + KT - 1) / KT;
    const int kt0 = blockIdx.z * kchunk;
    const int nk = max(0, min(nk_all - kt0, kchunk));

    if (threadIdx.x == 0) {
        s_fail = 0;
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&accum_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"((uint32_t)BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    int issued_tma = 0;  // producer: k-tiles whose copies were issued
    if (warp == 0 && lane == 0) {
        for (int kt = 0; kt < nk; ++kt) {
            int s = kt % kStages;
            if (kt >= kStages) {
                if (!mbar_wait(&empty_bar[s], ((kt / kStages) - 1) & 1, err)) {
                    s_fail = 1;
                    break;
                }
            }
            mbar_expect_tx(&full_bar[s], A_BYTES + B_BYTES);
            tma_load_2d(sA + s * A_BYTES, &mapA, &full_bar[s], (kt0 + kt) * KT, m0);
            tma_load_2d(sB + s * B_BYTES, &mapB, &full_bar[s], (kt0 + kt) * KT, n0);
            ++issued_tma;
        }
    } else if (warp == 1 && lane == 0) {
        // instruction descriptor: D f32, A/B bf16 (1) or tf32 (2), K-major, N, M
        const uint32_t fmt = (KIND == 0) ? 1u : 2u;
        const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(BN >> 3) << 17) |
                               ((uint32_t)(kBM >> 4) << 24);
        int kt = 0;
        for (; kt < nk; ++kt) {
            int s = kt % kStages;
            if (!mbar_wait(&full_bar[s], (kt / kStages) & 1, err)) {
                s_fail = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint32_t a0 = smem_u32(sA + s * A_BYTES), b0 = smem_u32(sB + s * B_BYTES);
#pragma unroll
            for (int k = 0; k < KT / KMMA; ++k) {
                mma<KIND>(tmem, sdesc(a0 + 32 * k), sdesc(b0 + 32 * k), idesc, (kt > 0 || k > 0) ? 1u : 0u);
            }
            mma_commit(&empty_bar[s]);
        }
        mma_commit(&accum_bar);  // fires when every issued MMA has completed
    }
    __syncwarp();
    // epilogue: all four warps
    bool ok = mbar_wait(&accum_bar, 0, err);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // the producer's copies must have landed before the CTA exits
    if (warp == 0 && lane == 0) {
        for (int kt = (issued_tma > kStages ? issued_tma - kStages : 0); kt < issued_tma; ++kt) {
            int s = kt % kStages;
            mbar_wait(&full_bar[s], (kt / kStages) & 1, err);
        }
    }
    if (ok && !s_fail && nk > 0) {
        const int row = m0 + warp * 32 + lane;
        // split-K: slice z of the partial buffer (M x N, leading dimension M)
        double* out = part ? part + (size_t)blockIdx.z * M * N : D;
        const size_t ldo = part ? (size_t)M : (size_t)ldd;
        const double bet = part ? 0.0 : beta;
#pragma unroll 1
        for (int c = 0; c < BN; c += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
            if (row < M) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    int col = n0 + c + j;
                    if (col < N) {
                        double* d = out + row + ldo * col;
                        double val = alpha * (double)v[j];
                        if (bet != 0.0) val += bet * (*d);
                        *d = val;
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BN)
                     : "memory");
    }
}

// D = sum_z part[z] + beta * D, the slices summed in order z = 0, 1, ...
__global__ void k_tc_reduce(int M, int N, int splits, const double* __restrict__ part, double beta,
                            double* __restrict__ D, int ldd) {
    const size_t tot = (size_t)M * N;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        double s = part[e];
        for (int z = 1; z < splits; ++z) s += part[(size_t)z * tot + e];
        double* d = D + (e % M) + (size_t)ldd * (e / M);
        if (beta != 0.0) s += beta * (*d);
        *d = s;
    }
}

// FP64 -> operand precision, K-major copy with zero padding:
// dst[r * ldo + k] = src(r, k) for k < K, 0 for K <= k < ldo.
// src(r, k) = src[k + lds * r] (the operand row r is column r of a
// column-major matrix), times scale[k] when scale is given.
template <typename T>
__global__ void k_to_operand(int R, int K, const double* __restrict__ src, int lds,
                             const double* __restrict__ scale, T* __restrict__ dst, int ldo) {
    size_t tot = (size_t)R * ldo;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        int k = (int)(e % ldo), r = (int)(e / ldo);
        double v = 0.0;
        if (k < K) {
            v = src[k + (size_t)lds * r];
            if (scale) v *= scale[k];
        }
        if constexpr (sizeof(T) == 2) {
            dst[e] = __float2bfloat16_rn((float)v);
        } else {
            // round to TF32 (10 explicit mantissa bits, nearest, ties away)
            uint32_t t;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"((float)v));
            dst[e] = __uint_as_float(t);
        }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    // resolved once (thread-safe initialisation of a local static)
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return (PFN_cuTensorMapEncodeTiled_v12000)p;
        return nullptr;
    }();
    return fn;
}

bool make_map(CUtensorMap* map, const void* base, bool bf16, int K, int rows, int ld, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    const int esz = bf16 ? 2 : 4;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * esz};
    cuuint32_t box[2] = {(cuuint32_t)(128 / esz), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                    const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int KIND, int BN>
cudaError_t launch_tc(cudaStream_t st, const CUtensorMap& a, const CUtensorMap& b, int M, int N, int K, double alpha,
                      double beta, double* D, int ldd, int splits, int kchunk, double* part, int* err,
                      int lowq) {
    const size_t smem = 1024 + (size_t)kStages * (kBM * 128 + BN * 128);
    static const bool attr = [&]() {
        cudaFuncSetAttribute(k_tc_gemm<KIND, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        return true;
    }();
    (void)attr;
    dim3 grid((M + kBM - 1) / kBM, (N + BN - 1) / BN, splits);
    k_tc_gemm<KIND, BN><<<grid, 128, smem, st>>>(a, b, M, N, K, alpha, beta, D, ldd, kchunk,
                                                  splits > 1 ? part : nullptr, err, splits > 1 ? 0 : lowq);
    if (splits > 1) {
        const size_t total = (size_t)M * N;
        const int blocks = (int)std::min<size_t>((total + 255) / 256, 4 * 152);
        k_tc_reduce<<<blocks, 256, 0, st>>>(M, N, splits, part, beta, D, ldd);
    }
    return cudaGetLastError();
}

template <int KIND>
cudaError_t launch_bn(int bn, cudaStream_t st, const CUtensorMap& a, const CUtensorMap& b, int M, int N, int K,
                      double alpha, double beta, double* D, int ldd, int splits, int kchunk, double* part, int* err,
                      int lowq) {
    if (bn == 64)
        return launch_tc<KIND, 64>(st, a, b, M, N, K, alpha, beta, D, ldd, splits, kchunk, part, err, lowq);
    if (bn == 128)
        return launch_tc<KIND, 128>(st, a, b, M, N, K, alpha, beta, D, ldd, splits, kchunk, part, err, lowq);
    return launch_tc<KIND, 256>(st, a, b, M, N, K, alpha, beta, D, ldd, splits, kchunk, part, err, lowq);
}

}  // namespace

int tc_ld(int K) { return ((K + 63) / 64) * 64; }

void to_operand(cudaStream_t st, bool bf16, int R, int K, const double* src, int lds, const double* scale,
                void* dst, int ldo) {
    size_t tot = (size_t)R * ldo;
    int grid = (int)std::min<size_t>((tot + 255) / 256, 152 * 16);
    if (grid < 1) grid = 1;
    if (bf16)
        k_to_operand<__nv_bfloat16><<<grid, 256, 0, st>>>(R, K, src, lds, scale, (__nv_bfloat16*)dst, ldo);
    else
        k_to_operand<float><<<grid, 256, 0, st>>>(R, K, src, lds, scale, (float*)dst, ldo);
}

TcPlan tc_default_plan(int M, int N, int K, bool bf16) {
    (void)M;
    (void)K;
    (void)bf16;
    return TcPlan{N > 128 ? 256 : 128, 1};
}

int tc_plan_slices(const TcPlan& p, int K, bool bf16, int* kchunk) {
    const int KT = bf16 ? 64 : 32;
    const int nk = (K + KT - 1) / KT;
    int s = std::max(1, std::min(p.splits, nk));
    const int ch = (nk + s - 1) / s;
    if (kchunk) *kchunk = ch;
    return (nk + ch - 1) / ch;  // no slice is left empty
}

cudaError_t tc_gemm(cudaStream_t st, bool bf16, int M, int N, int K, double alpha, const void* A, int lda,
                    const void* B, int ldb, double beta, double* D, int ldd, int* err, const TcPlan* plan,
                    double* part, size_t part_cap, int lowq) {
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    if ((lda % 64) || (ldb % 64)) return cudaErrorInvalidValue;
    const TcPlan p = plan ? *plan : tc_default_plan(M, N, K, bf16);
    if (p.bn != 64 && p.bn != 128 && p.bn != 256) return cudaErrorInvalidValue;
    int kchunk = 0;
    const int splits = tc_plan_slices(p, K, bf16, &kchunk);
    if (splits > 1 && (!part || (size_t)splits * M * N > part_cap)) return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, bf16, K, M, lda, kBM) || !make_map(&mb, B, bf16, K, N, ldb, p.bn))
        return cudaErrorInvalidValue;
    if (bf16) return launch_bn<0>(p.bn, st, ma, mb, M, N, K, alpha, beta, D, ldd, splits, kchunk, part, err, lowq);
    return launch_bn<1>(p.bn, st, ma, mb, M, N, K, alpha, beta, D, ldd, splits, kchunk, part, err, lowq);
}

}  // namespace ctm
