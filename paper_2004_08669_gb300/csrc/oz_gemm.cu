// oz_gemm.cu -- FP64-accurate GEMM emulated on the bf16 tensor cores
// (Ozaki-style error-free splitting), for the FP64-equivalent mixed form.
//
//   D (M x N, column-major FP64) = A . B^t,  A: M x K, B: N x K (FP64, rows
//   contiguous in K after k_oz_split).
//
// Splitting (k_oz_split_rows for row-contiguous operands, one CTA per row;
// k_oz_split in two passes over 32 x 32 tiles otherwise): each row r of an
// operand is scaled by a power of
// two 2^-e_r so that |x| < 1, rounded to a 7s-bit fixed-point integer X, and
// written as s balanced base-2^7 digits, X = sum_i d_i 2^{7(s-i)}, with
// |d_1| <= 128 and |d_i| <= 64 after: every digit is an integer that bf16
// holds exactly.  The digit planes are stored stacked (plane i, row r) as
// K-major bf16 with leading dimension ld.
//
// Products (k_oz_gemm): A.B^t = 2^{e_r + f_c} sum_{i,j} 2^{-7(i+j)} A_i B_j^t.
// Pairs with i + j <= s + 1 are kept; pairs of equal t = i + j share one
// TMEM accumulator.  Over a K-chunk of 512 the FP32 accumulation of every
// group is exact (all partial sums are integers below 2^24 for s <= 6), so
// after each chunk the eight epilogue warps read the groups back, scale them
// by 2^{-7t} (exact) and add them into a double-float (hi, lo) accumulator
// per output element; the end result is written in FP64.  A producer warp
// streams all digit planes of a 32-wide K-tile per stage (3-stage TMA ring,
// 64-byte swizzle) and an MMA warp issues the tcgen05.mma: one per A digit
// plane and run of up to four consecutive B planes (their groups are
// consecutive accumulators).  All mbarrier waits are bounded (error flag, TMEM freed, return).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "ctm_internal.cuh"
#include "oz_gemm.cuh"

namespace ctm {

namespace {

constexpr int kOzBM = 128;
constexpr int kOzBN = 64;
constexpr int kOzKT = 32;       // K per stage (64 bytes of bf16: one 64B-swizzle row)
constexpr int kOzChunk = 512;   // K per exact FP32 accumulation
constexpr long kOzSpin = 1L << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
    for (long i = 0; i < kOzSpin; ++i) {
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
// K-major, 64-byte swizzle: 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t sdesc64(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16u >> 4) << 16;
    d |= (uint64_t)(512u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
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

// (hi, lo) += v with an error-free sum (Knuth's TwoSum).
__device__ __forceinline__ void df_add(float& hi, float& lo, float v) {
    float s = hi + v;
    float bp = s - hi;
    float e = (hi - (s - bp)) + (v - bp);
    hi = s;
    lo += e;
}

// Row exponents of the split: rexp[r] holds the largest biased FP64 exponent
// of row r (subnormals count as 1), 0 for an all-zero row; the row scale is
// 2^e_r with e_r = rexp - 1022 (so |x| < 2^e_r), 0 for a zero row.
__device__ __forceinline__ int oz_e(int raw) { return raw == 0 ? 0 : raw - 1022; }

// The split runs over 32 x 32 tiles (rows r, K-index k) staged in shared
// memory, so that the reads are coalesced along whichever of the two indices
// is contiguous and every row is spread over many CTAs.  Pass 1 takes the row
// maxima of the exponents (atomicMax into rexp, zeroed before); pass 2 writes
// the digit planes, K-contiguous, zero beyond K up to ld.
// src(r, k) = src[r rs + k ks] (* scale[k]); planes[(i Rp + r) ld + k].
template <bool PASS2>
__global__ void __launch_bounds__(256) k_oz_split(int R, int K, int s, const double* __restrict__ src, long rs,
                                                  long ks, const double* __restrict__ scale,
                                                  __nv_bfloat16* __restrict__ planes, int Rp, int ld,
                                                  int* __restrict__ rexp) {
    __shared__ double tile[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int k0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    if (rs == 1 && ks != 1) {  // r contiguous
        for (int kk = ty; kk < 32; kk += 8) {
            const int r = r0 + tx, k = k0 + kk;
            double v = (r < R && k < K) ? src[r + ks * (long)k] : 0.0;
            if (scale && k < K) v *= scale[k];
            tile[tx][kk] = v;
        }
    } else {
        for (int rr = ty; rr < 32; rr += 8) {
            const int r = r0 + rr, k = k0 + tx;
            double v = (r < R && k < K) ? src[rs * (long)r + ks * (long)k] : 0.0;
            if (scale && k < K) v *= scale[k];
            tile[rr][tx] = v;
        }
    }
    __syncthreads();
    const int fbits = 7 * s;
    for (int rr = ty; rr < 32; rr += 8) {
        const int r = r0 + rr, k = k0 + tx;
        if (r >= R) break;  // uniform over the warp
        const double v = tile[rr][tx];
        const uint64_t bits = (uint64_t)__double_as_longlong(v);
        int E = (int)((bits >> 52) & 0x7FF);
        if (!PASS2) {
            int e = ((bits & 0x7FFFFFFFFFFFFFFFull) != 0) ? (E == 0 ? 1 : E) : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
            if (tx == 0 && e > 0) atomicMax(rexp + r, e);
        } else {
            if (k >= ld) continue;
            const int raw = rexp[r];
            long long X = 0;
            if (k < K && raw != 0) {
                const int er = raw - 1022;
                uint64_t mant = bits & 0xFFFFFFFFFFFFFull;
                if (E != 0) mant |= (1ull << 52);
                else E = 1;
                // X = round(|v| 2^(fbits - er)) = round(mant 2^(E - 1075 - er + fbits))
                const int sh = E - 1075 - er + fbits;
                uint64_t mag;
                if (sh >= 0) mag = mant << sh;  // sh <= fbits - 53 < 11 here
                else if (sh > -64) mag = (mant + (1ull << (-sh - 1))) >> (-sh);
                else mag = 0;
                X = (long long)mag;
                if (bits >> 63) X = -X;
            }
            for (int i = 0; i < s; ++i) {
                const int shf = 7 * (s - 1 - i);
                const long long d = (shf > 0) ? ((X + (1ll << (shf - 1))) >> shf) : X;
                X -= d * (1ll << shf);
                // |d| <= 128: an int32 conversion (int64 ones run on the slow FP64 pipe)
                planes[((size_t)i * Rp + r) * ld + k] = __float2bfloat16_rn((float)(int)d);
            }
        }
    }
}

// Shared pieces of the single-kernel splits below.
__device__ __forceinline__ int oz_raw_exp(double v) {
    const uint64_t bits = (uint64_t)__double_as_longlong(v);
    const int E = (int)((bits >> 52) & 0x7FF);
    return ((bits & 0x7FFFFFFFFFFFFFFFull) != 0) ? (E == 0 ? 1 : E) : 0;
}

// round(|v| 2^(fbits - e_r)) with v's sign, e_r = raw - 1022 (integer operations only)
__device__ __forceinline__ long long oz_fixed(double v, int raw, int fbits) {
    const uint64_t bits = (uint64_t)__double_as_longlong(v);
    int E = (int)((bits >> 52) & 0x7FF);
    uint64_t mant = bits & 0xFFFFFFFFFFFFFull;
    if (E != 0) mant |= (1ull << 52);
    else E = 1;
    const int sh = E - 1075 - (raw - 1022) + fbits;
    uint64_t mag;
    if (sh >= 0) mag = mant << sh;
    else if (sh > -64) mag = (mant + (1ull << (-sh - 1))) >> (-sh);
    else mag = 0;
    const long long X = (long long)mag;
    return (bits >> 63) ? -X : X;
}

// digit i of X's balanced base-2^7 expansion (most significant first)
__device__ __forceinline__ __nv_bfloat16 oz_digit(long long& X, int s, int i) {
    const int shf = 7 * (s - 1 - i);
    const long long d = (shf > 0) ? ((X + (1ll << (shf - 1))) >> shf) : X;
    X -= d * (1ll << shf);
    return __float2bfloat16_rn((float)(int)d);
}

// Single-kernel split of operands whose rows are contiguous (ks = 1): one CTA
// per row holds the row in registers (VPT values per thread), reduces the
// exponent and writes all digit planes, coalesced along k.
template <int VPT>
__global__ void __launch_bounds__(256) k_oz_split_rows(int R, int K, int s, const double* __restrict__ src, long rs,
                                                       const double* __restrict__ scale,
                                                       __nv_bfloat16* __restrict__ planes, int Rp, int ld,
                                                       int* __restrict__ rexp) {
    __shared__ int red[8];
    const int tid = threadIdx.x;
    const size_t pstride = (size_t)Rp * ld;
    const int fbits = 7 * s;
    for (int r = blockIdx.x; r < R; r += gridDim.x) {
        const double* row = src + rs * (long)r;
        double v[VPT];
        int e = 0;
#pragma unroll
        for (int j = 0; j < VPT; ++j) {
            const int k = tid + 256 * j;
            double x = 0.0;
            if (k < K) {
                x = row[k];
                if (scale) x *= scale[k];
            }
            v[j] = x;
            e = max(e, oz_raw_exp(x));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
        if ((tid & 31) == 0) red[tid >> 5] = e;
        __syncthreads();
        int raw = red[0];
#pragma unroll
        for (int w = 1; w < 8; ++w) raw = max(raw, red[w]);
        __syncthreads();  // red is reused by the next row
        if (tid == 0) rexp[r] = raw;
#pragma unroll
        for (int j = 0; j < VPT; ++j) {
            const int k = tid + 256 * j;
            if (k < ld) {
                long long X = (k < K && raw != 0) ? oz_fixed(v[j], raw, fbits) : 0;
                for (int i = 0; i < s; ++i) planes[i * pstride + (size_t)r * ld + k] = oz_digit(X, s, i);
            }
        }
    }
}

// Stages of the TMA ring: all S digit planes of A (8 KB each) and B (4 KB
// each) per stage; three stages fit in shared memory up to S = 6.  (A 16-wide
// K-tile with a four-stage ring was measured slower at S = 7.)
template <int S>
struct OzStages {
    static constexpr int value = (S <= 6) ? 3 : 2;
};

template <int S>
__global__ void __launch_bounds__(320, 1)
    k_oz_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M, int N, int K,
              int Mp, int Np, const int* __restrict__ eA, const int* __restrict__ eB, double* __restrict__ D, int ldd,
              int kper, int splits, double* __restrict__ part, int* err, int lowq) {
    constexpr int kOzStages = OzStages<S>::value;
    constexpr int NG = S;                           // groups t = 2 .. S + 1
    constexpr uint32_t A_PLANE = kOzBM * kOzKT * 2;  // 8 KB
    constexpr uint32_t B_PLANE = kOzBN * kOzKT * 2;  // 4 KB
    constexpr uint32_t STAGE = S * (A_PLANE + B_PLANE);
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[kOzStages];
    __shared__ __align__(8) uint64_t empty_bar[kOzStages];
    __shared__ __align__(8) uint64_t acc_full;
    __shared__ __align__(8) uint64_t acc_empty;
    __shared__ uint32_t tmem_slot;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Persistent: this CTA takes tiles blockIdx.x, + gridDim.x, ... of the
    // (row tile, column tile, K slice) space; the stage ring and the
    // accumulator hand-over keep their phases across tiles, so the producer
    // loads the next tile's stages and the MMA warp starts the next tile while
    // the epilogue warps convert and store the previous one.
    const int tm = (M + kOzBM - 1) / kOzBM, tn = (N + kOzBN - 1) / kOzBN;
    const long ntile = (long)tm * tn * splits;
    const int kt_per_chunk = kOzChunk / kOzKT;
    // tile t: its origin, K range, and whether it has work (lower q x q block
    // triangle only when lowq > 0: a tile whose block rows all lie above its
    // first block column is skipped)
    // The tile index runs fastest over the dimension with fewer tiles: the
    // CTAs that take consecutive tiles then share the other operand's tile
    // (C~'s digit planes in C~ V, X's in U^t X), read once from DRAM and
    // from L2 by the rest.
    const bool n_fast = tn < tm;
    auto tile_of = [&](long t, int& m0, int& n0, int& kbeg, int& nk) -> bool {
        const int z = (int)(t / ((long)tm * tn));
        const long xy = t - (long)z * tm * tn;
        m0 = (int)(n_fast ? xy / tn : xy % tm) * kOzBM;
        n0 = (int)(n_fast ? xy % tn : xy / tm) * kOzBN;
        kbeg = z * kper;
        nk = (min(K, kbeg + kper) - kbeg + kOzKT - 1) / kOzKT;
        return !(lowq > 0 && (min(m0 + kOzBM, M) - 1) / lowq < n0 / lowq);
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < kOzStages; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&acc_full, 1);
        mbar_init(&acc_empty, 256);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    if (warp == 8) {
        // ---- producer: all digit planes of one K-tile per stage
        if (lane == 0) {
            long issued = 0;  // K-tiles issued by this CTA over all its tiles
            bool ok = true;
            for (long t = blockIdx.x; t < ntile && ok; t += gridDim.x) {
                int m0, n0, kbeg, nk;
                if (!tile_of(t, m0, n0, kbeg, nk)) continue;
                for (int kt = 0; kt < nk; ++kt, ++issued) {
                    const int st = (int)(issued % kOzStages);
                    if (issued >= kOzStages &&
                        !mbar_wait(&empty_bar[st], (uint32_t)(((issued / kOzStages) - 1) & 1), err)) {
                        ok = false;
                        break;
                    }
                    uint8_t* base = smem + st * STAGE;
                    mbar_expect_tx(&full_bar[st], STAGE);
#pragma unroll
                    for (int i = 0; i < S; ++i) {
                        tma_load_2d(base + i * A_PLANE, &mapA, &full_bar[st], kbeg + kt * kOzKT, i * Mp + m0);
                        tma_load_2d(base + S * A_PLANE + i * B_PLANE, &mapB, &full_bar[st], kbeg + kt * kOzKT,
                                    i * Np + n0);
                    }
                }
            }
            // own copies must land before the CTA may exit
            for (long kt = (issued > kOzStages ? issued - kOzStages : 0); kt < issued; ++kt)
                mbar_wait(&full_bar[kt % kOzStages], (uint32_t)((kt / kOzStages) & 1), err);
        }
    } else if (warp == 9) {
        // ---- MMA issuer
        if (lane == 0) {
            // f32 accumulator, bf16 A and B, both K-major; N is set per MMA
            const uint32_t idesc0 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kOzBM >> 4) << 24);
            bool ok = true;
            long used = 0;    // K-tiles consumed over all tiles
            long chunks = 0;  // accumulator hand-overs over all tiles
            for (long t = blockIdx.x; t < ntile && ok; t += gridDim.x) {
                int m0, n0, kbeg, nk;
                if (!tile_of(t, m0, n0, kbeg, nk)) continue;
                const int nchunk = (nk + kt_per_chunk - 1) / kt_per_chunk;
                for (int c = 0; c < nchunk && ok; ++c, ++chunks) {
                    // the epilogue must have drained the previous hand-over
                    if (chunks > 0 && !mbar_wait(&acc_empty, (uint32_t)((chunks - 1) & 1), err)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const int kt0 = c * kt_per_chunk, kt1 = min(nk, kt0 + kt_per_chunk);
                    for (int kt = kt0; kt < kt1; ++kt, ++used) {
                        const int st = (int)(used % kOzStages);
                        if (!mbar_wait(&full_bar[st], (uint32_t)((used / kOzStages) & 1), err)) {
                            ok = false;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t base = smem_u32(smem + st * STAGE);
                        // A plane i meets B planes j = 0 .. S-1-i (0-based), whose
                        // groups g = i + j are consecutive accumulators, and the
                        // B planes lie consecutively in the stage with the same
                        // 8-row stride: so one MMA of N = 64 c covers c pairs
                        // (c <= 4, N <= 256), 10 MMAs per 16-wide K step for
                        // s = 7 instead of 28.  Every group's first product in
                        // a chunk is the i = 0 one, which overwrites it.
#pragma unroll
                        for (int i = 0; i < S; ++i) {
#pragma unroll
                            for (int j0 = 0; j0 < S - i; j0 += 4) {
                                const int c = (S - i - j0) < 4 ? (S - i - j0) : 4;
                                const uint32_t idesc = idesc0 | ((uint32_t)((c * kOzBN) >> 3) << 17);
                                const uint32_t a0 = base + i * A_PLANE;
                                const uint32_t b0 = base + S * A_PLANE + j0 * B_PLANE;
#pragma unroll
                                for (int kk = 0; kk < kOzKT / 16; ++kk) {
                                    const bool first = (kt == kt0) && (kk == 0) && (i == 0);
                                    mma_bf16(tmem + (uint32_t)((i + j0) * kOzBN), sdesc64(a0 + 32 * kk),
                                             sdesc64(b0 + 32 * kk), idesc, first ? 0u : 1u);
                                }
                            }
                        }
                        mma_commit(&empty_bar[st]);
                    }
                    mma_commit(&acc_full);
                }
            }
            if (!ok) mma_commit(&acc_full);
        }
    } else {
        // ---- epilogue warps 0..7: warp w reads TMEM lanes 32 (w % 4) .. + 31
        // (tile rows) and columns 32 (w / 4) .. + 31, so that each thread holds
        // 32 double-float accumulators of its tile
        const int quad = warp & 3, half = warp >> 2;
        constexpr int EC = kOzBN / 2;
        bool ok = true;
        long chunks = 0;
        for (long t = blockIdx.x; t < ntile && ok; t += gridDim.x) {
            int m0, n0, kbeg, nk;
            if (!tile_of(t, m0, n0, kbeg, nk)) continue;
            const int nchunk = (nk + kt_per_chunk - 1) / kt_per_chunk;
            float hi[EC], lo[EC];
#pragma unroll
            for (int j = 0; j < EC; ++j) {
                hi[j] = 0.f;
                lo[j] = 0.f;
            }
            for (int c = 0; c < nchunk; ++c, ++chunks) {
                if (!mbar_wait(&acc_full, (uint32_t)(chunks & 1), err)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
                for (int g = 0; g < NG; ++g) {
                    const float sc = exp2f(-7.0f * (float)(g + 2));
                    float v[32];
                    tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(g * kOzBN + half * EC), v);
#pragma unroll
                    for (int j = 0; j < EC; ++j) df_add(hi[j], lo[j], v[j] * sc);
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive(&acc_empty);
            }
            // the accumulators are free: this store overlaps the next tile's MMA
            const int row = m0 + quad * 32 + lane;
            if (ok && row < M) {
                const int er = oz_e(eA[row]);
                // split-K partials go to part + z M N (column-major, ld M)
                const int z = kbeg / kper;
                double* out = (splits > 1) ? part + (size_t)z * M * N : D;
                const size_t ldo = (splits > 1) ? (size_t)M : (size_t)ldd;
#pragma unroll
                for (int j = 0; j < EC; ++j) {
                    const int col = n0 + half * EC + j;
                    if (col < N)
                        out[row + ldo * col] = scale_pow2(f2d_bits(hi[j]) + f2d_bits(lo[j]), er + oz_e(eB[col]));
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 oz_encode_fn() {
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

bool oz_map(CUtensorMap* map, const void* base, int K, int rows, int ld, int box_rows) {
    auto fn = oz_encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)kOzKT, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// D = sum over the split-K partials (column-major M x N each).
__global__ void k_oz_reduce(int M, int N, int splits, const double* __restrict__ part, double* __restrict__ D,
                            int ldd) {
    const size_t total = (size_t)M * N;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        double sacc = 0.0;
        for (int z = 0; z < splits; ++z) sacc += part[e + (size_t)z * total];
        D[(e % M) + (size_t)ldd * (e / M)] = sacc;
    }
}

template <int S>
cudaError_t oz_launch(cudaStream_t st, const CUtensorMap& a, const CUtensorMap& b, int M, int N, int K, int Mp, int Np,
                      const int* eA, const int* eB, double* D, int ldd, int kper, int splits, double* part,
                      int* err, int lowq) {
    const size_t smem = 1024 + (size_t)OzStages<S>::value * S * (kOzBM * kOzKT * 2 + kOzBN * kOzKT * 2);
    static const bool attr = [&]() {
        cudaFuncSetAttribute(k_oz_gemm<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        return true;
    }();
    (void)attr;
    // persistent: one CTA per SM (the kernel holds all 512 tensor-memory
    // columns), each looping over tiles
    const long tiles = (long)((M + kOzBM - 1) / kOzBM) * ((N + kOzBN - 1) / kOzBN) * splits;
    int sms = 152, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)std::max<long>(1, std::min<long>(tiles, sms));
    k_oz_gemm<S><<<grid, 320, smem, st>>>(a, b, M, N, K, Mp, Np, eA, eB, D, ldd, kper, splits, part, err, lowq);
    if (splits > 1) {
        const size_t total = (size_t)M * N;
        const int blocks = (int)std::min<size_t>((total + 255) / 256, 4 * 152);
        k_oz_reduce<<<blocks, 256, 0, st>>>(M, N, splits, part, D, ldd);
    }
    return cudaGetLastError();
}

}  // namespace

int oz_rows_pad(int R, int box) { return ((R + box - 1) / box) * box; }
int oz_ld(int K) { return ((K + 63) / 64) * 64; }

size_t oz_operand_bytes(int R, int K, int s, bool is_a) {
    int Rp = oz_rows_pad(R, is_a ? kOzBM : kOzBN);
    return (size_t)s * Rp * oz_ld(K) * 2;
}

void oz_split(cudaStream_t st, int R, int K, int s, const double* src, int lds, const double* scale, void* planes,
              bool is_a, int* rexp) {
    oz_split_strided(st, R, K, s, src, lds, 1, scale, planes, is_a, rexp);
}

template <int VPT>
void oz_launch_rows(cudaStream_t st, int R, int K, int s, const double* src, long rs, const double* scale,
                    void* planes, int Rp, int ld, int* rexp) {
    const int grid = std::min(R, 152 * 16);
    k_oz_split_rows<VPT><<<grid, 256, 0, st>>>(R, K, s, src, rs, scale, (__nv_bfloat16*)planes, Rp, ld, rexp);
}

void oz_split_strided(cudaStream_t st, int R, int K, int s, const double* src, long rs, long ks,
                      const double* scale, void* planes, bool is_a, int* rexp) {
    if (R <= 0) return;
    const int Rp = oz_rows_pad(R, is_a ? kOzBM : kOzBN), ld = oz_ld(K);
    // rows contiguous: one kernel (a CTA per row); otherwise two passes over tiles
    if (ks == 1 && ld <= 256 * 24) {
        if (ld <= 256 * 2) oz_launch_rows<2>(st, R, K, s, src, rs, scale, planes, Rp, ld, rexp);
        else if (ld <= 256 * 8) oz_launch_rows<8>(st, R, K, s, src, rs, scale, planes, Rp, ld, rexp);
        else oz_launch_rows<24>(st, R, K, s, src, rs, scale, planes, Rp, ld, rexp);
        return;
    }
    cudaMemsetAsync(rexp, 0, sizeof(int) * (size_t)R, st);
    const dim3 blk(32, 8);
    k_oz_split<false><<<dim3((K + 31) / 32, (R + 31) / 32), blk, 0, st>>>(R, K, s, src, rs, ks, scale,
                                                                           (__nv_bfloat16*)planes, Rp, ld, rexp);
    k_oz_split<true><<<dim3((ld + 31) / 32, (R + 31) / 32), blk, 0, st>>>(R, K, s, src, rs, ks, scale,
                                                                          (__nv_bfloat16*)planes, Rp, ld, rexp);
}
int oz_plan_slices(int K, int splits_req) {
    const int chunks = (K + kOzChunk - 1) / kOzChunk;
    const int want = std::max(1, std::min(splits_req, chunks));
    const int kper = ((chunks + want - 1) / want) * kOzChunk;
    return (K + kper - 1) / kper;
}

cudaError_t oz_gemm(cudaStream_t st, int s, int M, int N, int K, const void* Aplanes, const int* eA,
                    const void* Bplanes, const int* eB, double* D, int ldd, int* err, double* part,
                    size_t part_cap, int splits_req, int lowq) {
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    if (s < 3 || s > 7) return cudaErrorInvalidValue;
    // split-K when the output tiles alone cannot fill the GPU, or as requested
    const long tiles = (long)((M + kOzBM - 1) / kOzBM) * ((N + kOzBN - 1) / kOzBN);
    int splits = 1, kper = K;
    if (splits_req > 0) {
        const int chunks = (K + kOzChunk - 1) / kOzChunk;
        const int want = std::max(1, std::min(splits_req, chunks));
        kper = ((chunks + want - 1) / want) * kOzChunk;
        splits = (K + kper - 1) / kper;
        if (splits < 2) {
            splits = 1;
            kper = K;
        } else if (!part || (size_t)splits * M * N > part_cap) {
            return cudaErrorInvalidValue;
        }
    } else if (part && tiles < 152 && K >= 2 * kOzChunk) {
        const long chunks = (K + kOzChunk - 1) / kOzChunk;
        long want = std::min<long>((2 * 152 + tiles - 1) / tiles, chunks);
        want = std::min<long>(want, (long)(part_cap / ((size_t)M * N)));
        if (want > 1) {
            kper = (int)(((chunks + want - 1) / want) * kOzChunk);
            splits = (K + kper - 1) / kper;
        }
        if (splits < 2) {
            splits = 1;
            kper = K;
        }
    }
    // B may be A's own planes (a Gram matrix A A^t): then its rows sit at A's
    // plane stride
    const bool sameAB = (Bplanes == Aplanes) && (eB == eA) && N <= M;
    const int Mp = oz_rows_pad(M, kOzBM), Np = sameAB ? Mp : oz_rows_pad(N, kOzBN), ld = oz_ld(K);
    CUtensorMap ma, mb;
    if (!oz_map(&ma, Aplanes, K, s * Mp, ld, kOzBM) || !oz_map(&mb, Bplanes, K, s * Np, ld, kOzBN))
        return cudaErrorInvalidValue;
    const int lq = splits > 1 ? 0 : lowq;  // partial tiles must all be written
    switch (s) {
        case 3: return oz_launch<3>(st, ma, mb, M, N, K, Mp, Np, eA, eB, D, ldd, kper, splits, part, err, lq);
        case 4: return oz_launch<4>(st, ma, mb, M, N, K, Mp, Np, eA, eB, D, ldd, kper, splits, part, err, lq);
        case 5: return oz_launch<5>(st, ma, mb, M, N, K, Mp, Np, eA, eB, D, ldd, kper, splits, part, err, lq);
        case 6: return oz_launch<6>(st, ma, mb, M, N, K, Mp, Np, eA, eB, D, ldd, kper, splits, part, err, lq);
        default: return oz_launch<7>(st, ma, mb, M, N, K, Mp, Np, eA, eB, D, ldd, kper, splits, part, err, lq);
    }
}

}  // namespace ctm
