// gemm_f64.cu -- FP64 contraction kernels of the CTMRG step (CUDA cores).
//
//  * k_gemm_f64: tiled FP64 GEMM (64 x 64 x 16 tiles, 4 x 4 register
//    micro-tiles) used for the extension X1 = P^t diag(omega) P, the block
//    products C~ V, V^t Y, V S, the Gram matrices and the P update
//    (Algorithm 3, the PDGEMM call sites), with split-K for the short-wide
//    products whose output is only b x b.
//  * k_wcontract: the vertex-weight contraction of Sub-CTMRG (the second
//    PDGEMM of Algorithm 3 together with both P-Index permutations).  The
//    matrix form w factorises into bond weights E(a,b) = exp(beta v_a.v_b):
//    with the corner order of Eq. (1), each q x q block M = X1_{gamma gamma'}
//    maps to E o (E (M o E) E), which is exactly the P-Index / X2 W /
//    P-Index sequence in 4 q^3 instead of 2 q^4 operations per block.
#include "ctm_internal.cuh"

namespace ctm {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm_f64(int M, int N, int K, int kchunk, double alpha,
                                                  const double* __restrict__ A, int lda,
                                                  const double* __restrict__ B, int ldb, double beta,
                                                  double* __restrict__ C, int ldc,
                                                  const double* __restrict__ scaleK,
                                                  double* __restrict__ partial, int lowq) {
    __shared__ double As[BK][BM];
    __shared__ double Bs[BK][BN + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    // lower q x q block triangle only: tiles entirely above it exit at once
    if (lowq > 0 && (min(m0 + BM, M) - 1) / lowq < n0 / lowq) return;
    const int kbeg = blockIdx.z * kchunk;
    const int kend = min(K, kbeg + kchunk);
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

    for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int l = tid + 256 * r;
            int i, k;
            if (!TA) {
                i = l & 63;
                k = l >> 6;
            } else {
                k = l & 15;
                i = l >> 4;
            }
            int gi = m0 + i, gk = k0 + k;
            double v = 0.0;
            if (gi < M && gk < kend) v = TA ? A[gk + (size_t)lda * gi] : A[gi + (size_t)lda * gk];
            As[k][i] = v;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int l = tid + 256 * r;
            int j, k;
            if (!TB) {
                k = l & 15;
                j = l >> 4;
            } else {
                j = l & 63;
                k = l >> 6;
            }
            int gj = n0 + j, gk = k0 + k;
            double v = 0.0;
            if (gj < N && gk < kend) {
                v = TB ? B[gj + (size_t)ldb * gk] : B[gk + (size_t)ldb * gj];
                if (scaleK) v *= scaleK[gk];
            }
            Bs[k][j] = v;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[k][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[k][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    if (gridDim.z > 1) {
        double* Pz = partial + (size_t)blockIdx.z * M * N;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int gj = n0 + ty + 16 * j;
            if (gj >= N) continue;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                int gi = m0 + tx + 16 * i;
                if (gi < M) Pz[gi + (size_t)M * gj] = alpha * acc[i][j];
            }
        }
        return;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        int gj = n0 + ty + 16 * j;
        if (gj >= N) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int gi = m0 + tx + 16 * i;
            if (gi >= M) continue;
            double* c = C + gi + (size_t)ldc * gj;
            double v = alpha * acc[i][j];
            if (beta != 0.0) v += beta * (*c);
            *c = v;
        }
    }
}

// Fixed-order sum of the split-K partials (deterministic).
__global__ void k_splitk_reduce(int M, int N, int splits, const double* __restrict__ partial,
                                double beta, double* __restrict__ C, int ldc) {
    size_t total = (size_t)M * N;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int z = 0; z < splits; ++z) s += partial[e + (size_t)z * total];
        int i = (int)(e % M), j = (int)(e / M);
        double* c = C + i + (size_t)ldc * j;
        *c = (beta != 0.0) ? s + beta * (*c) : s;
    }
}

// Block (g, g') of the blk-th contraction: all live^2 blocks, or with sym the
// lower triangle g >= g' only (row by row), whose transposes are written too.
__device__ __forceinline__ void wc_block(long blk, int live, bool sym, int& g, int& gp) {
    if (!sym) {
        g = (int)(blk % live);
        gp = (int)(blk / live);
        return;
    }
    int gg = (int)((sqrtf(8.0f * (float)blk + 1.0f) - 1.0f) * 0.5f);
    while (gg > 0 && (long)gg * (gg + 1) / 2 > blk) --gg;
    while ((long)(gg + 1) * (gg + 2) / 2 <= blk) ++gg;
    g = gg;
    gp = (int)(blk - (long)gg * (gg + 1) / 2);
}

// One thread per element of nb q x q blocks at a time.
__global__ void k_wcontract(int m, int q, double* __restrict__ X, int ldx,
                            const double* __restrict__ E, const double* __restrict__ E1,
                            const int* __restrict__ live_ptr, bool sym) {
    extern __shared__ double sh[];
    const int q2 = q * q;
    const int nb = max(1, (int)blockDim.x / q2);
    double* sE = sh;
    double* sE1 = sE + q2;
    double* G = sE1 + q2;       // nb blocks
    double* T1 = G + nb * q2;   // nb blocks
    for (int e = threadIdx.x; e < q2; e += blockDim.x) {
        sE[e] = E[e];
        sE1[e] = E1[e];
    }
    const int live = min(*live_ptr, m);
    const long nblk = sym ? (long)live * (live + 1) / 2 : (long)live * live;
    const int jb = threadIdx.x / q2;       // local block slot
    const int el = threadIdx.x - jb * q2;  // element within the block
    const bool act = jb < nb;
    const int i = el % q, j = el / q;      // (row spin, column spin)
    __syncthreads();
    for (long base = (long)blockIdx.x * nb; base < nblk; base += (long)gridDim.x * nb) {
        long blk = base + jb;
        bool ok = act && blk < nblk;
        size_t off = 0, offT = 0;
        int g = 0, gp = 0;
        if (ok) {
            wc_block(blk, live, sym, g, gp);
            off = (size_t)q * g + (size_t)ldx * ((size_t)q * gp);
            offT = (size_t)q * gp + (size_t)ldx * ((size_t)q * g);
            G[jb * q2 + el] = X[off + i + (size_t)ldx * j] * sE1[el];  // M o E1
        }
        __syncthreads();
        if (ok) {  // T1 = G E
            double s = 0.0;
            for (int k = 0; k < q; ++k) s = fma(G[jb * q2 + i + q * k], sE[k + q * j], s);
            T1[jb * q2 + el] = s;
        }
        __syncthreads();
        if (ok) {  // out = E o (E T1)
            double s = 0.0;
            for (int k = 0; k < q; ++k) s = fma(sE[i + q * k], T1[jb * q2 + k + q * j], s);
            const double v = sE[el] * s;
            X[off + i + (size_t)ldx * j] = v;
            if (sym && g != gp) X[offT + j + (size_t)ldx * i] = v;
        }
        __syncthreads();
    }
}

// ---- the same contraction in other arithmetic: plain FP32, or double-float
// (an unevaluated sum hi + lo of two floats, ~48 significant bits; Dekker's
// products and Knuth's sums) for the FP64-emulating form, where GB300's FP32
// pipe is 64 times faster than its FP64 pipe.
struct ArF32 {
    using T = float;
    struct Acc {
        float s;
    };
    __device__ static T load(double x) { return (float)x; }
    __device__ static double store(T a) { return (double)a; }
    __device__ static T mul(T a, T b) { return a * b; }
    __device__ static Acc acc0() { return Acc{0.f}; }
    __device__ static void acc(Acc& c, T a, T b) { c.s = fmaf(a, b, c.s); }
    __device__ static T fin(Acc c) { return c.s; }
};

struct ArDF {
    using T = float2;  // x = hi, y = lo
    __device__ static T quick(float s, float e) {
        float h = s + e;
        return make_float2(h, e - (h - s));
    }
    __device__ static T load(double x) {
        float h = (float)x;
        return make_float2(h, (float)(x - (double)h));
    }
    __device__ static double store(T a) { return (double)a.x + (double)a.y; }
    __device__ static T mul(T a, T b) {
        float p = a.x * b.x;
        float e = fmaf(a.x, b.x, -p);
        e = fmaf(a.x, b.y, fmaf(a.y, b.x, e));
        return quick(p, e);
    }
    __device__ static T add(T a, T b) {
        float s = a.x + b.x;
        float bb = s - a.x;
        float e = (a.x - (s - bb)) + (b.x - bb);
        e += a.y + b.y;
        return quick(s, e);
    }
    // Dot products in the manner of Ogita, Rump and Oishi's Dot2: the high
    // parts' products are summed by error-free two-sums, every low-order
    // term into one float, normalised once at the end.
    struct Acc {
        float h, l;
    };
    __device__ static Acc acc0() { return Acc{0.f, 0.f}; }
    __device__ static void acc(Acc& c, T a, T b) {
        const float p = a.x * b.x;
        const float pe = fmaf(a.x, b.x, -p);
        const float sum = c.h + p;
        const float bb = sum - c.h;
        const float e = (c.h - (sum - bb)) + (p - bb);
        c.h = sum;
        c.l += (e + pe) + fmaf(a.x, b.y, a.y * b.x);
    }
    __device__ static T fin(Acc c) { return quick(c.h, c.l); }
};

// One thread per row i and W consecutive columns j of a q x q block (W = 4,
// 2 or 1 as q allows): each shared-memory read of G or T1 feeds W
// accumulations, and the E entries it pairs with are broadcast across the
// warp.  nb blocks per CTA, each with its own G and T1 in shared memory.
template <class Ar, int W>
__global__ void k_wcontract_ar(int m, int q, double* __restrict__ X, int ldx, const double* __restrict__ E,
                               const double* __restrict__ E1, const int* __restrict__ live_ptr, bool sym) {
    using T = typename Ar::T;
    extern __shared__ __align__(16) unsigned char sh_raw[];
    T* sh = (T*)sh_raw;
    const int q2 = q * q;
    const int tpb = q * (q / W);  // threads per q x q block
    const int nb = max(1, (int)blockDim.x / tpb);
    T* sE = sh;
    T* sE1 = sE + q2;
    T* G = sE1 + q2;
    T* T1 = G + nb * q2;
    for (int e = threadIdx.x; e < q2; e += blockDim.x) {
        sE[e] = Ar::load(E[e]);
        sE1[e] = Ar::load(E1[e]);
    }
    const int live = min(*live_ptr, m);
    const long nblk = sym ? (long)live * (live + 1) / 2 : (long)live * live;
    const int jb = threadIdx.x / tpb;
    const int el = threadIdx.x - jb * tpb;
    const bool act = jb < nb;
    const int i = el % q, j0 = (el / q) * W;
    T* Gb = G + jb * q2;
    T* Tb = T1 + jb * q2;
    __syncthreads();
    for (long base = (long)blockIdx.x * nb; base < nblk; base += (long)gridDim.x * nb) {
        const long blk = base + jb;
        const bool ok = act && blk < nblk;
        size_t off = 0, offT = 0;
        int g = 0, gp = 0;
        if (ok) {
            wc_block(blk, live, sym, g, gp);
            off = (size_t)q * g + (size_t)ldx * ((size_t)q * gp);
            offT = (size_t)q * gp + (size_t)ldx * ((size_t)q * g);
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const int j = j0 + w;
                Gb[i + q * j] = Ar::mul(Ar::load(X[off + i + (size_t)ldx * j]), sE1[i + q * j]);
            }
        }
        __syncthreads();
        if (ok) {
            typename Ar::Acc c[W];
#pragma unroll
            for (int w = 0; w < W; ++w) c[w] = Ar::acc0();
            for (int k = 0; k < q; ++k) {
                const T gk = Gb[i + q * k];
#pragma unroll
                for (int w = 0; w < W; ++w) Ar::acc(c[w], gk, sE[k + q * (j0 + w)]);
            }
#pragma unroll
            for (int w = 0; w < W; ++w) Tb[i + q * (j0 + w)] = Ar::fin(c[w]);
        }
        __syncthreads();
        if (ok) {
            typename Ar::Acc c[W];
#pragma unroll
            for (int w = 0; w < W; ++w) c[w] = Ar::acc0();
            for (int k = 0; k < q; ++k) {
                const T ek = sE[i + q * k];
#pragma unroll
                for (int w = 0; w < W; ++w) Ar::acc(c[w], ek, Tb[k + q * (j0 + w)]);
            }
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const int j = j0 + w;
                const double v = Ar::store(Ar::mul(sE[i + q * j], Ar::fin(c[w])));
                X[off + i + (size_t)ldx * j] = v;
                if (sym && g != gp) X[offT + j + (size_t)ldx * i] = v;
            }
        }
        __syncthreads();
    }
}

}  // namespace

void wcontract_ar(cudaStream_t st, int arith, int m, int q, double* X, int ldx, const double* E, const double* E1,
                  const int* live, bool sym) {
    if (arith == 0) {
        wcontract_f64(st, m, q, X, ldx, E, E1, live, sym);
        return;
    }
    const int q2 = q * q;
    const int W = (q % 4 == 0) ? 4 : ((q % 2 == 0) ? 2 : 1);
    const int tpb = q * (q / W);
    int nb = tpb <= 256 ? 256 / tpb : 1;
    const int threads = ((nb * tpb + 31) / 32) * 32;
    long nblk = (long)m * m;
    long grid = (nblk + nb - 1) / nb;
    if (grid > 152 * 16) grid = 152 * 16;
    if (grid < 1) grid = 1;
    auto go = [&](auto ar, auto wt) {
        using A = decltype(ar);
        constexpr int WW = decltype(wt)::value;
        const size_t smem = (size_t)(2 * q2 + 2 * nb * q2) * sizeof(typename A::T);
        k_wcontract_ar<A, WW><<<(unsigned)grid, threads, smem, st>>>(m, q, X, ldx, E, E1, live, sym);
    };
    using W1 = std::integral_constant<int, 1>;
    using W2 = std::integral_constant<int, 2>;
    using W4 = std::integral_constant<int, 4>;
    if (arith == 1) {
        if (W == 4) go(ArF32{}, W4{});
        else if (W == 2) go(ArF32{}, W2{});
        else go(ArF32{}, W1{});
    } else {
        if (W == 4) go(ArDF{}, W4{});
        else if (W == 2) go(ArDF{}, W2{});
        else go(ArDF{}, W1{});
    }
}

int gemm_f64(cudaStream_t st, bool transA, bool transB, int M, int N, int K, double alpha,
             const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc,
             const double* scaleK, int splits, double* partial, int lowq) {
    if (M <= 0 || N <= 0) return 0;
    if (splits < 1 || K < 1) splits = 1;
    int kchunk = K < 1 ? BK : (K + splits - 1) / splits;
    kchunk = ((kchunk + BK - 1) / BK) * BK;
    splits = K < 1 ? 1 : (K + kchunk - 1) / kchunk;
    if (splits < 1) splits = 1;
    dim3 grid((M + BM - 1) / BM, (N + BN - 1) / BN, splits);
    dim3 block(256);
#define CTM_GEMM_LAUNCH(TA, TB)                                                                   \
    k_gemm_f64<TA, TB><<<grid, block, 0, st>>>(M, N, K, kchunk, alpha, A, lda, B, ldb, beta, C, \
                                               ldc, scaleK, partial, splits > 1 ? 0 : lowq)
    if (!transA && !transB) CTM_GEMM_LAUNCH(false, false);
    else if (!transA && transB) CTM_GEMM_LAUNCH(false, true);
    else if (transA && !transB) CTM_GEMM_LAUNCH(true, false);
    else CTM_GEMM_LAUNCH(true, true);
#undef CTM_GEMM_LAUNCH
    if (splits > 1) {
        size_t total = (size_t)M * N;
        int blocks = (int)((total + 255) / 256);
        if (blocks > 4096) blocks = 4096;
        k_splitk_reduce<<<blocks, 256, 0, st>>>(M, N, splits, partial, beta, C, ldc);
        return 2;
    }
    return 1;
}

void wcontract_f64(cudaStream_t st, int m, int q, double* X, int ldx, const double* E,
                   const double* E1, const int* live, bool sym) {
    int q2 = q * q;
    int threads = q2 <= 256 ? 256 : ((q2 + 31) / 32) * 32;
    int nb = threads / q2;
    if (nb < 1) nb = 1;
    size_t smem = (size_t)(2 * q2 + 2 * nb * q2) * sizeof(double);
    long nblk = (long)m * m;
    long grid = (nblk + nb - 1) / nb;
    if (grid > 152 * 16) grid = 152 * 16;
    if (grid < 1) grid = 1;
    k_wcontract<<<(unsigned)grid, threads, smem, st>>>(m, q, X, ldx, E, E1, live, sym);
}

}  // namespace ctm
