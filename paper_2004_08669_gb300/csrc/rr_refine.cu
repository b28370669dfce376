// rr_refine.cu -- Rayleigh-Ritz solve of a warm block by cluster-aware
// iterative refinement (mixed-precision forms).
//
// In the step's subspace iteration (the build's replacement of the dense
// diagonalisation in Algorithm 3) the Rayleigh-Ritz matrix H = V^t C~ V of a
// warm-started block is close to diagonal: its couplings are about the Ritz
// residual.  Cyclic Jacobi still needs ~5 sweeps of b - 1 dependent rounds
// each to bring every coupling below 2^-46.  This solver instead refines all
// eigenvectors at once (Ogita & Aishima, Japan J. Indust. Appl. Math. 35
// (2018) 1007, and their treatment of clustered eigenvalues, 36 (2019) 435):
// with X the current approximation (X = I at the start),
//   S = X^t H X,  R = I - X^t X,  lambda_i = S_ii / (X^t X)_ii,
//   c_ij = S_ij + R_ij (lambda_i + lambda_j) / 2
// (the coupling in the first-order orthonormalised basis).  Pairs with
// |c_ij| > tau |lambda_j - lambda_i| are strongly coupled; the connected
// components of those pairs are clusters, diagonalised exactly: T_c =
// (I + R_cc/2) S_cc (I + R_cc/2), T_c = Q_c Theta Q_c^t by a small Jacobi.
// Every other pair gets the first-order correction
//   E_ij = R_ij / 2 + c_ij / (lambda_j - lambda_i)   (E_ij = R_ij / 2 inside a
// cluster or when |c_ij| is below the Jacobi threshold), and
//   X <- X (I + E) Q,   Q = diag(Q_c).
// The iteration converges quadratically; couplings below eps sqrt|lambda_i
// lambda_j| (the Jacobi threshold, 2^-46) are not rotated, and it stops when
// every coupling is below 4 eps and |R| below 4 eps_r (the rounding floor of
// the recomputed products, a few 2^-46), or once the couplings, below 256 eps,
// stop falling.  All products are b x b x b in double-float arithmetic
// (pairs of FP32 words, about 48 significant bits) on the FP32 pipe, inside
// one cooperative launch with a grid barrier between phases.  If the
// refinement cannot proceed (a cluster above 32 states, too many strongly
// coupled pairs, no convergence within the iteration cap, non-finite values)
// it leaves ctl->rrc_ok = 0 and the Jacobi solver, launched behind it with a
// run-time skip flag, does the solve.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <mutex>

#include "ctm_internal.cuh"
#include "df_arith.cuh"
#include "eig_f64.cuh"

namespace ctm {
namespace {

constexpr int RT = 16;          // output tile edge of the b x b products
constexpr int RK = 64;          // K chunk staged in shared memory (two buffers)
constexpr int LDK = RK + 1;     // padded row of a staged chunk
constexpr int RMAXC = 32;       // largest cluster solved exactly
constexpr int RMAXN = 2048;     // largest b (shared-memory union-find)
constexpr int RTHREADS = 256;
constexpr int LDT = RMAXC + 1;  // leading dimension of the cluster matrices in shared memory

struct RrcP {
    int n, npad, max_iter, edge_cap;
    const double* H;
    int ldh;
    float2 *Hd, *X0, *X1, *W, *S, *G, *F, *Qc;
    double* lam;
    int *root, *cid, *cpos, *clist, *coff, *edges;
    float2* Sout;  // eigenvectors, npad x npad (the Jacobi solver's layout)
    double* diag;  // Ritz values (unsorted)
    DevCtl* ctl;
    double eps_c, eps_r, tau;
    int nhead;  // pairs with both indices >= nhead (guard vectors) are not rotated
};

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// block 0, thread 0: time since the refinement started, per phase
#define RRC_MARK(it_, ph_)                                                                          \
    do {                                                                                             \
        if (blockIdx.x == 0 && threadIdx.x == 0 && (it_) < 16)                                       \
            ctl->rrc_tph[(it_)][(ph_)] = (unsigned int)(gtimer() - ctl->rrc_t0);                     \
    } while (0)

__device__ __forceinline__ float2 ldf2(const float2* p) { return __ldcg(p); }
__device__ __forceinline__ void stf2(float2* p, float2 v) { __stcg(p, v); }

// Double-float accumulator of a dot product: the high parts summed by Knuth's
// two-sum, each product's rounding error (by FMA) and the cross terms of the
// low parts gathered in lo.
struct DAcc {
    float hi, lo;
};
__device__ __forceinline__ void dacc(DAcc& a, float2 x, float2 y) {
    const float p = x.x * y.x;
    const float e = fmaf(x.x, y.x, -p);
    const float s = a.hi + p;
    const float bb = s - a.hi;
    const float err = (a.hi - (s - bb)) + (p - bb);
    a.hi = s;
    a.lo += err + fmaf(x.x, y.y, fmaf(x.y, y.x, e));
}
__device__ __forceinline__ float2 dnorm(DAcc a) {
    const float h = a.hi + a.lo;
    return make_float2(h, a.lo - (h - a.hi));
}
__device__ __forceinline__ double df2d(float2 v) { return (double)v.x + (double)v.y; }

// Upper-triangular tile (I <= J) of an nt x nt tile grid from its index u.
__device__ __forceinline__ void upper_tile(int u, int nt, int& I, int& J) {
    I = 0;
    while (u >= nt - I) {
        u -= nt - I;
        ++I;
    }
    J = I + u;
}

// One 16 x 16 output tile of C = op(A) B (n x n, column-major, ld n, K = n):
// op(A)(i, k) = A[k + n i] when TA (A^t), else A[i + n k]; B(k, j) = B[k + n j].
// K runs in chunks of RK staged in shared memory (two buffers: the next
// chunk is loaded into registers while the current one is multiplied); each
// thread owns one output and sums its products in four interleaved
// double-float chains, combined at the end.
// lam_G (P2 only): the diagonal tile also writes lambda_i = C_ii / G_ii.
template <bool TA>
__device__ void df_tile(int n, int i0, int j0, const float2* A, const float2* B, float2* C, float2* sA,
                        float2* sB, const float2* lam_G, double* lam) {
    const int tid = threadIdx.x, ti = tid & (RT - 1), tj = tid / RT;
    constexpr int PER = RK * RT / RTHREADS;  // staged elements per thread and operand
    float2 ra[PER], rb[PER];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int e = tid + q * RTHREADS;
            int kk, ii;
            if (TA) {
                kk = e % RK;
                ii = e / RK;
            } else {
                ii = e % RT;
                kk = e / RT;
            }
            const int gi = i0 + ii, gk = k0 + kk;
            ra[q] = (gi < n && gk < n) ? (TA ? ldf2(A + gk + (size_t)n * gi) : ldf2(A + gi + (size_t)n * gk))
                                       : make_float2(0.f, 0.f);
            const int kb = e % RK, jj = e / RK;
            const int gj = j0 + jj, gkb = k0 + kb;
            rb[q] = (gj < n && gkb < n) ? ldf2(B + gkb + (size_t)n * gj) : make_float2(0.f, 0.f);
        }
    };
    // staged row-major with a padded row (LDK = RK + 1): the stores of
    // consecutive threads and the loads of a warp's 16 rows hit distinct banks
    auto stage = [&](float2* dA, float2* dB) {
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int e = tid + q * RTHREADS;
            int kk, ii;
            if (TA) {
                kk = e % RK;
                ii = e / RK;
            } else {
                ii = e % RT;
                kk = e / RT;
            }
            dA[ii * LDK + kk] = ra[q];
            dB[(e / RK) * LDK + e % RK] = rb[q];
        }
    };
    DAcc acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    const int nchunk = (n + RK - 1) / RK;
    fetch(0);
    stage(sA, sB);
    __syncthreads();
    for (int c = 0; c < nchunk; ++c) {
        const float2* cA = sA + (c & 1) * RT * LDK + ti * LDK;
        const float2* cB = sB + (c & 1) * RT * LDK + tj * LDK;
        if (c + 1 < nchunk) fetch((c + 1) * RK);
#pragma unroll
        for (int kk = 0; kk < RK; kk += 4) {
            dacc(acc[0], cA[kk], cB[kk]);
            dacc(acc[1], cA[kk + 1], cB[kk + 1]);
            dacc(acc[2], cA[kk + 2], cB[kk + 2]);
            dacc(acc[3], cA[kk + 3], cB[kk + 3]);
        }
        if (c + 1 < nchunk) stage(sA + ((c + 1) & 1) * RT * LDK, sB + ((c + 1) & 1) * RT * LDK);
        __syncthreads();
    }
    // (a0 + a1) + (a2 + a3) in double-float
    float2 v = JDF::add(JDF::add(dnorm(acc[0]), dnorm(acc[1])), JDF::add(dnorm(acc[2]), dnorm(acc[3])));
    const int gi = i0 + ti, gj = j0 + tj;
    if (gi < n && gj < n) {
        stf2(C + gi + (size_t)n * gj, v);
        if (lam && gi == gj) lam[gi] = df2d(v) / df2d(ldf2(lam_G + gi + (size_t)n * gi));
    }
}

// Float max over the block, then a global atomicMax on its bits (non-negative).
__device__ void block_max_to(float v, unsigned int* dst, float* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < RTHREADS / 32 ? red[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0 && v > 0.f) atomicMax(dst, __float_as_uint(v));
    }
    __syncthreads();
}

// E_ik of the update (double-float): R_ik / 2 plus, for pairs in different
// clusters whose coupling is above the Jacobi threshold, c_ik / (lambda_k -
// lambda_i).  S and G are stored in their upper triangles.
__device__ float2 e_entry(const RrcP& p, int i, int k) {
    const int n = p.n;
    const int a = min(i, k), b = max(i, k);
    const float2 g = ldf2(p.G + a + (size_t)n * b);
    if (i == k) return JDF::half(JDF::add(JDF::one(), JDF::neg(g)));
    const float2 rh = JDF::half(JDF::neg(g));
    if (a >= p.nhead) return rh;  // two guard vectors: orthonormality only
    const int ci = __ldcg(p.cid + i), ck = __ldcg(p.cid + k);
    if (ci >= 0 && ci == ck) return rh;
    const double li = __ldcg(p.lam + i), lk = __ldcg(p.lam + k);
    const double c = df2d(ldf2(p.S + a + (size_t)n * b)) - df2d(g) * 0.5 * (li + lk);
    const float sc = sqrtf(fabsf((float)li) * fabsf((float)lk));
    // a coupling already within the convergence threshold is not rotated:
    // between (nearly) degenerate Ritz values it is rounding over rounding,
    // and rotating by it would feed the orthonormality defect every iteration
    if (!(fabsf((float)c) > 4.0f * (float)p.eps_c * sc)) return rh;
    return JDF::add(rh, JDF::from(c / (lk - li)));
}

// Exact eigendecomposition of one cluster's block by cyclic Jacobi (round-
// robin parallel order) in shared memory, double-float; then the cluster's
// columns of F.  T, T2, V, V2: LDT x RMAXC float2 each.
__device__ void solve_cluster(const RrcP& p, int c, float2* T, float2* T2, float2* V, float2* V2, float2* al,
                              float2* be, int* partner) {
    const int n = p.n, tid = threadIdx.x;
    const int off = __ldcg(p.coff + c), s = __ldcg(p.coff + c + 1) - off;
    const int s2 = s + (s & 1);
    const int* mem = p.clist + off;
    // M = I + R_cc / 2 (R = I - G) into V2 (scratch), S_cc into T2
    for (int e = tid; e < s2 * s2; e += RTHREADS) {
        const int a = e % s2, b = e / s2;
        float2 mv = (a == b) ? JDF::one() : JDF::zero(), sv = JDF::zero();
        if (a < s && b < s) {
            const int ia = __ldcg(mem + a), ib = __ldcg(mem + b);
            const int lo = min(ia, ib), hi = max(ia, ib);
            const float2 g = ldf2(p.G + lo + (size_t)n * hi);
            // M = I + (I - G) / 2
            mv = (a != b) ? JDF::half(JDF::neg(g)) : JDF::add(JDF::one(), JDF::half(JDF::add(JDF::one(), JDF::neg(g))));
            sv = ldf2(p.S + lo + (size_t)n * hi);
        }
        V2[a + LDT * b] = mv;
        T2[a + LDT * b] = sv;
    }
    __syncthreads();
    // T = M S M: first U = S M into T, then M U into V (then swapped)
    for (int e = tid; e < s2 * s2; e += RTHREADS) {
        const int a = e % s2, b = e / s2;
        DAcc acc{0.f, 0.f};
        for (int k = 0; k < s2; ++k) dacc(acc, T2[a + LDT * k], V2[k + LDT * b]);
        T[a + LDT * b] = dnorm(acc);
    }
    __syncthreads();
    for (int e = tid; e < s2 * s2; e += RTHREADS) {
        const int a = e % s2, b = e / s2;
        DAcc acc{0.f, 0.f};
        for (int k = 0; k < s2; ++k) dacc(acc, V2[a + LDT * k], T[k + LDT * b]);
        V[a + LDT * b] = dnorm(acc);
    }
    __syncthreads();
    for (int e = tid; e < s2 * s2; e += RTHREADS) {
        const int a = e % s2, b = e / s2;
        // symmetrise; the padding index (odd s) stays zero
        const float2 t = JDF::half(JDF::add(V[a + LDT * b], V[b + LDT * a]));
        T[a + LDT * b] = (a < s && b < s) ? t : JDF::zero();
    }
    __syncthreads();
    for (int e = tid; e < s2 * s2; e += RTHREADS) {
        const int a = e % s2, b = e / s2;
        V[a + LDT * b] = (a == b) ? JDF::one() : JDF::zero();
    }
    __syncthreads();
    const double eps = p.eps_c;
    for (int sweep = 0; sweep < 24; ++sweep) {
        int any = 0;
        for (int e = tid; e < s2 * s2; e += RTHREADS) {
            const int a = e % s2, b = e / s2;
            if (a < b && JDF::above(T[a + LDT * a], T[b + LDT * b], T[a + LDT * b], eps, 0.0)) any = 1;
        }
        if (!__syncthreads_or(any)) break;
        for (int r = 0; r < s2 - 1; ++r) {
            if (tid < s2 / 2) {
                int pp, qq;
                rr_pair(r, tid, s2, pp, qq);
                const JDF::R R = JDF::rot(T[pp + LDT * pp], T[qq + LDT * qq], T[pp + LDT * qq], eps, 0.0);
                partner[pp] = qq;
                partner[qq] = pp;
                // v_p' = c v_p - s v_q, v_q' = s v_p + c v_q
                al[pp] = R.on ? R.c : JDF::one();
                be[pp] = R.on ? JDF::neg(R.s) : JDF::zero();
                al[qq] = R.on ? R.c : JDF::one();
                be[qq] = R.on ? R.s : JDF::zero();
            }
            __syncthreads();
            // rows: U_kj = al_k T_kj + be_k T_{pi(k) j}; V' = V J
            for (int e = tid; e < s2 * s2; e += RTHREADS) {
                const int a = e % s2, b = e / s2;
                const int pa = partner[a], pb = partner[b];
                T2[a + LDT * b] = JDF::lin(al[a], T[a + LDT * b], JDF::neg(be[a]), T[pa + LDT * b]);
                V2[a + LDT * b] = JDF::lin(al[b], V[a + LDT * b], JDF::neg(be[b]), V[a + LDT * pb]);
            }
            __syncthreads();
            // columns, upper triangle written to both halves (T stays symmetric)
            for (int e = tid; e < s2 * s2; e += RTHREADS) {
                const int a = e % s2, b = e / s2;
                if (a <= b) {
                    const int pb = partner[b];
                    const float2 t = JDF::lin(al[b], T2[a + LDT * b], JDF::neg(be[b]), T2[a + LDT * pb]);
                    T[a + LDT * b] = t;
                    T[b + LDT * a] = t;
                }
                V[a + LDT * b] = V2[a + LDT * b];
            }
            __syncthreads();
        }
    }
    // Q_c (column b: s entries); F's cluster columns are multiplied by it
    // after every column of F = I + E is in place (apply_cluster)
    for (int e = tid; e < s * s; e += RTHREADS) {
        const int a = e % s, b = e / s;
        stf2(p.Qc + (size_t)RMAXC * (off + b) + a, V[a + LDT * b]);
    }
}

// F[:, c] <- F[:, c] Q_c for one cluster, in chunks of 32 rows staged in
// shared memory (each chunk is read whole before it is overwritten).
__device__ void apply_cluster(const RrcP& p, int c, float2* Fs, float2* Qs) {
    const int n = p.n, tid = threadIdx.x;
    const int off = __ldcg(p.coff + c), s = __ldcg(p.coff + c + 1) - off;
    const int* mem = p.clist + off;
    for (int e = tid; e < s * s; e += RTHREADS) {
        const int a = e % s, b = e / s;
        Qs[a + LDT * b] = ldf2(p.Qc + (size_t)RMAXC * (off + b) + a);
    }
    for (int r0 = 0; r0 < n; r0 += 32) {
        __syncthreads();
        for (int e = tid; e < 32 * s; e += RTHREADS) {
            const int ii = e % 32, a = e / 32, i = r0 + ii;
            Fs[ii + LDT * a] = i < n ? ldf2(p.F + i + (size_t)n * __ldcg(mem + a)) : JDF::zero();
        }
        __syncthreads();
        for (int e = tid; e < 32 * s; e += RTHREADS) {
            const int ii = e % 32, b = e / 32, i = r0 + ii;
            if (i >= n) continue;
            DAcc acc{0.f, 0.f};
            for (int a = 0; a < s; ++a) dacc(acc, Fs[ii + LDT * a], Qs[a + LDT * b]);
            stf2(p.F + i + (size_t)n * __ldcg(mem + b), dnorm(acc));
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(RTHREADS, 3) k_rr_refine(RrcP p) {
    extern __shared__ float4 rsm4[];
    float2* sm = reinterpret_cast<float2*>(rsm4);
    __shared__ float red[RTHREADS / 32];
    __shared__ int s_wsum[2 * (RTHREADS / 32)];
    __shared__ int s_flag[4];
    const int n = p.n, tid = threadIdx.x;
    const int nt = (n + RT - 1) / RT;
    const int ntU = nt * (nt + 1) / 2;
    DevCtl* ctl = p.ctl;
    int* err = &ctl->jac_status;
    unsigned int epoch = 0;
    float2* sA = sm;                // two RT x LDK buffers
    float2* sB = sm + 2 * RT * LDK;  // two RT x LDK buffers

    // H (symmetrised) into double-float; X = I
    for (long e = blockIdx.x * (long)RTHREADS + tid; e < (long)n * n; e += (long)gridDim.x * RTHREADS) {
        const int i = (int)(e % n), j = (int)(e / n);
        const double h = 0.5 * (p.H[i + (size_t)p.ldh * j] + p.H[j + (size_t)p.ldh * i]);
        stf2(p.Hd + e, JDF::from(h));
        stf2(p.X0 + e, i == j ? JDF::one() : JDF::zero());
    }
    if (blockIdx.x == 0 && tid == 0) {
        ctl->rrc_t0 = gtimer();
        ctl->rrc_ok = 0;
        ctl->rrc_fail = 0;
        ctl->rrc_done = 0;
        ctl->rrc_iters = 0;
        ctl->rrc_maxcl = 0;
    }
    if (!grid_sync(&ctl->bar_count, epoch, err)) return;
    float2* X = p.X0;
    float2* Xn = p.X1;
    float mc_prev = INFINITY;  // block 0, thread 0: the previous iteration's largest coupling
    int it = 0;
    bool done = false;
    for (it = 0; it <= p.max_iter; ++it) {
        if (blockIdx.x == 0 && tid == 0) {
            ctl->rrc_nedges = 0;
            ctl->rrc_maxc = 0u;
            ctl->rrc_maxr = 0u;
        }
        // P1: W = H X (all tiles), G = X^t X (upper tiles); with X = I
        // (first iteration) S = H and G = I are taken directly
        if (it == 0) {
            for (long e = blockIdx.x * (long)RTHREADS + tid; e < (long)n * n; e += (long)gridDim.x * RTHREADS) {
                const int i = (int)(e % n), j = (int)(e / n);
                const float2 h = ldf2(p.Hd + e);
                stf2(p.S + e, h);
                stf2(p.G + e, i == j ? JDF::one() : JDF::zero());
                if (i == j) p.lam[i] = df2d(h);
            }
        }
        for (int u = blockIdx.x; it > 0 && u < nt * nt; u += gridDim.x)
            df_tile<false>(n, RT * (u % nt), RT * (u / nt), p.Hd, X, p.W, sA, sB, nullptr, nullptr);
        if (!grid_sync(&ctl->bar_count, epoch, err)) return;
        RRC_MARK(it, 0);
        // P2: S = X^t W and G = X^t X (upper tiles, one item each)
        for (int u = blockIdx.x; it > 0 && u < 2 * ntU; u += gridDim.x) {
            int I, J;
            upper_tile(u % ntU, nt, I, J);
            if (u < ntU) df_tile<true>(n, RT * I, RT * J, X, p.W, p.S, sA, sB, nullptr, nullptr);
            else df_tile<true>(n, RT * I, RT * J, X, X, p.G, sA, sB, nullptr, nullptr);
        }
        if (!grid_sync(&ctl->bar_count, epoch, err)) return;
        RRC_MARK(it, 1);
        // P3a: couplings, orthonormality defect, strongly coupled pairs
        {
            float mc = 0.f, mr = 0.f;
            for (long e = blockIdx.x * (long)RTHREADS + tid; e < (long)n * n; e += (long)gridDim.x * RTHREADS) {
                const int i = (int)(e % n), j = (int)(e / n);
                if (i > j) continue;
                const double g = df2d(ldf2(p.G + e));
                if (i == j) {
                    mr = fmaxf(mr, fabsf((float)(1.0 - g)));
                    if (it > 0) p.lam[i] = df2d(ldf2(p.S + e)) / g;  // for the update phase
                    continue;
                }
                mr = fmaxf(mr, fabsf((float)g));
                // A pair of guard vectors (both beyond the head) needs no
                // rotation: a rotation within their span leaves the head's
                // eigenvectors and span(X) unchanged, and their couplings,
                // relative to their small Ritz values, sit far above the
                // noise floor the head converges to.
                if (i >= p.nhead) continue;
                // Rayleigh quotients lambda = S_ii / G_ii (the first iteration: H_ii)
                const size_t di = (size_t)i * (n + 1), dj = (size_t)j * (n + 1);
                const double li = it > 0 ? df2d(ldf2(p.S + di)) / df2d(ldf2(p.G + di)) : __ldcg(p.lam + i);
                const double lj = it > 0 ? df2d(ldf2(p.S + dj)) / df2d(ldf2(p.G + dj)) : __ldcg(p.lam + j);
                const double c = df2d(ldf2(p.S + e)) - g * 0.5 * (li + lj);
                const float sc = sqrtf(fabsf((float)li) * fabsf((float)lj));
                const float ac = fabsf((float)c);
                const float ratio = sc > 0.f ? ac / sc : (ac > 0.f ? INFINITY : 0.f);
                if (!(ratio == ratio)) mc = INFINITY;  // NaN
                mc = fmaxf(mc, ratio);
                if (ratio > 4.0f * (float)p.eps_c && ac > (float)p.tau * fabsf((float)(lj - li))) {
                    const int k = atomicAdd(&ctl->rrc_nedges, 1);
                    if (k < p.edge_cap) {
                        p.edges[2 * k] = i;
                        p.edges[2 * k + 1] = j;
                    }
                }
            }
            if (!(mc == mc)) mc = INFINITY;
            block_max_to(mc, &ctl->rrc_maxc, red);
            block_max_to(mr, &ctl->rrc_maxr, red);
        }
        if (!grid_sync(&ctl->bar_count, epoch, err)) return;
        RRC_MARK(it, 2);
        // P3b (block 0): convergence, failure, clusters by union-find
        if (blockIdx.x == 0) {
            int* parent = reinterpret_cast<int*>(sm);
            int* cnt = parent + RMAXN;
            int* cidr = cnt + RMAXN;
            int* rootS = cidr + RMAXN;
            int* coffS = rootS + RMAXN;  // RMAXN / 2 + 1 cluster offsets
            if (tid == 0) {
                const float mc = __uint_as_float(*(volatile unsigned int*)&ctl->rrc_maxc);
                const float mr = __uint_as_float(*(volatile unsigned int*)&ctl->rrc_maxr);
                const int ne = *(volatile int*)&ctl->rrc_nedges;
                int flag = 0;  // 0 continue, 1 done, 2 fail
                int why = 0;
                if (!(mc < INFINITY) || !(mr < INFINITY)) {
                    flag = 2;
                    why = 4;
                } else if ((mc <= 4.0f * (float)p.eps_c && mr <= 4.0f * (float)p.eps_r) ||
                           (mc <= 256.0f * (float)p.eps_c && mr <= 16.0f * (float)p.eps_r && mc > 0.5f * mc_prev)) {
                    // couplings at the rounding floor of the double-float
                    // products (a few 2^-46 of sqrt|lambda_i lambda_j|), or no
                    // longer falling there: the refinement has converged
                    flag = 1;
                } else if (it == p.max_iter) {
                    flag = 2;
                    why = 3;
                } else if (ne > p.edge_cap) {
                    flag = 2;
                    why = 1;
                }
                mc_prev = mc;
                s_flag[0] = flag;
                s_flag[1] = why;
                s_flag[2] = min(ne, p.edge_cap);
                s_flag[3] = 0;
                ctl->rrc_iters = it + 1;
                if (it < 16) {
                    ctl->rrc_hist_c[it] = mc;
                    ctl->rrc_hist_r[it] = mr;
                    ctl->rrc_hist_ne[it] = ne;
                    ctl->rrc_hist_cl[it] = 0;
                }
            }
            __syncthreads();
            if (s_flag[0] == 0) {
                const int ne = s_flag[2];
                for (int i = tid; i < n; i += RTHREADS) {
                    parent[i] = i;
                    cnt[i] = 0;
                }
                __syncthreads();
                // lock-free union: hook the larger root under the smaller
                for (int e = tid; e < ne; e += RTHREADS) {
                    int u = __ldcg(p.edges + 2 * e), v = __ldcg(p.edges + 2 * e + 1);
                    for (int guard = 0; guard < 4 * RMAXN; ++guard) {
                        while (true) {
                            const int pu = *(volatile int*)&parent[u];
                            if (pu == u) break;
                            u = pu;
                        }
                        while (true) {
                            const int pv = *(volatile int*)&parent[v];
                            if (pv == v) break;
                            v = pv;
                        }
                        if (u == v) break;
                        if (u > v) {
                            const int t = u;
                            u = v;
                            v = t;
                        }
                        if (atomicCAS(&parent[v], v, u) == v) break;
                    }
                }
                __syncthreads();
                for (int i = tid; i < n; i += RTHREADS) {
                    int r = i;
                    for (int guard = 0; guard < RMAXN && parent[r] != r; ++guard) r = parent[r];
                    rootS[i] = r;
                    p.root[i] = r;
                    atomicAdd(&cnt[r], 1);
                }
                __syncthreads();
                // clusters numbered by their smallest member (the root):
                // an exclusive scan over the roots of clusters and of their
                // sizes, 8 consecutive indices per thread
                {
                    int* wsum = s_wsum;  // per-warp totals (clusters, members)
                    const int base = tid * 8;
                    int nc = 0, ns = 0, mx = 0;
                    for (int k = 0; k < 8; ++k) {
                        const int r = base + k;
                        if (r < n && cnt[r] > 1) {
                            ++nc;
                            ns += cnt[r];
                            mx = max(mx, cnt[r]);
                        }
                    }
                    int ic = nc, is = ns;
                    for (int o = 1; o < 32; o <<= 1) {
                        const int tc = __shfl_up_sync(0xffffffffu, ic, o), ts = __shfl_up_sync(0xffffffffu, is, o);
                        if ((tid & 31) >= o) {
                            ic += tc;
                            is += ts;
                        }
                    }
                    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                    if ((tid & 31) == 31) {
                        wsum[2 * (tid >> 5)] = ic;
                        wsum[2 * (tid >> 5) + 1] = is;
                    }
                    if ((tid & 31) == 0) atomicMax(&s_flag[3], mx);
                    __syncthreads();
                    int pc = 0, ps = 0;
                    for (int w = 0; w < (tid >> 5); ++w) {
                        pc += wsum[2 * w];
                        ps += wsum[2 * w + 1];
                    }
                    int cc = pc + ic - nc, ss = ps + is - ns;  // exclusive prefix of this thread
                    for (int k = 0; k < 8; ++k) {
                        const int r = base + k;
                        if (r >= n) break;
                        if (cnt[r] > 1) {
                            cidr[r] = cc;
                            coffS[cc] = ss;
                            p.coff[cc] = ss;
                            ++cc;
                            ss += cnt[r];
                        } else {
                            cidr[r] = -1;
                        }
                    }
                    if (tid == RTHREADS - 1) {
                        p.coff[cc] = ss;  // the last thread's end is the total
                        ctl->rrc_ncl = cc;
                    }
                    __syncthreads();
                    if (tid == 0) {
                        const int mxc = s_flag[3];
                        if (it < 16) ctl->rrc_hist_cl[it] = mxc;
                        ctl->rrc_maxcl = max(ctl->rrc_maxcl, mxc);
                        if (mxc > RMAXC) {
                            s_flag[0] = 2;
                            s_flag[1] = 2;
                        }
                    }
                    __syncthreads();
                }
                // members in ascending order within each cluster (deterministic)
                for (int i = tid; i < n; i += RTHREADS) {
                    const int r = rootS[i];
                    const int c = cidr[r];
                    p.cid[i] = c;
                    if (c >= 0) {
                        int pos = 0;
                        for (int j = 0; j < i; ++j) pos += (rootS[j] == r);
                        p.cpos[i] = pos;
                        p.clist[coffS[c] + pos] = i;
                    } else {
                        p.cpos[i] = 0;
                    }
                }
            }
            __syncthreads();
            if (tid == 0) {
                if (s_flag[0] == 2) ctl->rrc_fail = s_flag[1];
                ctl->rrc_done = s_flag[0];
            }
        }
        if (!grid_sync(&ctl->bar_count, epoch, err)) return;
        RRC_MARK(it, 3);
        const int state = *(volatile int*)&ctl->rrc_done;
        if (state == 2) return;  // the Jacobi solver behind this launch takes over
        if (state == 1) {
            done = true;
            break;
        }
        // P3c/d: clusters' rotations and F's columns in them; F = I + E elsewhere
        {
            const int ncl = *(volatile int*)&ctl->rrc_ncl;
            float2* T = sm;
            float2* T2 = T + LDT * RMAXC;
            float2* V = T2 + LDT * RMAXC;
            float2* V2 = V + LDT * RMAXC;
            float2* al = V2 + LDT * RMAXC;
            float2* be = al + RMAXC;
            int* partner = reinterpret_cast<int*>(be + RMAXC);
            // the clusters' Jacobi solves take the last blocks of the grid,
            // the other blocks form F = I + E (every column) meanwhile
            const int nsolve = ncl > 0 ? max(1, min(ncl, (int)gridDim.x / 2)) : 0;
            const int first = (int)gridDim.x - nsolve;
            const int fblocks = max(first, 1);  // a grid of one block does both, in turn
            if ((int)blockIdx.x >= first) {
                for (int c = blockIdx.x - first; c < ncl; c += nsolve) {
                    solve_cluster(p, c, T, T2, V, V2, al, be, partner);
                    __syncthreads();
                }
            }
            if ((int)blockIdx.x < fblocks) {
                for (long e = blockIdx.x * (long)RTHREADS + tid; e < (long)n * n; e += (long)fblocks * RTHREADS) {
                    const int i = (int)(e % n), j = (int)(e / n);
                    float2 f = e_entry(p, i, j);
                    if (i == j) f = JDF::add(f, JDF::one());
                    stf2(p.F + e, f);
                }
            }
            if (ncl > 0) {
                if (!grid_sync(&ctl->bar_count, epoch, err)) return;
                RRC_MARK(it, 4);
                for (int c = blockIdx.x; c < ncl; c += gridDim.x) apply_cluster(p, c, T, V);
            }
        }
        if (!grid_sync(&ctl->bar_count, epoch, err)) return;
        RRC_MARK(it, 5);
        // P4: X <- X F
        for (int u = blockIdx.x; u < nt * nt; u += gridDim.x)
            df_tile<false>(n, RT * (u % nt), RT * (u / nt), X, p.F, Xn, sA, sB, nullptr, nullptr);
        if (!grid_sync(&ctl->bar_count, epoch, err)) return;
        RRC_MARK(it, 6);
        float2* t = X;
        X = Xn;
        Xn = t;
    }
    if (!done) return;
    // eigenvectors and Ritz values where the Jacobi solver leaves them
    for (long e = blockIdx.x * (long)RTHREADS + tid; e < (long)n * n; e += (long)gridDim.x * RTHREADS) {
        const int i = (int)(e % n), j = (int)(e / n);
        stf2(p.Sout + i + (size_t)p.npad * j, ldf2(X + e));
    }
    for (int i = blockIdx.x * RTHREADS + tid; i < n; i += gridDim.x * RTHREADS) p.diag[i] = __ldcg(p.lam + i);
    if (blockIdx.x == 0 && tid == 0) {
        ctl->rrc_ok = 1;
        ctl->jac_sweeps = 0;
    }
}

size_t smem_bytes() {
    const size_t gemm = 4 * (size_t)LDK * RT * sizeof(float2);
    const size_t uf = (4 * (size_t)RMAXN + RMAXN / 2 + 1) * sizeof(int);
    const size_t cl = 4 * (size_t)LDT * RMAXC * sizeof(float2) + 2 * RMAXC * sizeof(float2) + RMAXC * sizeof(int);
    return std::max(gemm, std::max(uf, cl));
}

cudaError_t launch_coop_rrc(const void* fn, int grid, void** args, size_t smem, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(RTHREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace

size_t rrc_workspace_bytes(int n) {
    const size_t nn = (size_t)n * n;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    return 7 * al(nn * sizeof(float2)) + al((size_t)RMAXC * n * sizeof(float2)) + al(n * sizeof(double)) +
           4 * al(n * sizeof(int)) + al((n + 1) * sizeof(int)) + al(2 * (size_t)8 * n * sizeof(int));
}

void rrc_carve(void* base, int n, RrcWork& w) {
    const size_t nn = (size_t)n * n;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    char* c = (char*)base;
    auto take = [&](size_t bytes) {
        char* r = c;
        c += al(bytes);
        return r;
    };
    w.Hd = (float2*)take(nn * sizeof(float2));
    w.X0 = (float2*)take(nn * sizeof(float2));
    w.X1 = (float2*)take(nn * sizeof(float2));
    w.W = (float2*)take(nn * sizeof(float2));
    w.S = (float2*)take(nn * sizeof(float2));
    w.G = (float2*)take(nn * sizeof(float2));
    w.F = (float2*)take(nn * sizeof(float2));
    w.Qc = (float2*)take((size_t)RMAXC * n * sizeof(float2));
    w.lam = (double*)take(n * sizeof(double));
    w.root = (int*)take(n * sizeof(int));
    w.cid = (int*)take(n * sizeof(int));
    w.cpos = (int*)take(n * sizeof(int));
    w.clist = (int*)take(n * sizeof(int));
    w.coff = (int*)take((n + 1) * sizeof(int));
    w.edge_cap = 8 * n;
    w.edges = (int*)take(2 * (size_t)w.edge_cap * sizeof(int));
    w.nmax = n;
}

bool rrc_supported(int n) { return n >= 2 && n <= RMAXN; }

cudaError_t rr_cluster_refine(cudaStream_t st, int n, const double* H, int ldh, RrcWork& w, EigWork& ew,
                              DevCtl* ctl, int max_iter, int nhead) {
    if (!rrc_supported(n) || n > w.nmax) return cudaErrorInvalidValue;
    const size_t smem = smem_bytes();
    static std::mutex mu;
    static int limit = 0;
    {
        std::lock_guard<std::mutex> g(mu);
        if (limit == 0) {
            cudaFuncSetAttribute((const void*)k_rr_refine, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            limit = coop_grid_limit((const void*)k_rr_refine, RTHREADS, smem);
        }
    }
    int grid = std::min(limit, 3 * 152);
    const int nt = (n + RT - 1) / RT;
    grid = std::min(grid, std::max(nt * nt, nt * (nt + 1)));  // one round of P1 (W) and of P2 (S and G)
    if (grid < 1) grid = 1;
    RrcP p{};
    p.n = n;
    p.npad = n + (n & 1) < 2 ? 2 : n + (n & 1);
    p.max_iter = max_iter;
    p.nhead = (nhead > 0 && nhead < n) ? nhead : n;
    p.edge_cap = w.edge_cap;
    p.H = H;
    p.ldh = ldh;
    p.Hd = w.Hd;
    p.X0 = w.X0;
    p.X1 = w.X1;
    p.W = w.W;
    p.S = w.S;
    p.G = w.G;
    p.F = w.F;
    p.Qc = w.Qc;
    p.lam = w.lam;
    p.root = w.root;
    p.cid = w.cid;
    p.cpos = w.cpos;
    p.clist = w.clist;
    p.coff = w.coff;
    p.edges = w.edges;
    p.Sout = (float2*)ew.S;
    p.diag = ew.diag;
    p.ctl = ctl;
    p.eps_c = 1.4210854715202004e-14;  // 2^-46, the double-float Jacobi threshold
    p.eps_r = 5.6843418860808015e-14;  // 2^-44
    p.tau = 0.3;
    cudaMemsetAsync(&ctl->bar_count, 0, sizeof(unsigned int), st);
    cudaMemsetAsync(&ctl->jac_status, 0, sizeof(int), st);
    void* args[] = {&p};
    return launch_coop_rrc((const void*)k_rr_refine, grid, args, smem, st);
}

}  // namespace ctm
