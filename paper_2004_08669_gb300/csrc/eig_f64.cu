// eig_f64.cu -- FP64 kernels of the leading-eigenpair stage of a CTMRG step.
//
// The paper diagonalises the whole extended corner (Algorithm 3, the
// EigenExa call, with a dense solver).  Here only its leading b = m + p
// eigenpairs are computed, by block subspace iteration:
//   Y = C~ V;  H = V^t Y;  H = S Theta S^t (cyclic Jacobi, FP64);
//   Z = V S;  T = Y S;  residual ||T_i - theta_i Z_i||;
//   V <- orth([T_i / theta_i or Z_i]) by (shifted) Cholesky QR.
// The kernels below are the small dense FP64 pieces: a parallel-order
// two-sided Jacobi eigensolver (Golub & Van Loan 8.5, round-robin ordering)
// for cold starts, simultaneous Jacobi rotations for warm starts (end of
// file), a blocked Cholesky factorisation, a triangular inverse, the
// residual test with the multiplet-aware truncation rule, and the gauge
// alignment of Ritz vectors to the previous step's (sign per singlet,
// orthogonal Procrustes per doublet) that keeps the renormalised basis
// consistent between steps.
#include "ctm_internal.cuh"
#include "eig_f64.cuh"
#include "df_arith.cuh"

#include <math.h>

#include <algorithm>
#include <mutex>

namespace ctm {

namespace {


template <class JA>
__global__ void k_jacobi_init(int n, int npad, const double* __restrict__ H, int ldh,
                              typename JA::T* __restrict__ A0, typename JA::T* __restrict__ S,
                              int* __restrict__ act, const int* __restrict__ skip) {
    if (skip && *skip) return;  // another solver already produced S and diag
    size_t tot = (size_t)npad * npad;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot;
         e += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(e % npad), j = (int)(e / npad);
        if (j == 0) act[i] = 0;
        double v = 0.0;
        if (i < n && j < n) v = 0.5 * (H[i + (size_t)ldh * j] + H[j + (size_t)ldh * i]);
        A0[e] = JA::from(v);
        S[e] = (i == j) ? JA::one() : JA::zero();
    }
}

// Pair k of round r of the tournament over the first s2 entries of perm, or
// one of the fixed (never rotated) pairs of the entries beyond s2.
__device__ __forceinline__ void jac_pair(int r, int k, int s2, const int* perm, int& p, int& q) {
    const int nh = s2 >> 1;
    if (k < nh) {
        int a, b;
        rr_pair(r, k, s2, a, b);
        p = perm[a];
        q = perm[b];
    } else {
        p = perm[s2 + 2 * (k - nh)];
        q = perm[s2 + 2 * (k - nh) + 1];
    }
}

constexpr int JT = 8;        // pairs per side of an A unit (JT x JT 2x2 blocks)
constexpr int JS_ROWS = 32;  // rows of S per pass of an S unit (JT pairs x JS_ROWS rows)
constexpr int JS_PASS = 2;   // passes per S unit: each thread owns JS_PASS rows, JS_ROWS apart

// The pair of index x in round r of the tournament over the first s2 entries
// of perm (inv: positions in perm): its partner y, the pair's slot k (as in
// jac_pair; k >= s2 / 2 is a fixed pair that is never rotated) and whether x
// is the pair's first index p.
struct JPartner {
    int y, k;
    bool isp;
};
__device__ __forceinline__ JPartner jac_partner(int r, int x, int s2, const int* perm, const int* inv) {
    const int a = inv[x];
    if (a >= s2) {
        const int o = a - s2;
        return JPartner{perm[s2 + (o ^ 1)], (s2 >> 1) + (o >> 1), (o & 1) == 0};
    }
    const int n1 = s2 - 1;
    if (a == n1) return JPartner{perm[r], 0, true};
    if (a == r) return JPartner{perm[n1], 0, false};
    int d = a - r;
    if (d < 0) d += n1;
    if (d <= (n1 - 1) / 2) {  // a = r + d: x is p of pair d, q sits at r - d
        int b = r - d;
        if (b < 0) b += n1;
        return JPartner{perm[b], d, true};
    }
    const int k = n1 - d;  // a = r - k: x is q of pair k, p sits at r + k
    int b = r + k;
    if (b >= n1) b -= n1;
    return JPartner{perm[b], k, false};
}

// alpha u + beta v
template <class JA>
__device__ __forceinline__ typename JA::T jcomb(typename JA::T al, typename JA::T u, typename JA::T be,
                                                typename JA::T v) {
    return JA::lin(al, u, JA::neg(be), v);
}

// Entry (x, y) of J^t A J for one round, J acting on x as x' = ax x + bx pi(x)
// (and likewise on y): from A[x][y], A[x][pi y], A[pi x][y], A[pi x][pi y].
template <class JA>
__device__ __forceinline__ typename JA::T jprime(typename JA::T ax, typename JA::T bx, typename JA::T ay,
                                                 typename JA::T by, typename JA::T a_xy, typename JA::T a_xpy,
                                                 typename JA::T a_pxy, typename JA::T a_pxpy) {
    return jcomb<JA>(ay, jcomb<JA>(ax, a_xy, bx, a_pxy), by, jcomb<JA>(ax, a_xpy, bx, a_pxpy));
}

// Two consecutive rounds r, r + 1 of the tournament between two grid
// barriers.  Each output entry of round r + 1, A''[x][y] with x, y in the
// round's pairs, is a combination of the 2 x 2 block of A' (the state after
// round r) on those pairs, and each entry of A' one of a 2 x 2 block of A
// on the round-r partners: 16 reads of A per 2 x 2 output block instead of 4.
// A unit recomputes the round-r rotations of all indices in its pairs and the
// round-(r + 1) rotations of its pairs (whose inputs, the diagonal blocks of
// A', it forms from A the same way), so one barrier, one round of reads and
// two rotation chains replace two of each.  S reads the four columns of the
// round-r partners and writes the other buffer.
// Thread roles in an A unit (JT x JT tile of round-(r + 1) pair blocks):
//   [0, 2 JT^2)             one row of a 2 x 2 output block each (its row of
//                           A' goes through shared memory to the other row);
//   [2 JT^2, 2 JT^2 + 4 JT) the round-r rotation of one index of the tile's pairs;
//   [.., + 2 JT)            the round-(r + 1) rotation of one of the tile's pairs.
// In an S unit (JT pairs x JS_PASS JS_ROWS rows) every thread owns JS_PASS rows of a pair
// and threads [0, 2 JT) / [2 JT, 3 JT) also take the rotations.
template <class JA>
__device__ __forceinline__ void jac_fused(int r, int s2, int nh, int npad, int half, int nT, int nA, int nRC, int nU,
                                          const int* perm, const int* inv, const typename JA::T* Ac,
                                          typename JA::T* An, const typename JA::T* Sc, typename JA::T* Sn,
                                          double eps, double floor_abs, int& my_rot, typename JA::T* f_al,
                                          typename JA::T* f_be, typename JA::T* f_c, typename JA::T* f_s,
                                          int* f_on, typename JA::T* f_ap) {
    using T = typename JA::T;
    const int tid = threadIdx.x;
    for (int u = blockIdx.x; u < nU; u += gridDim.x) {
        const bool isA = u < nA;
        int kA0 = 0, kB0 = 0, rc = 0;
        bool diagT = false;
        if (isA) {
            int I = 0, rem = u;
            while (rem >= nT - I) {
                rem -= nT - I;
                ++I;
            }
            kA0 = JT * I;
            kB0 = JT * (I + rem);
            diagT = rem == 0;
        } else {
            const int v = u - nA;
            kA0 = JT * (v / nRC);
            rc = v % nRC;
        }
        // ---- reads first (every role), so that all round trips overlap.  One
        // buffer serves all roles: an A-unit thread has one role; an S-unit
        // thread keeps its row in L[0..3] and a rotation's inputs after it.
        T L[20];
        int X0 = 0, X1 = 0, Y0 = 0, Y1 = 0, row = -1;
        int ka = -1, kb = -1, kk = -1, xi = 0, blk = 0;
        int rslot = -1, nslot = -1;  // round-r index slot, round-(r + 1) pair slot of this thread
        bool rrot = false, risp = true, nrot = false;
        const int nslots_r = isA ? 4 * JT : 2 * JT;
        const int base_r = isA ? 2 * JT * JT : 0;
        const int base_n = isA ? 2 * JT * JT + 4 * JT : 2 * JT;
        const int nslots_n = isA ? 2 * JT : JT;
        if (isA) {
            if (tid < 2 * JT * JT) {
                blk = tid >> 1;
                xi = tid & 1;
                const int a = blk % JT, b = blk / JT;
                if (kA0 + a < half && kB0 + b < half && (!diagT || a <= b)) {
                    ka = kA0 + a;
                    kb = kB0 + b;
                    jac_pair(r + 1, ka, s2, perm, X0, X1);
                    jac_pair(r + 1, kb, s2, perm, Y0, Y1);
                    const int x = xi ? X1 : X0;
                    const int px = jac_partner(r, x, s2, perm, inv).y;
                    const int ys[2] = {Y0, Y1};
                    const int py[2] = {jac_partner(r, Y0, s2, perm, inv).y, jac_partner(r, Y1, s2, perm, inv).y};
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        L[4 * j + 0] = JA::ld(Ac + x + (size_t)npad * ys[j]);
                        L[4 * j + 1] = JA::ld(Ac + x + (size_t)npad * py[j]);
                        L[4 * j + 2] = JA::ld(Ac + px + (size_t)npad * ys[j]);
                        L[4 * j + 3] = JA::ld(Ac + px + (size_t)npad * py[j]);
                    }
                }
            }
        } else {
            kk = tid / JS_ROWS;
            const int rw = rc * JS_ROWS * JS_PASS + tid % JS_ROWS;
            if (kk < JT && kA0 + kk < half && rw < npad) {
                ka = kA0 + kk;
                row = rw;
                jac_pair(r + 1, ka, s2, perm, X0, X1);
                const int p0 = jac_partner(r, X0, s2, perm, inv).y, p1 = jac_partner(r, X1, s2, perm, inv).y;
                L[0] = JA::ld(Sc + row + (size_t)npad * X0);
                L[1] = JA::ld(Sc + row + (size_t)npad * p0);
                L[2] = JA::ld(Sc + row + (size_t)npad * X1);
                L[3] = JA::ld(Sc + row + (size_t)npad * p1);
                if (row + JS_ROWS < npad) {
                    L[16] = JA::ld(Sc + row + JS_ROWS + (size_t)npad * X0);
                    L[17] = JA::ld(Sc + row + JS_ROWS + (size_t)npad * p0);
                    L[18] = JA::ld(Sc + row + JS_ROWS + (size_t)npad * X1);
                    L[19] = JA::ld(Sc + row + JS_ROWS + (size_t)npad * p1);
                }
            }
        }
        // round-r rotation of one index of the unit's round-(r + 1) pairs
        if (tid >= base_r && tid < base_r + nslots_r) {
            rslot = tid - base_r;
            const int ps = rslot >> 1;
            const int k1 = ps < JT ? kA0 + ps : kB0 + ps - JT;
            if (k1 < half) {
                int p1, q1;
                jac_pair(r + 1, k1, s2, perm, p1, q1);
                const int x = (rslot & 1) ? q1 : p1;
                const JPartner P = jac_partner(r, x, s2, perm, inv);
                if (P.k < nh) {
                    const int rp = P.isp ? x : P.y, rq = P.isp ? P.y : x;
                    const T v0 = JA::ld(Ac + rp + (size_t)npad * rp);
                    const T v1 = JA::ld(Ac + rq + (size_t)npad * rq);
                    const T v2 = JA::ld(Ac + rp + (size_t)npad * rq);
                    if (isA) {
                        L[0] = v0;
                        L[1] = v1;
                        L[2] = v2;
                    } else {
                        L[4] = v0;
                        L[5] = v1;
                        L[6] = v2;
                    }
                    rrot = true;
                    risp = P.isp;
                }
            }
        }
        // round-(r + 1) rotation of one of the unit's pairs: its diagonal block of A'
        int np1 = 0, nq1 = 0;
        if (tid >= base_n && tid < base_n + nslots_n) {
            nslot = tid - base_n;
            const int k1 = nslot < JT ? kA0 + nslot : kB0 + nslot - JT;
            if (k1 < half && k1 < nh) {
                jac_pair(r + 1, k1, s2, perm, np1, nq1);
                const int pp = jac_partner(r, np1, s2, perm, inv).y, pq = jac_partner(r, nq1, s2, perm, inv).y;
                const int ra[10] = {np1, np1, pp, nq1, nq1, pq, np1, np1, pp, pp};
                const int cb[10] = {np1, pp, pp, nq1, pq, pq, nq1, pq, nq1, pq};
                if (isA) {
#pragma unroll
                    for (int i = 0; i < 10; ++i) L[i] = JA::ld(Ac + ra[i] + (size_t)npad * cb[i]);
                } else {
#pragma unroll
                    for (int i = 0; i < 10; ++i) L[4 + i] = JA::ld(Ac + ra[i] + (size_t)npad * cb[i]);
                }
                nrot = true;
            }
        }
        // ---- phase 1: round-r coefficients (x' = al x + be pi(x))
        if (rslot >= 0) {
            T al = JA::one(), be = JA::zero();
            if (rrot) {
                const T v0 = isA ? L[0] : L[4], v1 = isA ? L[1] : L[5], v2 = isA ? L[2] : L[6];
                const typename JA::R R = JA::rot(v0, v1, v2, eps, floor_abs);
                if (R.on) {
                    al = R.c;
                    be = risp ? JA::neg(R.s) : R.s;
                    if (!isA && rc == 0 && risp) ++my_rot;
                }
            }
            f_al[rslot] = al;
            f_be[rslot] = be;
        }
        __syncthreads();
        // ---- phase 2: round-(r + 1) rotations from A' = (round r applied to A),
        // and each block row's entries of A'
        if (isA && ka >= 0) {
            const int a = ka - kA0, b = kb - kB0;
            const int sx = 2 * a + xi, sy = 2 * (JT + b);  // round-r slots of this row and of Y0
#pragma unroll
            for (int j = 0; j < 2; ++j)
                f_ap[4 * blk + 2 * xi + j] =
                    jprime<JA>(f_al[sx], f_be[sx], f_al[sy + j], f_be[sy + j], L[4 * j], L[4 * j + 1], L[4 * j + 2],
                               L[4 * j + 3]);
        }
        if (nslot >= 0) {
            typename JA::R R{JA::one(), JA::zero(), false};
            if (nrot) {
                const T ap = f_al[2 * nslot], bp = f_be[2 * nslot];
                const T aq = f_al[2 * nslot + 1], bq = f_be[2 * nslot + 1];
                T nv[10];
#pragma unroll
                for (int i = 0; i < 10; ++i) nv[i] = isA ? L[i] : L[4 + i];
                const T app = jprime<JA>(ap, bp, ap, bp, nv[0], nv[1], nv[1], nv[2]);
                const T aqq = jprime<JA>(aq, bq, aq, bq, nv[3], nv[4], nv[4], nv[5]);
                const T apq = jprime<JA>(ap, bp, aq, bq, nv[6], nv[7], nv[8], nv[9]);
                R = JA::rot(app, aqq, apq, eps, floor_abs);
                if (R.on && !isA && rc == 0) ++my_rot;
            }
            f_c[nslot] = R.c;
            f_s[nslot] = R.s;
            f_on[nslot] = R.on ? 1 : 0;
        }
        __syncthreads();
        // ---- phase 3: outputs
        if (ka >= 0) {
            if (isA) {
                const int a = ka - kA0, b = kb - kB0;
                const T* ap = f_ap + 4 * blk;  // A' on rows {X0, X1} x cols {Y0, Y1}, row-major
                // round r + 1: x' = al x + be partner, (al, be) = (c, -s) for p, (c, s) for q
                const bool ona = f_on[a] != 0, onb = f_on[JT + b] != 0;
                const T ca = ona ? f_c[a] : JA::one(), sa = ona ? f_s[a] : JA::zero();
                const T cb = onb ? f_c[JT + b] : JA::one(), sb = onb ? f_s[JT + b] : JA::zero();
                const T bx = xi ? sa : JA::neg(sa);
                const T by[2] = {JA::neg(sb), sb};
                const int i = xi;
                T o[2];
#pragma unroll
                for (int j = 0; j < 2; ++j)
                    o[j] = jprime<JA>(ca, bx, cb, by[j], ap[2 * i + j], ap[2 * i + 1 - j], ap[2 * (1 - i) + j],
                                      ap[2 * (1 - i) + 1 - j]);
                const int x = xi ? X1 : X0;
                if (ka == kb) {
                    if (xi == 0) {
                        An[X0 + (size_t)npad * X0] = o[0];
                        An[X0 + (size_t)npad * X1] = o[1];
                        An[X1 + (size_t)npad * X0] = o[1];
                    } else {
                        An[X1 + (size_t)npad * X1] = o[1];
                    }
                } else {
                    An[x + (size_t)npad * Y0] = o[0];
                    An[Y0 + (size_t)npad * x] = o[0];
                    An[x + (size_t)npad * Y1] = o[1];
                    An[Y1 + (size_t)npad * x] = o[1];
                }
            } else {
                const int sx = 2 * kk;
                const bool on = f_on[kk] != 0;
                const T c = on ? f_c[kk] : JA::one(), sn = on ? f_s[kk] : JA::zero();
                {
                    const T s0 = jcomb<JA>(f_al[sx], L[0], f_be[sx], L[1]);
                    const T s1 = jcomb<JA>(f_al[sx + 1], L[2], f_be[sx + 1], L[3]);
                    Sn[row + (size_t)npad * X0] = jcomb<JA>(c, s0, JA::neg(sn), s1);
                    Sn[row + (size_t)npad * X1] = jcomb<JA>(c, s1, sn, s0);
                }
                if (row + JS_ROWS < npad) {
                    const T s0 = jcomb<JA>(f_al[sx], L[16], f_be[sx], L[17]);
                    const T s1 = jcomb<JA>(f_al[sx + 1], L[18], f_be[sx + 1], L[19]);
                    Sn[row + JS_ROWS + (size_t)npad * X0] = jcomb<JA>(c, s0, JA::neg(sn), s1);
                    Sn[row + JS_ROWS + (size_t)npad * X1] = jcomb<JA>(c, s1, sn, s0);
                }
            }
        }
        __syncthreads();
    }
}

// Cooperative: all blocks co-resident (cudaLaunchAttributeCooperative).
//
// Each sweep starts with one parallel pass over all pairs that tags every
// index with a coupling above the threshold (act[i] = sweep + 1).  No tagged
// index means convergence, so no sweep is spent only to confirm it.  The
// sweep then runs the round-robin tournament over the tagged indices alone
// (padded to an even count with one untagged index): s - 1 rounds instead of
// npad - 1 once few pairs are left, while the untagged indices sit in fixed
// pairs that are never rotated.  When more than 3/4 of the indices are
// tagged, the tournament covers all of them.
//
// A round is split into units of similar FP64 cost, one or more per block:
// an A unit is a JT x JT tile of the upper triangle of 2x2 blocks of A (the
// transposed block is written from the same values, so A stays exactly
// symmetric); an S unit is JT column pairs x JS_PASS x JS_ROWS rows of S.  A unit
// computes only the (at most 2 JT) rotations it needs, with its input loads
// issued before the rotations so that both memory round trips overlap.  A is
// double-buffered (read from one buffer, written in full to the other); S is
// updated in place (the round's column pairs are disjoint).
template <class JA, bool FUSE>
__global__ void __launch_bounds__(256, FUSE ? 2 : JA::kMinBlocks) k_jacobi(int n, int npad, typename JA::T* A0, typename JA::T* A1,
                                                typename JA::T* S, typename JA::T* S1, double* __restrict__ diag,
                                                int* act, int max_sweeps, double eps, double floor_rel,
                                                DevCtl* ctl, const int* skip, int nhead) {
    using T = typename JA::T;
    // another solver already produced S and diag: every block leaves before
    // the first barrier
    if (skip && *(volatile const int*)skip) return;
    extern __shared__ int jsh[];
    int* perm = jsh;             // npad: tagged indices first
    int* flg = jsh + npad;       // npad: tag flags of this sweep
    int* inv = jsh + 2 * npad;   // npad: position of each index in perm
    __shared__ T u_c[2 * JT], u_s[2 * JT];
    __shared__ int u_on[2 * JT];
    // fused rounds: round-r coefficients per index slot, round-(r+1) rotations per pair slot
    __shared__ T f_al[4 * JT], f_be[4 * JT], f_c[2 * JT], f_s[2 * JT], f_ap[4 * JT * JT];
    __shared__ int f_on[2 * JT];
    __shared__ double s_red[8];
    __shared__ int s_cnt;
    const int half = npad / 2;
    const int nT = (half + JT - 1) / JT;
    const int nA = nT * (nT + 1) / 2;
    const int nRC = (npad + JS_ROWS * JS_PASS - 1) / (JS_ROWS * JS_PASS);
    const int nU = nA + nT * nRC;
    const long gtid = blockIdx.x * (long)blockDim.x + threadIdx.x;
    const long gstride = (long)gridDim.x * blockDim.x;
    const int tid = threadIdx.x;
    int* err = &ctl->jac_status;
    unsigned int epoch = 0;

    // absolute floor relative to the largest diagonal entry (same in all blocks)
    double mx = 0.0;
    for (int i = tid; i < n; i += blockDim.x) mx = fmax(mx, fabs(JA::to(JA::ld(A0 + i + (size_t)npad * i))));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((tid & 31) == 0) s_red[tid >> 5] = mx;
    __syncthreads();
    if (tid == 0) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = fmax(v, s_red[w]);
        s_red[0] = v;
    }
    __syncthreads();
    const double floor_abs = floor_rel * s_red[0];

    long rt = 0;  // rounds done: selects the current A buffer
    int sweep = 0, my_rot = 0;
    bool converged = false;
    for (sweep = 0;; ++sweep) {
        const T* Acur = (rt & 1) ? A1 : A0;
        const int tag = sweep + 1;
        for (long e = gtid; e < (long)npad * npad; e += gstride) {
            const int i = (int)(e % npad), j = (int)(e / npad);
            // pairs of two guard vectors (both >= nhead) need not converge
            if (i < j && i < nhead) {
                const T aij = JA::ld(Acur + i + (size_t)npad * j);
                if (JA::nz(aij) && JA::above(JA::ld(Acur + i + (size_t)npad * i), JA::ld(Acur + j + (size_t)npad * j),
                                             aij, eps, floor_abs)) {
                    act[i] = tag;
                    act[j] = tag;
                }
            }
        }
        if (!grid_sync(&ctl->bar_count, epoch, err)) return;
        // compaction by warp 0: tagged indices ascending, then the others
        for (int i = tid; i < npad; i += blockDim.x) flg[i] = __ldcg(act + i) == tag;
        __syncthreads();
        if (tid < 32) {
            int base = 0;
            for (int c0 = 0; c0 < npad; c0 += 32) {
                const int i = c0 + tid;
                const bool on = i < npad && flg[i];
                const unsigned bal = __ballot_sync(0xffffffffu, on);
                if (on) perm[base + __popc(bal & ((1u << tid) - 1u))] = i;
                base += __popc(bal);
            }
            const int ntag = base;
            for (int c0 = 0; c0 < npad; c0 += 32) {
                const int i = c0 + tid;
                const bool off = i < npad && !flg[i];
                const unsigned bal = __ballot_sync(0xffffffffu, off);
                if (off) perm[base + __popc(bal & ((1u << tid) - 1u))] = i;
                base += __popc(bal);
            }
            if (tid == 0) s_cnt = ntag;
        }
        __syncthreads();
        for (int a = tid; a < npad; a += blockDim.x) inv[perm[a]] = a;
        __syncthreads();
        const int ntag = s_cnt;
        if (ntag == 0) {
            converged = true;
            break;
        }
        if (sweep >= max_sweeps) break;
        int s2 = ntag + (ntag & 1);  // ntag odd => ntag < npad: an untagged index exists
        if (4 * s2 > 3 * npad) s2 = npad;
        const int nh = s2 / 2;
        for (int r = 0; r < s2 - 1;) {
            const T* Ac = (rt & 1) ? A1 : A0;
            T* An = (rt & 1) ? A0 : A1;
            // S is double-buffered when S1 is given (a fused pair of rounds
            // reads columns that other units write), else updated in place
            const T* Sc = (S1 && (rt & 1)) ? S1 : S;
            T* Sn = S1 ? ((rt & 1) ? S : S1) : S;
            const bool fuse = FUSE && S1 != nullptr && r + 2 <= s2 - 1;
            if (fuse) {
                jac_fused<JA>(r, s2, nh, npad, half, nT, nA, nRC, nU, perm, inv, Ac, An, Sc, Sn, eps, floor_abs,
                              my_rot, f_al, f_be, f_c, f_s, f_on, f_ap);
                r += 2;
                ++rt;
                if (!grid_sync(&ctl->bar_count, epoch, err)) return;
                continue;
            }
            for (int u = blockIdx.x; u < nU; u += gridDim.x) {
                const bool isA = u < nA;
                int kA0, kB0 = 0, rc = 0;
                bool diagT = false;
                if (isA) {  // upper-triangular tile (I, J), I <= J, row by row
                    int I = 0, rem = u;
                    while (rem >= nT - I) {
                        rem -= nT - I;
                        ++I;
                    }
                    kA0 = JT * I;
                    kB0 = JT * (I + rem);
                    diagT = rem == 0;
                } else {
                    const int v = u - nA;
                    kA0 = JT * (v / nRC);
                    rc = v % nRC;
                }
                // item inputs first
                int ka = -1, kb = -1, row = -1, p = 0, q = 0, pr = 0, pt = 0;
                T x0 = JA::zero(), x1 = JA::zero(), x2 = JA::zero(), x3 = JA::zero();
                if (isA) {
                    if (tid < JT * JT) {
                        const int a = tid % JT, b = tid / JT;
                        if (kA0 + a < half && kB0 + b < half && (!diagT || a <= b)) {
                            ka = kA0 + a;
                            kb = kB0 + b;
                            jac_pair(r, ka, s2, perm, p, q);
                            if (ka == kb) {
                                x0 = JA::ld(Ac + p + (size_t)npad * p);
                                x1 = JA::ld(Ac + q + (size_t)npad * q);
                                x2 = JA::ld(Ac + p + (size_t)npad * q);
                            } else {
                                jac_pair(r, kb, s2, perm, pr, pt);
                                x0 = JA::ld(Ac + p + (size_t)npad * pr);
                                x1 = JA::ld(Ac + p + (size_t)npad * pt);
                                x2 = JA::ld(Ac + q + (size_t)npad * pr);
                                x3 = JA::ld(Ac + q + (size_t)npad * pt);
                            }
                        }
                    }
                } else {
                    // rows rw and rw + JS_ROWS (x0, x1 and x2, x3)
                    const int kk = tid / JS_ROWS;
                    const int rw = rc * JS_ROWS * JS_PASS + tid % JS_ROWS;
                    if (kk < JT && kA0 + kk < half && rw < npad) {
                        ka = kA0 + kk;
                        row = rw;
                        jac_pair(r, ka, s2, perm, p, q);
                        x0 = JA::ld(Sc + row + (size_t)npad * p);
                        x1 = JA::ld(Sc + row + (size_t)npad * q);
                        if (row + JS_ROWS < npad) {
                            x2 = JA::ld(Sc + row + JS_ROWS + (size_t)npad * p);
                            x3 = JA::ld(Sc + row + JS_ROWS + (size_t)npad * q);
                        }
                    }
                }
                // the unit's rotations
                const int nrot = isA ? 2 * JT : JT;
                const int rtid = isA ? tid - JT * JT : tid;  // A units: threads after the items
                if (rtid >= 0 && rtid < nrot) {
                    const int k = rtid < JT ? kA0 + rtid : kB0 + rtid - JT;
                    typename JA::R R{JA::one(), JA::zero(), false};
                    if (k < nh) {
                        int rp, rq;
                        jac_pair(r, k, s2, perm, rp, rq);
                        R = JA::rot(JA::ld(Ac + rp + (size_t)npad * rp), JA::ld(Ac + rq + (size_t)npad * rq),
                                    JA::ld(Ac + rp + (size_t)npad * rq), eps, floor_abs);
                    }
                    u_c[rtid] = R.c;
                    u_s[rtid] = R.s;
                    u_on[rtid] = R.on ? 1 : 0;
                    if (!isA && rc == 0 && R.on) ++my_rot;
                }
                __syncthreads();
                if (ka >= 0) {
                    if (isA) {
                        const int ia = ka - kA0, ib = JT + kb - kB0;
                        const T ca = u_c[ia], sa = u_s[ia];
                        const bool ona = u_on[ia] != 0;
                        if (ka == kb) {
                            if (ona) {
                                // J^t [[app, apq], [apq, aqq]] J with J = [[c, s], [-s, c]]
                                const T app = x0, aqq = x1, apq = x2, nca = JA::neg(ca);
                                const T y_pp = JA::lin(ca, app, sa, apq), y_pq = JA::lin(ca, apq, sa, aqq);
                                const T y_qp = JA::lin(sa, app, nca, apq), y_qq = JA::lin(sa, apq, nca, aqq);
                                const T npq =
                                    JA::half(JA::add(JA::lin(sa, y_pp, nca, y_pq), JA::lin(ca, y_qp, sa, y_qq)));
                                An[p + (size_t)npad * p] = JA::lin(ca, y_pp, sa, y_pq);
                                An[q + (size_t)npad * q] = JA::lin(sa, y_qp, nca, y_qq);
                                An[p + (size_t)npad * q] = npq;
                                An[q + (size_t)npad * p] = npq;
                            } else {
                                An[p + (size_t)npad * p] = x0;
                                An[q + (size_t)npad * q] = x1;
                                An[p + (size_t)npad * q] = x2;
                                An[q + (size_t)npad * p] = x2;
                            }
                        } else {
                            const T cb = u_c[ib], sb = u_s[ib];
                            const bool onb = u_on[ib] != 0;
                            T o_pr = x0, o_pt = x1, o_qr = x2, o_qt = x3;
                            if (ona || onb) {
                                // J_a^t from the left (rows p, q), J_b from the right (columns r, t)
                                const T nca = JA::neg(ca), ncb = JA::neg(cb);
                                const T y_pr = JA::lin(ca, x0, sa, x2), y_pt = JA::lin(ca, x1, sa, x3);
                                const T y_qr = JA::lin(sa, x0, nca, x2), y_qt = JA::lin(sa, x1, nca, x3);
                                o_pr = JA::lin(cb, y_pr, sb, y_pt);
                                o_pt = JA::lin(sb, y_pr, ncb, y_pt);
                                o_qr = JA::lin(cb, y_qr, sb, y_qt);
                                o_qt = JA::lin(sb, y_qr, ncb, y_qt);
                            }
                            An[p + (size_t)npad * pr] = o_pr;
                            An[p + (size_t)npad * pt] = o_pt;
                            An[q + (size_t)npad * pr] = o_qr;
                            An[q + (size_t)npad * pt] = o_qt;
                            An[pr + (size_t)npad * p] = o_pr;
                            An[pt + (size_t)npad * p] = o_pt;
                            An[pr + (size_t)npad * q] = o_qr;
                            An[pt + (size_t)npad * q] = o_qt;
                        }
                    } else {
                        const int ia = ka - kA0;
                        const bool two = row + JS_ROWS < npad;
                        if (u_on[ia]) {
                            const T c = u_c[ia], sn = u_s[ia];
                            Sn[row + (size_t)npad * p] = JA::lin(c, x0, sn, x1);
                            Sn[row + (size_t)npad * q] = JA::lin(sn, x0, JA::neg(c), x1);
                            if (two) {
                                Sn[row + JS_ROWS + (size_t)npad * p] = JA::lin(c, x2, sn, x3);
                                Sn[row + JS_ROWS + (size_t)npad * q] = JA::lin(sn, x2, JA::neg(c), x3);
                            }
                        } else if (Sn != Sc) {
                            Sn[row + (size_t)npad * p] = x0;
                            Sn[row + (size_t)npad * q] = x1;
                            if (two) {
                                Sn[row + JS_ROWS + (size_t)npad * p] = x2;
                                Sn[row + JS_ROWS + (size_t)npad * q] = x3;
                            }
                        }
                    }
                }
                __syncthreads();
            }
            ++r;
            ++rt;
            if (!grid_sync(&ctl->bar_count, epoch, err)) return;
        }
        if (my_rot) atomicAdd(&ctl->rot_count[sweep < 64 ? sweep : 63], my_rot);
        my_rot = 0;
    }
    const T* Af = (rt & 1) ? A1 : A0;
    for (long i = gtid; i < n; i += gstride) diag[i] = JA::to(JA::ld(Af + i + (size_t)npad * i));
    // the eigenvectors end in S (every block passed the last barrier)
    if (S1 && (rt & 1))
        for (long e = gtid; e < (long)npad * npad; e += gstride) S[e] = JA::ld(S1 + e);
    if (gtid == 0) {
        ctl->jac_sweeps = sweep;
        if (!converged) atomicMax(err, 1);
    }
}

// Sort Ritz pairs by |theta| descending (ties by index): rank, then gather.
__global__ void k_rank_ritz(int n, const double* __restrict__ diag, int* __restrict__ rank,
                            double* __restrict__ theta) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        double aj = fabs(diag[j]);
        int r = 0;
        for (int k = 0; k < n; ++k) {
            double ak = fabs(diag[k]);
            r += (ak > aj) || (ak == aj && k < j);
        }
        rank[j] = r;
        theta[r] = diag[j];
    }
}

template <class JA>
__global__ void k_gather_ritz(int n, int npad, const int* __restrict__ rank, const typename JA::T* __restrict__ S,
                              double* __restrict__ Sout, int ldo) {
    size_t tot = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot;
         e += (size_t)gridDim.x * blockDim.x) {
        int row = (int)(e % n), j = (int)(e / n);
        Sout[row + (size_t)ldo * rank[j]] = JA::to(S[row + (size_t)npad * j]);
    }
}

// Blocked right-looking Cholesky G + shift I = L L^t (lower, in place),
// panel width 32.  Cooperative launch, two grid barriers per panel: every
// block factors the 32 x 32 diagonal block itself (identical arithmetic in
// each, so all agree) and solves its share of the panel rows (one row per
// thread, held in registers, with the pivots' reciprocals taken once); the
// trailing update then runs on 16 x 16 lower tiles, so that it spreads over
// many SMs (FP64 throughput per SM is low on this part).
// 1/sqrt(d) for d > 0: FP32 seed refined by two Newton-Raphson steps
// y <- y (3 - d y^2) / 2 (FP64 square roots and divisions are slow on this
// part); the library path outside FP32's comfortable range.
__device__ __forceinline__ double rsqrt_nr(double d) {
    if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
    double y = (double)rsqrtf((float)d);
    y = y * (1.5 - 0.5 * d * y * y);
    y = y * (1.5 - 0.5 * d * y * y);
    return y;
}

// Arithmetic of the Cholesky factorisation (G stays FP64 in memory).  C64:
// FP64.  CDF: double-float pairs on the FP32 pipe for the mixed-precision
// forms, whose last orthonormalisation pass (Newton-Schulz) corrects the
// factor's rounding to O(|E|^2).
struct C64 {
    using T = double;
    __device__ static T from(double x) { return x; }
    __device__ static double to(T a) { return a; }
    __device__ static T zero() { return 0.0; }
    __device__ static T mul(T a, T b) { return a * b; }
    __device__ static T sub(T a, T b) { return a - b; }
    __device__ static T neg(T a) { return -a; }
    __device__ static T rsq(T d) { return rsqrt_nr(d); }
    __device__ static T shfl(T a, int l) { return __shfl_sync(0xffffffffu, a, l); }
    struct Acc {
        double a0, a1;
    };
    __device__ static Acc acc0() { return Acc{0.0, 0.0}; }
    __device__ static void acc2(Acc& c, T x0, T y0, T x1, T y1) {
        c.a0 = fma(x0, y0, c.a0);
        c.a1 = fma(x1, y1, c.a1);
    }
    __device__ static T fin(Acc c) { return c.a0 + c.a1; }
};

struct CDF {
    using T = float2;
    __device__ static T quick(float s, float e) {
        const float h = s + e;
        return make_float2(h, e - (h - s));
    }
    __device__ static T from(double x) {
        const float h = (float)x;
        return make_float2(h, (float)(x - (double)h));
    }
    __device__ static double to(T a) { return f2d_bits(a.x) + f2d_bits(a.y); }
    __device__ static T zero() { return make_float2(0.f, 0.f); }
    __device__ static T mul(T a, T b) {
        const float p = a.x * b.x;
        return quick(p, fmaf(a.x, b.x, -p) + fmaf(a.x, b.y, a.y * b.x));
    }
    __device__ static T add(T a, T b) {
        const float s = a.x + b.x, bb = s - a.x;
        const float e = (a.x - (s - bb)) + (b.x - bb);
        return quick(s, e + (a.y + b.y));
    }
    __device__ static T sub(T a, T b) { return add(a, make_float2(-b.x, -b.y)); }
    __device__ static T neg(T a) { return make_float2(-a.x, -a.y); }
    // 1/sqrt(d): FP32 seed, two double-float Newton steps y <- y + y (1 - d y^2)/2
    __device__ static T rsq(T d) {
        T y = make_float2(rsqrtf(d.x), 0.f);
#pragma unroll
        for (int it = 0; it < 2; ++it) {
            const T r = sub(make_float2(1.f, 0.f), mul(d, mul(y, y)));
            y = add(y, make_float2(0.5f * y.x * r.x, 0.f));
        }
        return y;
    }
    __device__ static T shfl(T a, int l) {
        return make_float2(__shfl_sync(0xffffffffu, a.x, l), __shfl_sync(0xffffffffu, a.y, l));
    }
    struct Acc {
        float h, l;
    };
    __device__ static Acc acc0() { return Acc{0.f, 0.f}; }
    __device__ static void acc1(Acc& c, T a, T b) {
        const float p = a.x * b.x, pe = fmaf(a.x, b.x, -p);
        const float s = c.h + p, bb = s - c.h;
        const float e = (c.h - (s - bb)) + (p - bb);
        c.h = s;
        c.l += (e + pe) + fmaf(a.x, b.y, a.y * b.x);
    }
    __device__ static void acc2(Acc& c, T x0, T y0, T x1, T y1) {
        acc1(c, x0, y0);
        acc1(c, x1, y1);
    }
    __device__ static T fin(Acc c) { return quick(c.h, c.l); }
};

template <class CA>
__global__ void __launch_bounds__(256, 2) k_cholesky(int n, double* G, int ld, double shift_rel, DevCtl* ctl,
                                                    const int* skip) {
    using T = typename CA::T;
    // a Newton-Schulz correction replaces this factorisation: every block
    // leaves before the first barrier
    if (skip && *(volatile const int*)skip) return;
    __shared__ T D[32][33];
    __shared__ T dinv[32];
    __shared__ T dinv2[32];
    __shared__ T PI[32][17];  // panel rows of tile I (l-major)
    __shared__ T PJ[32][17];  // panel rows of tile J
    __shared__ double s_red[8];
    int* err = &ctl->chol_status;
    const long gtid = blockIdx.x * (long)blockDim.x + threadIdx.x;
    const long gstride = (long)gridDim.x * blockDim.x;
    const int tid = threadIdx.x, lane = tid & 31;
    const unsigned full = 0xffffffffu;
    unsigned int epoch = 0;
    if (shift_rel > 0.0) {
        // trace(G), reduced in the same order in every block
        double t = 0.0;
        for (int i = tid; i < n; i += blockDim.x) t += G[i + (size_t)ld * i];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(full, t, o);
        if (lane == 0) s_red[tid >> 5] = t;
        __syncthreads();
        double tr = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tr += s_red[w];
        const double shift = tr * shift_rel;
        if (!grid_sync(&ctl->bar_count, epoch, err)) return;
        for (long i = gtid; i < n; i += gstride) G[i + (size_t)ld * i] = __ldcg(G + i + (size_t)ld * i) + shift;
        if (!grid_sync(&ctl->bar_count, epoch, err)) return;
    }
    for (int k0 = 0; k0 < n; k0 += 32) {
        const int kb = min(32, n - k0);
        // --- diagonal block, factored redundantly in every block by all its
        //     threads (FP64 work in one warp is slow on this part).  Columns
        //     stay unscaled until the end: step j subtracts
        //     D[i][j] D[l][j] / d_j from the trailing entries, and the thread
        //     that updates the next pivot takes its reciprocal square root.
        for (int e = tid; e < 32 * 32; e += blockDim.x) {
            const int i = e % 32, j = e / 32;
            D[i][j] = (i < kb && j < kb && j <= i) ? CA::from(__ldcg(G + (k0 + i) + (size_t)ld * (k0 + j)))
                                                   : CA::zero();
        }
        __syncthreads();
        if (tid == 0) {
            T d = D[0][0];
            const double dd = CA::to(d);
            if (!(dd > 0.0) || !isfinite(dd)) {
                if (blockIdx.x == 0) atomicMax(err, 1);
                d = CA::from(1.0);
                D[0][0] = d;
            }
            const T inv = CA::rsq(d);
            dinv[0] = inv;
            dinv2[0] = CA::mul(inv, inv);
        }
        __syncthreads();
        // Fixed ownership (256 threads): lane = row i, warp w holds columns
        // w, w + 8, w + 16, w + 24, so a pivot step is four predicated
        // updates per thread with no index arithmetic on the chain.
        for (int j = 0; j + 1 < kb; ++j) {
            const T w = dinv2[j];
            const int i = lane;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int l = (tid >> 5) + 8 * r;
                if (l > j && l <= i && i < kb) {
                    T v = CA::sub(D[i][l], CA::mul(CA::mul(D[i][j], D[l][j]), w));
                    if (i == j + 1 && l == j + 1) {  // the next pivot
                        const double vv = CA::to(v);
                        if (!(vv > 0.0) || !isfinite(vv)) {
                            if (blockIdx.x == 0) atomicMax(err, 1);
                            v = CA::from(1.0);
                        }
                        const T inv = CA::rsq(v);
                        dinv[j + 1] = inv;
                        dinv2[j + 1] = CA::mul(inv, inv);
                    }
                    D[i][l] = v;
                }
            }
            __syncthreads();
        }
        // scale: L[i][j] = D[i][j] / sqrt(d_j) (i > j), L[j][j] = d_j / sqrt(d_j)
        for (int e = tid; e < 32 * 32; e += blockDim.x) {
            const int i = e % 32, j = e / 32;
            if (j < kb && i < kb && j <= i) D[i][j] = CA::mul(D[i][j], dinv[j]);
        }
        __syncthreads();
        if (blockIdx.x == 0)
            for (int e = tid; e < kb * kb; e += blockDim.x) {
                const int i = e % kb, j = e / kb;
                G[(k0 + i) + (size_t)ld * (k0 + j)] = CA::to(D[i][j]);
            }
        const int k1 = k0 + kb;
        // --- panel rows below: L[i, k0:k1] = G[i, k0:k1] L_kk^{-t}, one warp
        //     per row (lane j holds column j), rows spread over the grid
        {
            const long gw = gtid >> 5, nw = gstride >> 5;
            for (long i = k1 + gw; i < n; i += nw) {
                T acc = (lane < kb) ? CA::from(__ldcg(G + i + (size_t)ld * (k0 + lane))) : CA::zero();
                T x = CA::zero();
#pragma unroll
                for (int l = 0; l < 32; ++l) {
                    if (l < kb) {
                        const T xl = CA::mul(CA::shfl(acc, l), dinv[l]);
                        if (lane == l) x = xl;
                        if (lane > l) acc = CA::sub(acc, CA::mul(xl, D[lane][l]));
                    }
                }
                if (lane < kb) G[i + (size_t)ld * (k0 + lane)] = CA::to(x);
            }
        }
        if (!grid_sync(&ctl->bar_count, epoch, err)) return;
        if (k1 >= n) break;
        // --- trailing update on 16 x 16 tiles of the lower triangle
        const int nt = n - k1;
        const int T = (nt + 15) / 16;
        const long ntiles = (long)T * (T + 1) / 2;
        const int tx = tid & 15, ty = tid >> 4;
        for (long tIdx = blockIdx.x; tIdx < ntiles; tIdx += gridDim.x) {
            // tile (I, J), I >= J, enumerated row by row
            int I = (int)((sqrtf(8.0f * (float)tIdx + 1.0f) - 1.0f) * 0.5f);  // corrected below
            while ((long)(I + 1) * (I + 2) / 2 <= tIdx) ++I;
            while ((long)I * (I + 1) / 2 > tIdx) --I;
            const int J = (int)(tIdx - (long)I * (I + 1) / 2);
            const int i0 = k1 + 16 * I, j0 = k1 + 16 * J;
            for (int e = tid; e < 16 * 32; e += blockDim.x) {
                const int r = e & 15, l = e >> 4;
                PI[l][r] = (l < kb && i0 + r < n) ? CA::from(__ldcg(G + (i0 + r) + (size_t)ld * (k0 + l)))
                                                  : CA::zero();
                PJ[l][r] = (l < kb && j0 + r < n) ? CA::from(__ldcg(G + (j0 + r) + (size_t)ld * (k0 + l)))
                                                  : CA::zero();
            }
            __syncthreads();
            const int i = i0 + tx, j = j0 + ty;
            if (i < n && j < n && j <= i) {
                typename CA::Acc c = CA::acc0();
#pragma unroll
                for (int l = 0; l < 32; l += 2) CA::acc2(c, PI[l][tx], PJ[l][ty], PI[l + 1][tx], PJ[l + 1][ty]);
                double* g = G + i + (size_t)ld * j;
                *g = CA::to(CA::sub(CA::from(__ldcg(g)), CA::fin(c)));
            }
            __syncthreads();
        }
        if (!grid_sync(&ctl->bar_count, epoch, err)) return;
    }
}

// Inverses of the 32 x 32 diagonal blocks of the lower triangular L
// (column-major, ld): Dinv + 1024 I holds the inverse of block I, column-major
// and zero-padded.  One warp per block, one column of the inverse per lane
// (forward substitution with the pivots' reciprocals taken once).
__global__ void __launch_bounds__(32) k_trinv_diag(int n, const double* __restrict__ L, int ld,
                                                   double* __restrict__ Dinv, const int* __restrict__ skip) {
    if (skip && *skip) return;
    __shared__ double Ls[32][33];
    __shared__ double rd[32];
    const int I = blockIdx.x, r0 = 32 * I, nbI = min(32, n - r0);
    const int c = threadIdx.x;
    for (int i = 0; i < 32; ++i)
        Ls[i][c] = (i < nbI && c < nbI && c <= i) ? L[(r0 + i) + (size_t)ld * (r0 + c)] : 0.0;
    __syncwarp();
    rd[c] = (c < nbI) ? 1.0 / Ls[c][c] : 0.0;
    __syncwarp();
    double x[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        double sacc = (i == c) ? 1.0 : 0.0;
#pragma unroll
        for (int k = 0; k < i; ++k) sacc -= Ls[i][k] * x[k];
        x[i] = (i >= c && i < nbI && c < nbI) ? sacc * rd[i] : 0.0;
    }
    double* out = Dinv + (size_t)1024 * I + 32 * c;
#pragma unroll
    for (int i = 0; i < 32; ++i) out[i] = x[i];
}

// X = L^{-1} (lower triangular) by blocked forward substitution over 32-row
// blocks, eight columns j per CTA (one warp each, all in the same block J):
// x_J = Dinv_J e_j, then for each later block x_I = -Dinv_I (L_{I, J:I}
// x_{J:I}).  The 32 x 32 tiles of L are staged in shared memory, shared by
// the eight warps, with the next tile prefetched into registers.
template <class CA>
__global__ void __launch_bounds__(256) k_trinv_cols(int n, const double* __restrict__ L, int ld,
                                                    const double* __restrict__ Dinv, double* __restrict__ X,
                                                    int ldx, const int* __restrict__ skip) {
    using T = typename CA::T;
    static_assert(sizeof(T) == sizeof(double), "shared-memory layout assumes 8-byte elements");
    if (skip && *skip) return;
    extern __shared__ double tsh_raw[];
    T* tsh = reinterpret_cast<T*>(tsh_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int npad = ((n + 31) / 32) * 32, nb = npad / 32;
    T* xs = tsh + (size_t)warp * npad;  // this warp's column of X
    T* Tt = tsh + (size_t)8 * npad;     // [2][32][33] tiles of L
    T* Di = Tt + 2 * 32 * 33;           // [32][33] Dinv_I
    T* ys = Di + 32 * 33;               // [8][32]
    const int j0 = blockIdx.x * 8, j = j0 + warp;
    const bool live_col = j < n;
    const int J = j0 / 32, c = j % 32;
    if (live_col)
        for (int i = lane; i < 32 * J; i += 32) X[i + (size_t)ldx * j] = 0.0;
    {
        const double v = live_col ? Dinv[(size_t)1024 * J + 32 * c + lane] : 0.0;  // zero above row c
        xs[32 * J + lane] = CA::from(v);
        if (live_col && 32 * J + lane < n) X[(32 * J + lane) + (size_t)ldx * j] = v;
    }
    double reg[4];
    for (int I = J + 1; I < nb; ++I) {
        __syncthreads();  // Di and the tiles of the previous I are consumed
        for (int e = tid; e < 1024; e += 256) Di[(e % 32) * 33 + e / 32] = CA::from(Dinv[(size_t)1024 * I + e]);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 256 * q, r = 32 * I + (e % 32), col = 32 * J + e / 32;
            reg[q] = (r < n) ? L[r + (size_t)ld * col] : 0.0;
        }
        typename CA::Acc acc = CA::acc0();
        for (int kb = J, buf = 0; kb < I; ++kb, buf ^= 1) {
            T* Tb = Tt + buf * 32 * 33;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int e = tid + 256 * q;
                Tb[(e % 32) * 33 + e / 32] = CA::from(reg[q]);
            }
            __syncthreads();
            if (kb + 1 < I) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int e = tid + 256 * q, r = 32 * I + (e % 32), col = 32 * (kb + 1) + e / 32;
                    reg[q] = (r < n) ? L[r + (size_t)ld * col] : 0.0;
                }
            }
            const T* xk = xs + 32 * kb;
#pragma unroll
            for (int cc = 0; cc < 32; cc += 2)
                CA::acc2(acc, Tb[lane * 33 + cc], xk[cc], Tb[lane * 33 + cc + 1], xk[cc + 1]);
        }
        ys[warp * 32 + lane] = CA::fin(acc);
        __syncwarp();
        typename CA::Acc ax = CA::acc0();
#pragma unroll
        for (int s2 = 0; s2 < 32; s2 += 2)
            CA::acc2(ax, Di[lane * 33 + s2], ys[warp * 32 + s2], Di[lane * 33 + s2 + 1], ys[warp * 32 + s2 + 1]);
        const T xi = CA::neg(CA::fin(ax));
        xs[32 * I + lane] = xi;
        if (live_col && 32 * I + lane < n) X[(32 * I + lane) + (size_t)ldx * j] = CA::to(xi);
        __syncwarp();
    }
}

// res[i] = || T_i - theta_i Z_i ||_2 for i < ncol; one block per column.
__global__ void k_resid(int N, int ncol, const double* __restrict__ T, const double* __restrict__ Z,
                        int ld, const double* __restrict__ theta, double* __restrict__ res) {
    __shared__ double red[32];
    int i = blockIdx.x;
    if (i >= ncol) return;
    double th = theta[i];
    double s = 0.0;
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
        double d = T[r + (size_t)ld * i] - th * Z[r + (size_t)ld * i];
        s += d * d;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) res[i] = sqrt(s);
    }
}

// Multiplet-aware truncation and the convergence test of the Ritz pairs.
__global__ void k_decide(int b, int L, int m, double tol, double tol_c, const double* __restrict__ theta,
                         const double* __restrict__ res, DevCtl* ctl) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int Le = min(b, L);
    double a1 = fabs(theta[0]);
    bool bad = !isfinite(a1) || a1 == 0.0;
    int meff = min(m, Le);
    while (meff > 0 && meff < Le && fabs(fabs(theta[meff - 1]) - fabs(theta[meff])) <= tol_c * a1) --meff;
    while (meff > 0 && fabs(theta[meff - 1]) <= tol_c * a1) --meff;
    int nchk = min(m + 1, Le);
    double rmax = 0.0;
    for (int i = 0; i < nchk; ++i) {
        double r = res[i];
        if (!isfinite(r) || !isfinite(theta[i])) bad = true;
        rmax = fmax(rmax, r);
    }
    ctl->meff_new = bad ? 0 : meff;
    ctl->resid = bad ? INFINITY : rmax / a1;
    ctl->theta0 = theta[0];
    // dynamic range of the Ritz values the next block is divided by (those
    // above 1e-12 |theta_0|)
    double tmin = a1;
    for (int i = 1; i < b; ++i) {
        const double t = fabs(theta[i]);
        if (t > 1e-12 * a1) tmin = fmin(tmin, t);
    }
    ctl->theta_range = (bad || !(a1 > 0.0)) ? 0.0 : tmin / a1;
    ctl->sub_converged = (!bad && rmax <= tol * a1) ? 1 : 0;
    if (bad) ctl->numeric_bad = 1;
}

// Column-wise combinations of N x b blocks, out_i = alpha_i X_i + beta_i W_i,
// with the coefficients of column i computed once per column (this part's
// FP64 division is slow: one per element cost more than the memory traffic).
enum BlockMode { BM_NEXT = 0, BM_CHEB2 = 1, BM_CHEB3 = 2 };

// BM_NEXT: X = T = C~ V, W = Z: T_i / theta_i, or Z_i for a negligible
//   theta_i (keeps the Gram matrix well conditioned).
// BM_CHEB2: X = Y = C~ (C~ V / theta), W = V: the pair of power steps as the
//   degree-2 Chebyshev polynomial on [-a, a], a = |theta_{b-1}| (the block's
//   smallest Ritz value, an estimate of the unwanted spectrum's edge),
//   normalised at theta_i: (c Y_i / theta_i - V_i) / (c - 1), c = 2 u^2,
//   u = |theta_i| / a, when c >= 4.5; else Y_i / theta_i.
// BM_CHEB3: X = Y = C~^3 V / theta^2, W = T = C~ V / theta: three steps as
//   T_3: (4u^3 Y_i / theta_i - 3u T_i) / (4u^3 - 3u) when u >= 1.5; else
//   Y_i / theta_i.  Components with |lambda| <= a shrink by 1/T_k(u) instead
//   of u^-k.
__device__ void block_coeffs(int mode, int i, int b, const double* __restrict__ theta, double eps_theta,
                             double& al, double& be) {
    const double a1 = fabs(theta[0]);
    const double th = theta[i];
    if (!(fabs(th) > eps_theta * a1)) {  // negligible Ritz value: keep W_i
        al = 0.0;
        be = 1.0;
        return;
    }
    al = 1.0 / th;
    be = 0.0;
    if (mode == BM_NEXT) return;
    const double a = fabs(theta[b - 1]);
    if (!(a > eps_theta * a1)) return;
    const double u = fabs(th) / a;
    if (mode == BM_CHEB2) {
        const double c = 2.0 * u * u;  // T_2(u) = c - 1
        if (c >= 4.5) {
            al = c / (th * (c - 1.0));
            be = -1.0 / (c - 1.0);
        }
    } else if (u >= 1.5) {
        const double u3 = 4.0 * u * u * u, u1 = 3.0 * u;  // T_3(u) = u3 - u1
        al = u3 / (th * (u3 - u1));
        be = -u1 / (u3 - u1);
    }
}

// out may alias W (each element reads only its own position)
__global__ void k_col_combine(int mode, int N, int b, const double* __restrict__ X, const double* W, double* out,
                              int ld, const double* __restrict__ theta, double eps_theta) {
    __shared__ double s_al, s_be;
    const int i = blockIdx.y;
    if (threadIdx.x == 0) {
        double al, be;
        block_coeffs(mode, i, b, theta, eps_theta, al, be);
        s_al = al;
        s_be = be;
    }
    __syncthreads();
    const double al = s_al, be = s_be;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < N; r += gridDim.x * blockDim.x) {
        const size_t o = r + (size_t)ld * i;
        out[o] = (be == 0.0) ? al * X[o] : (al == 0.0 ? be * W[o] : fma(al, X[o], be * W[o]));
    }
}

void col_combine(cudaStream_t st, int mode, int N, int b, const double* X, const double* W, double* out, int ld,
                 const double* theta, double eps_theta) {
    if (N <= 0 || b <= 0) return;
    const dim3 grid((unsigned)std::min((N + 255) / 256, 16), (unsigned)b);
    k_col_combine<<<grid, 256, 0, st>>>(mode, N, b, X, W, out, ld, theta, eps_theta);
}

// Dot products for the gauge alignment: d[3 i + 0] = z_i.v_i,
// d[3 i + 1] = z_i.v_{i+1}, d[3 i + 2] = z_{i+1}.v_i.
__global__ void k_gauge_dots(int N, int b, const double* __restrict__ Z, const double* __restrict__ V,
                             int ld, double* __restrict__ d) {
    __shared__ double red[3][32];
    int i = blockIdx.x;
    if (i >= b) return;
    bool nx = (i + 1 < b);
    double s0 = 0, s1 = 0, s2 = 0;
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
        double zi = Z[r + (size_t)ld * i], vi = V[r + (size_t)ld * i];
        s0 += zi * vi;
        if (nx) {
            s1 += zi * V[r + (size_t)ld * (i + 1)];
            s2 += Z[r + (size_t)ld * (i + 1)] * vi;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = s0;
        red[1][w] = s1;
        red[2][w] = s2;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        int nw = blockDim.x >> 5;
        s0 = threadIdx.x < nw ? red[0][threadIdx.x] : 0.0;
        s1 = threadIdx.x < nw ? red[1][threadIdx.x] : 0.0;
        s2 = threadIdx.x < nw ? red[2][threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        if (threadIdx.x == 0) {
            d[3 * i + 0] = s0;
            d[3 * i + 1] = s1;
            d[3 * i + 2] = s2;
        }
    }
}

// Plan: per Ritz column a 2x2 block Q (singlet: sign in Q00; doublet of
// equal theta: orthogonal polar factor of K = Z_c^t V_c).  kind[i]: 0
// singlet, 1 first of a doublet, 2 second of a doublet.
// One thread per column; the thread of a cluster's first column plans it.
__global__ void k_gauge_plan(int b, const double* __restrict__ theta, double tol_c,
                             const double* __restrict__ d, double* __restrict__ Q, int* __restrict__ kind) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b) return;
    const double a1 = fabs(theta[0]);
    if (i > 0 && fabs(theta[i] - theta[i - 1]) <= tol_c * a1) return;  // not a cluster's first column
    {
        int j = i + 1;
        while (j < b && fabs(theta[j] - theta[j - 1]) <= tol_c * a1) ++j;
        int sz = j - i;
        if (sz == 2) {
            double k00 = d[3 * i + 0], k01 = d[3 * i + 1], k10 = d[3 * i + 2], k11 = d[3 * (i + 1) + 0];
            double det = k00 * k11 - k01 * k10;
            double sg = det >= 0.0 ? 1.0 : -1.0;
            double q00 = k00 + sg * k11, q01 = k01 - sg * k10;
            double q10 = k10 - sg * k01, q11 = k11 + sg * k00;
            double nrm = sqrt(q00 * q00 + q10 * q10);
            if (nrm > 1e-300) {
                q00 /= nrm; q01 /= nrm; q10 /= nrm; q11 /= nrm;
            } else {
                q00 = 1.0; q01 = 0.0; q10 = 0.0; q11 = 1.0;
            }
            Q[4 * i + 0] = q00; Q[4 * i + 1] = q10; Q[4 * i + 2] = q01; Q[4 * i + 3] = q11;
            kind[i] = 1;
            kind[i + 1] = 2;
        } else {
            for (int k = i; k < j; ++k) {
                Q[4 * k + 0] = (d[3 * k] < 0.0) ? -1.0 : 1.0;
                kind[k] = 0;
            }
        }
    }
}

// Z_c <- Z_c Q_c for every cluster, row-parallel.
__global__ void k_gauge_apply(int N, int b, double* __restrict__ Z, int ld, const double* __restrict__ Q,
                              const int* __restrict__ kind) {
    size_t tot = (size_t)N * b;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot;
         e += (size_t)gridDim.x * blockDim.x) {
        int r = (int)(e % N), i = (int)(e / N);
        int kd = kind[i];
        if (kd == 0) {
            Z[r + (size_t)ld * i] *= Q[4 * i];
        } else if (kd == 1) {
            double z0 = Z[r + (size_t)ld * i], z1 = Z[r + (size_t)ld * (i + 1)];
            // Q stored column-major: Q00, Q10, Q01, Q11
            Z[r + (size_t)ld * i] = Q[4 * i + 0] * z0 + Q[4 * i + 1] * z1;
            Z[r + (size_t)ld * (i + 1)] = Q[4 * i + 2] * z0 + Q[4 * i + 3] * z1;
        }
    }
}

// Counter-based Gaussian block (splitmix64 + Box-Muller) for cold starts.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__global__ void k_randn(int N, int b, double* __restrict__ V, int ld, uint64_t seed) {
    size_t tot = (size_t)N * b;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot;
         e += (size_t)gridDim.x * blockDim.x) {
        int r = (int)(e % N), i = (int)(e / N);
        uint64_t h1 = splitmix64(seed ^ (2 * e));
        uint64_t h2 = splitmix64(seed ^ (2 * e + 1));
        double u1 = ((h1 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        double u2 = (h2 >> 11) * (1.0 / 9007199254740992.0);
        V[r + (size_t)ld * i] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
    }
}

__global__ void k_identity_block(int N, int b, double* __restrict__ V, int ld) {
    size_t tot = (size_t)N * b;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot;
         e += (size_t)gridDim.x * blockDim.x) {
        int r = (int)(e % N), i = (int)(e / N);
        V[r + (size_t)ld * i] = (r == i) ? 1.0 : 0.0;
    }
}

inline int grid_for(size_t work, int threads = 256, int cap = 152 * 8) {
    size_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > (size_t)cap) g = cap;
    return (int)g;
}

cudaError_t launch_coop(const void* fn, int grid, int block, void** args, size_t smem, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace

int coop_grid_limit(const void* fn, int block, size_t smem) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, block, smem);
    if (per < 1) per = 1;
    return sms * per;
}

template <class JA>
cudaError_t jacobi_launch(cudaStream_t st, int n, const double* H, int ldh, EigWork& w, double* theta, double* Sout,
                          int ldo, int max_sweeps, DevCtl* ctl, double eps, double floor_rel, const int* skip,
                          int nhead) {
    using T = typename JA::T;
    static_assert(sizeof(T) == sizeof(double), "A and S buffers hold one 8-byte element each");
    int npad = n + (n & 1);
    if (npad < 2) npad = 2;
    T* A0 = (T*)w.A0;
    T* A1 = (T*)w.A1;
    T* S = (T*)w.S;
    k_jacobi_init<JA><<<grid_for((size_t)npad * npad), 256, 0, st>>>(n, npad, H, ldh, A0, S, w.rank, skip);
    cudaMemsetAsync(&ctl->rot_count[0], 0, sizeof(ctl->rot_count), st);
    cudaMemsetAsync(&ctl->jac_status, 0, sizeof(int), st);
    cudaMemsetAsync(&ctl->bar_count, 0, sizeof(unsigned int), st);
    if (max_sweeps > 64) max_sweeps = 64;
    const long half = npad / 2;
    const long nT = (half + JT - 1) / JT;
    const long nU = nT * (nT + 1) / 2 + nT * ((npad + JS_ROWS * JS_PASS - 1) / (JS_ROWS * JS_PASS));
    int grid = (int)nU;
    const size_t smem = 3 * (size_t)npad * sizeof(int);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    // two instantiations: two rounds per barrier (more registers, two blocks
    // per SM) and one round per barrier (fewer registers, more blocks)
    const void* fF = (const void*)k_jacobi<JA, true>;
    const void* fS = (const void*)k_jacobi<JA, false>;
    static std::mutex mu;  // host threads may drive handles concurrently
    static int limF = 0, limS = 0;
    static size_t limit_smem = 0;
    int lf, ls;
    {
        std::lock_guard<std::mutex> g(mu);
        if (limF == 0 || smem > limit_smem) {
            if (smem > 48 * 1024) {
                cudaFuncSetAttribute(fF, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                cudaFuncSetAttribute(fS, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            }
            limF = coop_grid_limit(fF, 256, smem);
            limS = coop_grid_limit(fS, 256, smem);
            limit_smem = smem;
        }
        lf = limF;
        ls = limS;
    }
    // two rounds per barrier only when every unit has its own block (and a
    // second S buffer exists): with several units per block (large n) the
    // recomputed rotations and the extra reads make a fused round cost more
    // than two single ones
    const bool fused = w.S1 != nullptr && nU <= lf;
    if (grid > (fused ? lf : ls)) grid = fused ? lf : ls;
    if (grid < 1) grid = 1;
    double fl = floor_rel > 0.0 ? floor_rel : 0.0;
    double* diag = w.diag;
    int* act = w.rank;  // the sweep tags; rank is rewritten by the sort below
    T* S1 = fused ? (T*)w.S1 : nullptr;  // NULL: one round per barrier, S in place
    int nh = (nhead > 0 && nhead < n) ? nhead : npad;
    void* args[] = {&n, &npad, &A0, &A1, &S, &S1, &diag, &act, &max_sweeps, &eps, &fl, &ctl, &skip, &nh};
    cudaError_t e = launch_coop(fused ? fF : fS, grid, 256, args, smem, st);
    if (e != cudaSuccess) return e;
    k_rank_ritz<<<grid_for((size_t)n), 256, 0, st>>>(n, w.diag, w.rank, theta);
    k_gather_ritz<JA><<<grid_for((size_t)n * n), 256, 0, st>>>(n, npad, w.rank, S, Sout, ldo);
    return cudaGetLastError();
}

cudaError_t jacobi_f64(cudaStream_t st, int n, const double* H, int ldh, EigWork& w, double* theta,
                       double* Sout, int ldo, int max_sweeps, DevCtl* ctl, double rel_tol, double floor_rel,
                       bool df, const int* skip, int nhead) {
    if (df) {
        // double-float: rotate while the coupling exceeds ~2^-46 of the
        // diagonal scale (four times the pair's unit roundoff)
        const double eps = rel_tol > 1.4210854715202004e-14 ? rel_tol : 1.4210854715202004e-14;
        return jacobi_launch<JDF>(st, n, H, ldh, w, theta, Sout, ldo, max_sweeps, ctl, eps, floor_rel, skip, nhead);
    }
    const double eps = rel_tol > 2.220446049250313e-16 ? rel_tol : 2.220446049250313e-16;
    return jacobi_launch<J64>(st, n, H, ldh, w, theta, Sout, ldo, max_sweeps, ctl, eps, floor_rel, skip, nhead);
}

cudaError_t cholesky_f64(cudaStream_t st, int n, double* G, int ld, double shift, DevCtl* ctl, bool df,
                         const int* skip) {
    // shift is relative: the kernel adds shift * trace(G) to the diagonal.
    // ctl->chol_status is sticky (atomicMax): the caller clears it.
    cudaMemsetAsync(&ctl->bar_count, 0, sizeof(unsigned int), st);
    static const int limit = std::min(coop_grid_limit((const void*)k_cholesky<C64>, 256, 0),
                                      coop_grid_limit((const void*)k_cholesky<CDF>, 256, 0));
    const long T = (n + 15) / 16;
    int grid = (int)std::max<long>(T * (T + 1) / 2, (n + 255) / 256);
    if (grid > limit) grid = limit;
    // one block per SM: measured 6% faster per factorisation than two
    // (fewer participants per grid barrier), and 76 blocks slower again
    if (grid > 152) grid = 152;
    if (grid < 1) grid = 1;
    void* args[] = {&n, &G, &ld, &shift, &ctl, &skip};
    return launch_coop(df ? (const void*)k_cholesky<CDF> : (const void*)k_cholesky<C64>, grid, 256, args, 0, st);
}

void trinv_f64(cudaStream_t st, int n, const double* L, int ld, double* X, int ldx, double* scratch,
               const int* skip, bool df) {
    // scratch: ceil(n / 32) * 1024 doubles (the diagonal blocks' inverses)
    const int nb = (n + 31) / 32;
    k_trinv_diag<<<nb, 32, 0, st>>>(n, L, ld, scratch, skip);
    const size_t smem = ((size_t)8 * nb * 32 + 3 * 32 * 33 + 8 * 32) * sizeof(double);
    static std::mutex mu;
    static size_t attr = 48 * 1024;
    {
        std::lock_guard<std::mutex> g(mu);
        if (smem > attr) {
            cudaFuncSetAttribute(k_trinv_cols<C64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            cudaFuncSetAttribute(k_trinv_cols<CDF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            attr = smem;
        }
    }
    if (df) k_trinv_cols<CDF><<<(n + 7) / 8, 256, smem, st>>>(n, L, ld, scratch, X, ldx, skip);
    else k_trinv_cols<C64><<<(n + 7) / 8, 256, smem, st>>>(n, L, ld, scratch, X, ldx, skip);
}

// X = (3 I - (G + G^t)/2) / 2.
__global__ void k_ns_coeff(int b, const double* __restrict__ G, int ldg, double* __restrict__ X, int ldx) {
    const size_t tot = (size_t)b * b;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % b), j = (int)(e / b);
        const double g = 0.5 * (G[i + (size_t)ldg * j] + G[j + (size_t)ldg * i]);
        X[i + (size_t)ldx * j] = (i == j ? 1.5 : 0.0) - 0.5 * g;
    }
}

void ns_coeff_f64(cudaStream_t st, int b, const double* G, int ldg, double* X, int ldx) {
    k_ns_coeff<<<grid_for((size_t)b * b), 256, 0, st>>>(b, G, ldg, X, ldx);
}

// One block: the defect d = max|G - I| of a Gram matrix; when d <= thresh it
// sets ctl->orth_ns and writes the Newton-Schulz coefficient X = (3I - G)/2
// (the factorisation behind it is then skipped), else clears the flag.
// max |G - I| over a b x b Gram matrix: a CTA per column, the maximum by an
// atomic max on the bits of the non-negative doubles (their order; a NaN's
// bits exceed every finite value's, so it propagates).
__global__ void __launch_bounds__(256) k_orth_max(int b, const double* __restrict__ G, int ldg, DevCtl* ctl) {
    __shared__ double red[8];
    const int j = blockIdx.x;
    double d = 0.0;
    for (int i = threadIdx.x; i < b; i += blockDim.x) {
        const double v = fabs(G[i + (size_t)ldg * j] - (i == j ? 1.0 : 0.0));
        d = (v > d || v != v) ? v : d;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double t = __shfl_xor_sync(0xffffffffu, d, o);
        d = (t > d || t != t) ? t : d;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = (red[w] > m || red[w] != red[w]) ? red[w] : m;
        atomicMax(&ctl->orth_max_bits, (unsigned long long)__double_as_longlong(m));
    }
}

// The decision and, below the threshold, X = (3I - G)/2 (G symmetrised).
__global__ void __launch_bounds__(256) k_orth_apply(int b, const double* __restrict__ G, int ldg, double thresh,
                                                    double* __restrict__ X, int ldx, DevCtl* ctl, int slot) {
    const double m = __longlong_as_double((long long)*(volatile unsigned long long*)&ctl->orth_max_bits);
    const int ns = (m <= thresh) ? 1 : 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->orth_ns = ns;
        ctl->orth_defect = (float)m;
        int k = 0;
        for (double t = 1.0; k < 9 && !(m >= t); t *= 0.1) ++k;
        atomicAdd(&ctl->orth_hist[slot ? 1 : 0][k], 1u);
    }
    if (!ns) return;
    const int j = blockIdx.x;
    for (int i = threadIdx.x; i < b; i += blockDim.x) {
        const double g = 0.5 * (G[i + (size_t)ldg * j] + G[j + (size_t)ldg * i]);
        X[i + (size_t)ldx * j] = (i == j ? 1.5 : 0.0) - 0.5 * g;
    }
}

void orth_check(cudaStream_t st, int b, const double* G, int ldg, double thresh, double* X, int ldx, DevCtl* ctl,
                int slot) {
    cudaMemsetAsync(&ctl->orth_max_bits, 0, sizeof(unsigned long long), st);
    k_orth_max<<<b, 256, 0, st>>>(b, G, ldg, ctl);
    k_orth_apply<<<b, 256, 0, st>>>(b, G, ldg, thresh, X, ldx, ctl, slot);
}

void resid_f64(cudaStream_t st, int N, int ncol, const double* T, const double* Z, int ld,
               const double* theta, double* res) {
    if (ncol <= 0) return;
    k_resid<<<ncol, 256, 0, st>>>(N, ncol, T, Z, ld, theta, res);
}

void decide(cudaStream_t st, int b, int L, int m, double tol, double tol_c, const double* theta,
            const double* res, DevCtl* ctl) {
    k_decide<<<1, 32, 0, st>>>(b, L, m, tol, tol_c, theta, res, ctl);
}

void next_block(cudaStream_t st, int N, int b, const double* T, const double* Z, int ld,
                const double* theta, double eps_theta, double* Vn) {
    col_combine(st, BM_NEXT, N, b, T, Z, Vn, ld, theta, eps_theta);
}

void cheb3_block(cudaStream_t st, int N, int b, const double* Y, const double* T, double* V, int ld,
                 const double* theta, double eps_theta) {
    col_combine(st, BM_CHEB3, N, b, Y, T, V, ld, theta, eps_theta);
}

void cheb2_block(cudaStream_t st, int N, int b, const double* Y, double* V, int ld, const double* theta,
                 double eps_theta) {
    col_combine(st, BM_CHEB2, N, b, Y, V, V, ld, theta, eps_theta);
}

void gauge_align(cudaStream_t st, int N, int b, double* Z, const double* V, int ld, const double* theta,
                 double tol_c, EigWork& w) {
    k_gauge_dots<<<b, 256, 0, st>>>(N, b, Z, V, ld, w.gdots);
    k_gauge_plan<<<(b + 127) / 128, 128, 0, st>>>(b, theta, tol_c, w.gdots, w.gQ, w.gkind);
    k_gauge_apply<<<grid_for((size_t)N * b), 256, 0, st>>>(N, b, Z, ld, w.gQ, w.gkind);
}

void randn_block(cudaStream_t st, int N, int b, double* V, int ld, uint64_t seed) {
    k_randn<<<grid_for((size_t)N * b), 256, 0, st>>>(N, b, V, ld, seed);
}

void identity_block(cudaStream_t st, int N, int b, double* V, int ld) {
    k_identity_block<<<grid_for((size_t)N * b), 256, 0, st>>>(N, b, V, ld);
}

}  // namespace ctm

// ---------------------------------------------------------------------------
// Warm-start Rayleigh-Ritz: simultaneous Jacobi rotations.
// For a warm start H = V^t C~ V is nearly diagonal.  Instead of sweeping the
// pairs one round at a time (a grid barrier per round), every pair (i, j) is
// rotated at once by its own Jacobi angle, taken from the current
//   S = X^t H X,  R = I - X^t X   (X = I at the start):
//   t_ij = tan of the angle that zeroes s_ij in the 2 x 2 problem
//          [[s_ii, s_ij], [s_ij, s_jj]] (its small root, |t| <= 1), for pairs
//          with |s_ij| > 64 eps sqrt|s_ii s_jj| (Jacobi's relative rule with a
//          margin that leaves rounding-level couplings inside exact
//          multiplets alone), else 0;
//   E_ij = t_ij + r_ij / 2,  E_ii = r_ii / 2;  X <- X (I + E).
// Only pairs with an index in the head (the kept states and the first
// discarded ones) are rotated; the oversampling tail keeps its basis and only
// has its orthonormality restored, so every column stays orthonormal.
// Pairs inside a multiplet are strongly coupled relative to their tiny gap
// (the other rotations mix them at second order); rotating them by their
// O(1) angle all at once would break the first-order scheme, so adjacent
// strongly coupled pairs are left alone and diagonalised exactly (one 2 x 2
// Jacobi rotation each, disjoint, hence commuting) after convergence.
// For well separated pairs t_ij = s_ij / (s_jj - s_ii) to first order and the
// iteration is the quadratically convergent refinement of Ogita & Aishima
// (Japan J. Indust. Appl. Math. 35, 2018); the r_ij / 2 terms restore
// orthonormality.  It stops when no head pair needs a rotation larger than
// tol and |I - X^t X| is below tol;
// if that does not happen within max_iter the host falls back to the
// cooperative Jacobi solver.
namespace ctm {
namespace {

// E for one refinement step.  Head pairs (an index below `head`) whose
// coupling is small against their diagonal gap, |s_ij| < gap / 10, get the
// Jacobi tangent of their 2 x 2 problem; an adjacent pair that is strongly
// coupled (an exact or near multiplet) is marked in clus[min(i, j)] and left
// for an exact rotation at the end; any other strongly coupled pair marks the
// refinement as failed (part[gridDim.x] = 1).
__global__ void k_oa_E(int b, int head, const double* __restrict__ S, const double* __restrict__ R,
                       double* __restrict__ E, double* __restrict__ part, int* __restrict__ clus) {
    __shared__ double red[32];
    __shared__ int s_bad;
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    double mx = 0.0;
    const double eps = 2.220446049250313e-16;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)b * b; e += (long)gridDim.x * blockDim.x) {
        int i = (int)(e % b), j = (int)(e / b);
        double rij = R ? 0.5 * (R[e] + R[j + (size_t)b * i]) : 0.0;
        double v = 0.5 * rij;
        mx = fmax(mx, fabs(rij));  // orthonormality must converge for every column
        if (i != j && (i < head || j < head)) {
            double sii = S[i + (size_t)b * i], sjj = S[j + (size_t)b * j];
            double c = 0.5 * (S[e] + S[j + (size_t)b * i]);
            double t = 0.0;
            if (c != 0.0 && fabs(c) > 64.0 * eps * sqrt(fabs(sii * sjj))) {
                double gap = sjj - sii;
                if (fabs(c) < 0.1 * fabs(gap)) {
                    double tau = gap / (2.0 * c);
                    if (fabs(tau) > 1e150) t = 0.5 / tau;
                    else t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                } else if (j == i + 1) {
                    clus[i] = 1;
                } else if (i != j + 1) {
                    s_bad = 1;
                }
            }
            v += t;
            mx = fmax(mx, fabs(t));
        }
        E[e] = v;
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
        mx = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (threadIdx.x == 0) part[blockIdx.x] = s_bad ? INFINITY : mx;
    }
}

// Exact rotations inside the marked doublets (disjoint pairs: they commute)
// and the Ritz values.  S = X^t H X of the converged X.  A triplet (two
// adjacent marks) cannot be handled here: ctl->oa_maxE = inf then.
__global__ void k_oa_clusters(int b, const double* __restrict__ S, const int* __restrict__ clus,
                              double* __restrict__ X, double* __restrict__ theta_unsorted, DevCtl* ctl) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)b * b; e += (long)gridDim.x * blockDim.x) {
        int row = (int)(e % b), i = (int)(e / b);
        bool first = clus[i] && i + 1 < b;
        bool second = i > 0 && clus[i - 1];
        if (first && second) {
            if (row == 0) ctl->oa_maxE = INFINITY;
            continue;
        }
        if (!first) {
            if (!second && row == 0) theta_unsorted[i] = S[i + (size_t)b * i];
            continue;
        }
        double a = S[i + (size_t)b * i], d = S[(i + 1) + (size_t)b * (i + 1)];
        double c = 0.5 * (S[i + (size_t)b * (i + 1)] + S[(i + 1) + (size_t)b * i]);
        double t = 0.0;
        if (c != 0.0) {
            double tau = (d - a) / (2.0 * c);
            if (fabs(tau) > 1e150) t = 0.5 / tau;
            else t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        }
        double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
        double xi = X[row + (size_t)b * i], xj = X[row + (size_t)b * (i + 1)];
        X[row + (size_t)b * i] = cs * xi - sn * xj;
        X[row + (size_t)b * (i + 1)] = sn * xi + cs * xj;
        if (row == 0) {
            theta_unsorted[i] = a - t * c;
            theta_unsorted[i + 1] = d + t * c;
        }
    }
}

// max over the partial maxima -> ctl->oa_maxE
__global__ void k_oa_finish(int nparts, const double* __restrict__ part, DevCtl* ctl) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double mx = 0.0;
    for (int i = 0; i < nparts; ++i) mx = fmax(mx, part[i]);
    ctl->oa_maxE = mx;
}

__global__ void k_identity_minus(int b, double* __restrict__ G) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)b * b; e += (long)gridDim.x * blockDim.x) {
        int i = (int)(e % b), j = (int)(e / b);
        G[e] = (i == j ? 1.0 : 0.0) - G[e];
    }
}

__global__ void k_copy_sym(int b, const double* __restrict__ H, int ldh, double* __restrict__ S) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)b * b; e += (long)gridDim.x * blockDim.x) {
        int i = (int)(e % b), j = (int)(e / b);
        S[e] = 0.5 * (H[i + (size_t)ldh * j] + H[j + (size_t)ldh * i]);
    }
}

__global__ void k_add_identity(int b, const double* __restrict__ E, double* __restrict__ X) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)b * b; e += (long)gridDim.x * blockDim.x) {
        int i = (int)(e % b), j = (int)(e / b);
        X[e] = (i == j ? 1.0 : 0.0) + E[e];
    }
}

inline int gfor(long work) {
    long g = (work + 255) / 256;
    if (g < 1) g = 1;
    if (g > 152 * 4) g = 152 * 4;
    return (int)g;
}

}  // namespace

int rr_refine_f64(cudaStream_t st, int b, int head, const double* H, int ldh, OaWork& w, EigWork& ew,
                  double* theta, double* Sout, int ldo, double tol, int max_iter, DevCtl* ctl, DevCtl* hctl,
                  int* nlaunch) {
    const long bb = (long)b * b;
    const int nparts = gfor(bb);
    w.fail_reason = 0;
    w.last_max = 0.0;
    w.last_iter = 0;
    // split-K for the b x b x b products: about 150 blocks, K chunks >= 32
    const int tiles = ((b + 63) / 64) * ((b + 63) / 64);
    int splits = std::max(1, std::min(std::min(w.max_splits, (2 * 152 + tiles - 1) / tiles), std::max(1, b / 32)));
    int nk = 0;
    // X = I + E(H): the first simultaneous rotation, from S = H and R = 0
    cudaMemsetAsync(w.clus, 0, sizeof(int) * b, st);
    k_copy_sym<<<gfor(bb), 256, 0, st>>>(b, H, ldh, w.S);
    k_oa_E<<<nparts, 256, 0, st>>>(b, head, w.S, nullptr, w.E, w.part, w.clus);
    k_add_identity<<<gfor(bb), 256, 0, st>>>(b, w.E, w.X);
    nk += 3;
    bool conv = false;
    int it = 1;
    for (; it <= max_iter; ++it) {
        // S = X^t (H X), R = I - X^t X
        nk += gemm_f64(st, false, false, b, b, b, 1.0, H, ldh, w.X, b, 0.0, w.W1, b, nullptr, splits, w.gpart);
        nk += gemm_f64(st, true, false, b, b, b, 1.0, w.X, b, w.W1, b, 0.0, w.S, b, nullptr, splits, w.gpart);
        nk += gemm_f64(st, true, false, b, b, b, 1.0, w.X, b, w.X, b, 0.0, w.R, b, nullptr, splits, w.gpart);
        k_identity_minus<<<gfor(bb), 256, 0, st>>>(b, w.R);
        cudaMemsetAsync(w.clus, 0, sizeof(int) * b, st);
        k_oa_E<<<nparts, 256, 0, st>>>(b, head, w.S, w.R, w.E, w.part, w.clus);
        k_oa_finish<<<1, 32, 0, st>>>(nparts, w.part, ctl);
        nk += 3;
        cudaMemcpyAsync(&hctl->oa_maxE, &ctl->oa_maxE, sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        const double mx = hctl->oa_maxE;
        w.last_max = mx;
        w.last_iter = it;
        if (!(mx <= 0.5)) {  // not a small correction any more: give up
            w.fail_reason = isinf(mx) ? 1 : 2;
            break;
        }
        // X <- X + X E (on convergence this only restores orthonormality)
        cudaMemcpyAsync(w.W1, w.X, sizeof(double) * bb, cudaMemcpyDeviceToDevice, st);
        nk += gemm_f64(st, false, false, b, b, b, 1.0, w.W1, b, w.E, b, 1.0, w.X, b, nullptr, splits, w.gpart);
        if (mx <= tol) {
            conv = true;
            break;
        }
    }
    if (!conv) {
        if (w.fail_reason == 0) w.fail_reason = 3;
        if (nlaunch) *nlaunch += nk;
        return -1;
    }
    // exact rotations inside the doublets, Ritz values, then sort by |theta|
    nk += gemm_f64(st, false, false, b, b, b, 1.0, H, ldh, w.X, b, 0.0, w.W1, b, nullptr, splits, w.gpart);
    nk += gemm_f64(st, true, false, b, b, b, 1.0, w.X, b, w.W1, b, 0.0, w.S, b, nullptr, splits, w.gpart);
    k_oa_clusters<<<gfor(bb), 256, 0, st>>>(b, w.S, w.clus, w.X, ew.diag, ctl);
    cudaMemcpyAsync(&hctl->oa_maxE, &ctl->oa_maxE, sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    nk += 1;
    if (nlaunch) *nlaunch += nk + 2;
    if (!(hctl->oa_maxE <= 0.5)) {  // a multiplet of three or more: use Jacobi
        w.fail_reason = 4;
        return -1;
    }
    k_rank_ritz<<<gfor(b), 256, 0, st>>>(b, ew.diag, ew.rank, theta);
    k_gather_ritz<J64><<<gfor(bb), 256, 0, st>>>(b, b, ew.rank, w.X, Sout, ldo);
    return it;
}

}  // namespace ctm
