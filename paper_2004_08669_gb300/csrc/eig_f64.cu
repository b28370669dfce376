// eig_f64.cu -- FP64 kernels of the leading-eigenpair stage of a CTMRG step.
//
// The paper diagonalises the whole extended corner (Algorithm 3, the
// EigenExa call, with a dense solver).  Here only its leading b = m + p
// eigenpairs are computed, by block subspace iteration:
//   Y = C~ V;  H = V^t Y;  H = S Theta S^t (cyclic Jacobi, FP64);
//   Z = V S;  T = Y S;  residual ||T_i - theta_i Z_i||;
//   V <- orth([T_i / theta_i or Z_i]) by (shifted) Cholesky QR.
// The kernels below are the small dense FP64 pieces: a parallel-order
// two-sided Jacobi eigensolver (Golub & Van Loan 8.5, round-robin ordering),
// a blocked Cholesky factorisation, a triangular inverse, the residual test
// with the multiplet-aware truncation rule, and the gauge alignment of Ritz
// vectors to the previous step's (sign per singlet, orthogonal Procrustes per
// doublet) that keeps the renormalised basis consistent between steps.
#include "ctm_internal.cuh"
#include "eig_f64.cuh"

#include <math.h>

namespace ctm {

namespace {

__device__ __forceinline__ void rr_pair(int r, int k, int npad, int& p, int& q) {
    const int n1 = npad - 1;
    if (k == 0) {
        p = n1;
        q = r;
    } else {
        p = (r + k) % n1;
        q = (r - k + n1) % n1;
    }
}

struct Rot {
    double c, s, t;
    bool on;
};

__device__ __forceinline__ Rot rot_of(const double* A, int ld, int p, int q, double eps,
                                      double floor_abs) {
    Rot R{1.0, 0.0, 0.0, false};
    double apq = __ldcg(A + p + (size_t)ld * q);
    if (apq == 0.0) return R;
    double app = __ldcg(A + p + (size_t)ld * p), aqq = __ldcg(A + q + (size_t)ld * q);
    if (fabs(apq) <= fmax(eps * sqrt(fabs(app * aqq)), floor_abs)) return R;
    double tau = (aqq - app) / (2.0 * apq);
    double t;
    if (fabs(tau) > 1e150) t = 0.5 / tau;
    else t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
    R.c = 1.0 / sqrt(1.0 + t * t);
    R.s = t * R.c;
    R.t = t;
    R.on = true;
    return R;
}

__global__ void k_jacobi_init(int n, int npad, const double* __restrict__ H, int ldh,
                              double* __restrict__ A0, double* __restrict__ S) {
    size_t tot = (size_t)npad * npad;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot;
         e += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(e % npad), j = (int)(e / npad);
        double v = 0.0;
        if (i < n && j < n) v = 0.5 * (H[i + (size_t)ldh * j] + H[j + (size_t)ldh * i]);
        A0[e] = v;
        S[e] = (i == j) ? 1.0 : 0.0;
    }
}

// Cooperative: all blocks co-resident (cudaLaunchAttributeCooperative).
__global__ void k_jacobi(int n, int npad, double* A0, double* A1,
                         double* S, double* __restrict__ diag, int max_sweeps,
                         double eps, double floor_abs, DevCtl* ctl) {
    const int half = npad / 2;
    const long nblk_items = (long)half * half;
    const long nS_items = (long)npad * half;
    const long W = nblk_items + nS_items;
    const long gtid = blockIdx.x * (long)blockDim.x + threadIdx.x;
    const long gstride = (long)gridDim.x * blockDim.x;
    int* err = &ctl->jac_status;
    long round_total = 0;
    int sweep = 0;
    bool converged = false;
    for (sweep = 0; sweep < max_sweeps && !converged; ++sweep) {
        for (int r = 0; r < npad - 1; ++r, ++round_total) {
            const double* Ac = (round_total & 1) ? A1 : A0;
            double* An = (round_total & 1) ? A0 : A1;
            for (long it = gtid; it < W; it += gstride) {
                if (it < nblk_items) {
                    int ka = (int)(it % half), kb = (int)(it / half);
                    int p, q, rr, tt;
                    rr_pair(r, ka, npad, p, q);
                    rr_pair(r, kb, npad, rr, tt);
                    Rot Ra = rot_of(Ac, npad, p, q, eps, floor_abs);
                    if (ka == kb) {
                        double app = __ldcg(Ac + p + (size_t)npad * p);
                        double aqq = __ldcg(Ac + q + (size_t)npad * q);
                        double apq = __ldcg(Ac + p + (size_t)npad * q);
                        if (Ra.on) {
                            An[p + (size_t)npad * p] = app - Ra.t * apq;
                            An[q + (size_t)npad * q] = aqq + Ra.t * apq;
                            An[p + (size_t)npad * q] = 0.0;
                            An[q + (size_t)npad * p] = 0.0;
                            atomicAdd(&ctl->rot_count[sweep], 1);
                        } else {
                            An[p + (size_t)npad * p] = app;
                            An[q + (size_t)npad * q] = aqq;
                            An[p + (size_t)npad * q] = apq;
                            An[q + (size_t)npad * p] = __ldcg(Ac + q + (size_t)npad * p);
                        }
                    } else {
                        Rot Rb = rot_of(Ac, npad, rr, tt, eps, floor_abs);
                        double a_pr = __ldcg(Ac + p + (size_t)npad * rr);
                        double a_pt = __ldcg(Ac + p + (size_t)npad * tt);
                        double a_qr = __ldcg(Ac + q + (size_t)npad * rr);
                        double a_qt = __ldcg(Ac + q + (size_t)npad * tt);
                        // J_a^t from the left (rows p, q)
                        double x_pr = Ra.c * a_pr - Ra.s * a_qr, x_pt = Ra.c * a_pt - Ra.s * a_qt;
                        double x_qr = Ra.s * a_pr + Ra.c * a_qr, x_qt = Ra.s * a_pt + Ra.c * a_qt;
                        // J_b from the right (columns r, t)
                        An[p + (size_t)npad * rr] = Rb.c * x_pr - Rb.s * x_pt;
                        An[p + (size_t)npad * tt] = Rb.s * x_pr + Rb.c * x_pt;
                        An[q + (size_t)npad * rr] = Rb.c * x_qr - Rb.s * x_qt;
                        An[q + (size_t)npad * tt] = Rb.s * x_qr + Rb.c * x_qt;
                    }
                } else {
                    long e = it - nblk_items;
                    int row = (int)(e % npad), k = (int)(e / npad);
                    int p, q;
                    rr_pair(r, k, npad, p, q);
                    Rot Ra = rot_of(Ac, npad, p, q, eps, floor_abs);
                    if (Ra.on) {
                        double sp = __ldcg(S + row + (size_t)npad * p);
                        double sq = __ldcg(S + row + (size_t)npad * q);
                        S[row + (size_t)npad * p] = Ra.c * sp - Ra.s * sq;
                        S[row + (size_t)npad * q] = Ra.s * sp + Ra.c * sq;
                    }
                }
            }
            if (!grid_barrier(&ctl->bar_count, &ctl->bar_gen, gridDim.x, err)) return;
        }
        converged = (*(volatile int*)&ctl->rot_count[sweep]) == 0;
    }
    const double* Af = (round_total & 1) ? A1 : A0;
    for (long i = gtid; i < n; i += gstride) diag[i] = __ldcg(Af + i + (size_t)npad * i);
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

__global__ void k_gather_ritz(int n, int npad, const int* __restrict__ rank, const double* __restrict__ S,
                              double* __restrict__ Sout, int ldo) {
    size_t tot = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot;
         e += (size_t)gridDim.x * blockDim.x) {
        int row = (int)(e % n), j = (int)(e / n);
        Sout[row + (size_t)ldo * rank[j]] = S[row + (size_t)npad * j];
    }
}

// Blocked right-looking Cholesky G + shift I = L L^t (lower, in place),
// panel width 32.  Cooperative launch.
__global__ void k_cholesky(int n, double* G, int ld, double shift_rel, DevCtl* ctl) {
    __shared__ double D[32][33];
    int* err = &ctl->chol_status;
    const long gtid = blockIdx.x * (long)blockDim.x + threadIdx.x;
    const long gstride = (long)gridDim.x * blockDim.x;
    double shift = 0.0;
    if (shift_rel > 0.0) {
        for (int i = 0; i < n; ++i) shift += G[i + (size_t)ld * i];
        shift *= shift_rel;
    }
    if (!grid_barrier(&ctl->bar_count, &ctl->bar_gen, gridDim.x, err)) return;
    if (shift != 0.0)
        for (long i = gtid; i < n; i += gstride) G[i + (size_t)ld * i] = __ldcg(G + i + (size_t)ld * i) + shift;
    if (!grid_barrier(&ctl->bar_count, &ctl->bar_gen, gridDim.x, err)) return;
    for (int k0 = 0; k0 < n; k0 += 32) {
        const int kb = min(32, n - k0);
        if (blockIdx.x == 0) {
            for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
                int i = e % kb, j = e / kb;
                D[i][j] = __ldcg(G + (k0 + i) + (size_t)ld * (k0 + j));
            }
            __syncthreads();
            for (int j = 0; j < kb; ++j) {
                if (threadIdx.x == 0) {
                    double d = D[j][j];
                    if (!(d > 0.0) || !isfinite(d)) {
                        atomicMax(err, 1);
                        d = 1.0;
                    }
                    D[j][j] = sqrt(d);
                }
                __syncthreads();
                for (int i = j + 1 + threadIdx.x; i < kb; i += blockDim.x) D[i][j] /= D[j][j];
                __syncthreads();
                for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
                    int i = e % kb, l = e / kb;
                    if (l > j && i >= l) D[i][l] -= D[i][j] * D[l][j];
                }
                __syncthreads();
            }
            for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
                int i = e % kb, j = e / kb;
                G[(k0 + i) + (size_t)ld * (k0 + j)] = (i >= j) ? D[i][j] : 0.0;
            }
        }
        if (!grid_barrier(&ctl->bar_count, &ctl->bar_gen, gridDim.x, err)) return;
        const int k1 = k0 + kb;
        if (k1 >= n) break;
        // panel solve: rows below the diagonal block
        for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
            int i = e % kb, j = e / kb;
            D[i][j] = __ldcg(G + (k0 + i) + (size_t)ld * (k0 + j));
        }
        __syncthreads();
        for (long i = k1 + gtid; i < n; i += gstride) {
            double x[32];
            for (int j = 0; j < kb; ++j) {
                double s = __ldcg(G + i + (size_t)ld * (k0 + j));
                for (int l = 0; l < j; ++l) s -= x[l] * D[j][l];
                x[j] = s / D[j][j];
            }
            for (int j = 0; j < kb; ++j) G[i + (size_t)ld * (k0 + j)] = x[j];
        }
        __syncthreads();
        if (!grid_barrier(&ctl->bar_count, &ctl->bar_gen, gridDim.x, err)) return;
        // trailing update of the lower triangle
        const long nt = n - k1;
        for (long e = gtid; e < nt * nt; e += gstride) {
            int i = k1 + (int)(e % nt), j = k1 + (int)(e / nt);
            if (j > i) continue;
            double s = 0.0;
            for (int l = 0; l < kb; ++l)
                s += __ldcg(G + i + (size_t)ld * (k0 + l)) * __ldcg(G + j + (size_t)ld * (k0 + l));
            G[i + (size_t)ld * j] = __ldcg(G + i + (size_t)ld * j) - s;
        }
        if (!grid_barrier(&ctl->bar_count, &ctl->bar_gen, gridDim.x, err)) return;
    }
}

// Linv = L^{-1} (lower triangular), one warp per column.
__global__ void k_trinv(int n, const double* __restrict__ L, int ld, double* __restrict__ X, int ldx) {
    extern __shared__ double xs[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    double* x = xs + (size_t)warp * n;
    for (int j = blockIdx.x * wpb + warp; j < n; j += gridDim.x * wpb) {
        for (int i = lane; i < j; i += 32) X[i + (size_t)ldx * j] = 0.0;
        double xj = 1.0 / L[j + (size_t)ld * j];
        if (lane == 0) x[j] = xj;
        __syncwarp();
        for (int i = j + 1; i < n; ++i) {
            double s = 0.0;
            for (int k = j + lane; k < i; k += 32) s += L[i + (size_t)ld * k] * x[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            double xi = -s / L[i + (size_t)ld * i];
            __syncwarp();
            if (lane == 0) x[i] = xi;
            __syncwarp();
        }
        for (int i = j + lane; i < n; i += 32) X[i + (size_t)ldx * j] = x[i];
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
    ctl->sub_converged = (!bad && rmax <= tol * a1) ? 1 : 0;
    if (bad) ctl->numeric_bad = 1;
}

// Next block before re-orthonormalisation: T_i / theta_i, or Z_i when
// |theta_i| is negligible (keeps the Gram matrix well conditioned).
__global__ void k_next_block(int N, int b, const double* __restrict__ T, const double* __restrict__ Z,
                             int ld, const double* __restrict__ theta, double eps_theta,
                             double* __restrict__ Vn) {
    double a1 = fabs(theta[0]);
    size_t tot = (size_t)N * b;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot;
         e += (size_t)gridDim.x * blockDim.x) {
        int r = (int)(e % N), i = (int)(e / N);
        double th = theta[i];
        size_t o = r + (size_t)ld * i;
        Vn[o] = (fabs(th) > eps_theta * a1) ? T[o] / th : Z[o];
    }
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
__global__ void k_gauge_plan(int b, const double* __restrict__ theta, double tol_c,
                             const double* __restrict__ d, double* __restrict__ Q, int* __restrict__ kind) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a1 = fabs(theta[0]);
    int i = 0;
    while (i < b) {
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
        i = j;
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

cudaError_t jacobi_f64(cudaStream_t st, int n, const double* H, int ldh, EigWork& w, double* theta,
                       double* Sout, int ldo, int max_sweeps, DevCtl* ctl) {
    int npad = n + (n & 1);
    if (npad < 2) npad = 2;
    k_jacobi_init<<<grid_for((size_t)npad * npad), 256, 0, st>>>(n, npad, H, ldh, w.A0, w.S);
    cudaMemsetAsync(&ctl->rot_count[0], 0, sizeof(ctl->rot_count), st);
    cudaMemsetAsync(&ctl->jac_status, 0, sizeof(int), st);
    if (max_sweeps > 64) max_sweeps = 64;
    long half = npad / 2;
    long W = half * half + (long)npad * half;
    int grid = (int)((W + 255) / 256);
    static int limit = 0;
    if (limit == 0) limit = coop_grid_limit((const void*)k_jacobi, 256, 0);
    if (grid > limit) grid = limit;
    if (grid < 1) grid = 1;
    double eps = 2.220446049250313e-16, floor_abs = 0.0;
    double* A0 = w.A0;
    double* A1 = w.A1;
    double* S = w.S;
    double* diag = w.diag;
    void* args[] = {&n, &npad, &A0, &A1, &S, &diag, &max_sweeps, &eps, &floor_abs, &ctl};
    cudaError_t e = launch_coop((const void*)k_jacobi, grid, 256, args, 0, st);
    if (e != cudaSuccess) return e;
    k_rank_ritz<<<grid_for((size_t)n), 256, 0, st>>>(n, w.diag, w.rank, theta);
    k_gather_ritz<<<grid_for((size_t)n * n), 256, 0, st>>>(n, npad, w.rank, w.S, Sout, ldo);
    return cudaGetLastError();
}

cudaError_t cholesky_f64(cudaStream_t st, int n, double* G, int ld, double shift, DevCtl* ctl) {
    // shift is relative: the kernel adds shift * trace(G) to the diagonal
    cudaMemsetAsync(&ctl->chol_status, 0, sizeof(int), st);
    static int limit = 0;
    if (limit == 0) limit = coop_grid_limit((const void*)k_cholesky, 256, 0);
    long work = (long)n * n / 2;
    int grid = (int)((work + 255) / 256);
    if (grid > limit) grid = limit;
    if (grid > 152) grid = 152;
    if (grid < 1) grid = 1;
    void* args[] = {&n, &G, &ld, &shift, &ctl};
    return launch_coop((const void*)k_cholesky, grid, 256, args, 0, st);
}

void trinv_f64(cudaStream_t st, int n, const double* L, int ld, double* X, int ldx) {
    const int wpb = 4;
    int grid = (n + wpb - 1) / wpb;
    size_t smem = (size_t)wpb * n * sizeof(double);
    k_trinv<<<grid, 32 * wpb, smem, st>>>(n, L, ld, X, ldx);
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
    k_next_block<<<grid_for((size_t)N * b), 256, 0, st>>>(N, b, T, Z, ld, theta, eps_theta, Vn);
}

void gauge_align(cudaStream_t st, int N, int b, double* Z, const double* V, int ld, const double* theta,
                 double tol_c, EigWork& w) {
    k_gauge_dots<<<b, 256, 0, st>>>(N, b, Z, V, ld, w.gdots);
    k_gauge_plan<<<1, 32, 0, st>>>(b, theta, tol_c, w.gdots, w.gQ, w.gkind);
    k_gauge_apply<<<grid_for((size_t)N * b), 256, 0, st>>>(N, b, Z, ld, w.gQ, w.gkind);
}

void randn_block(cudaStream_t st, int N, int b, double* V, int ld, uint64_t seed) {
    k_randn<<<grid_for((size_t)N * b), 256, 0, st>>>(N, b, V, ld, seed);
}

void identity_block(cudaStream_t st, int N, int b, double* V, int ld) {
    k_identity_block<<<grid_for((size_t)N * b), 256, 0, st>>>(N, b, V, ld);
}

}  // namespace ctm
