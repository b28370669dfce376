// tangent.cu -- kernels of the forward-mode beta tangent of one CTMRG step
// (the derivative of the step of Algorithm 3 of arXiv:2004.08669).  The
// step's products reuse the FP64 GEMM and the vertex-weight contraction;
// the kernels here are the derivative of that contraction with respect to
// beta, the eigen tangent's coupling and deflated iteration, and the small
// reductions of the normalisation.
#include <cuda_runtime.h>
#include <math.h>

#include "tangent.cuh"

namespace ctm {

namespace {

inline int grid_of(size_t n, int per = 256, int cap = 152 * 8) {
    size_t b = (n + per - 1) / per;
    if (b < 1) b = 1;
    if (b > (size_t)cap) b = cap;
    return (int)b;
}

// One CTA per q x q block at a time (grid-stride over the live x live
// blocks), one thread per element.  With G = M o E, T1 = G E and the output
// form E o (E T1) (the same factor order as the contraction itself):
//   d out = Ed o (E T1) + E o (Ed T1) + E o (E T1d),
//   T1d = (M o Ed) E + (M o E) Ed,   Ed = (v.v) E = -Eh.
// With inner_h the inner factor is the bond-impurity table Eh = -(v.v) E
// (the energy inserted on one bond) instead of E, and its derivative
// d Eh / d beta = -(v.v)^2 E = -Eh^2 / E.
__global__ void k_wcontract_dbeta(int q, int live, const double* __restrict__ X, int ldx,
                                  const double* __restrict__ E, const double* __restrict__ Eh, int inner_h,
                                  double* __restrict__ out, int ldo) {
    extern __shared__ double sh[];
    const int q2 = q * q;
    double* sE = sh;
    double* sD = sE + q2;
    double* sI = sD + q2;
    double* sID = sI + q2;
    double* G = sID + q2;
    double* Gd = G + q2;
    double* T1 = Gd + q2;
    double* T1d = T1 + q2;
    for (int e = threadIdx.x; e < q2; e += blockDim.x) {
        const double ee = E[e], eh = Eh[e];
        sE[e] = ee;
        sD[e] = -eh;
        sI[e] = inner_h ? eh : ee;
        sID[e] = inner_h ? -eh * eh / ee : -eh;
    }
    __syncthreads();
    const int el = threadIdx.x;
    const bool act = el < q2;
    const int i = act ? el % q : 0, j = act ? el / q : 0;
    const long nblk = (long)live * live;
    for (long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        const int g = (int)(blk % live), gp = (int)(blk / live);
        const size_t off = (size_t)q * g + (size_t)ldx * ((size_t)q * gp);
        const size_t offo = (size_t)q * g + (size_t)ldo * ((size_t)q * gp);
        if (act) {
            const double x = X[off + i + (size_t)ldx * j];
            G[el] = x * sI[el];
            Gd[el] = x * sID[el];
        }
        __syncthreads();
        if (act) {
            double t = 0.0, td = 0.0;
            for (int k = 0; k < q; ++k) {
                t = fma(G[i + q * k], sE[k + q * j], t);
                td = fma(Gd[i + q * k], sE[k + q * j], td);
                td = fma(G[i + q * k], sD[k + q * j], td);
            }
            T1[el] = t;
            T1d[el] = td;
        }
        __syncthreads();
        if (act) {
            double a = 0.0, bd = 0.0, c = 0.0;
            for (int k = 0; k < q; ++k) {
                a = fma(sE[i + q * k], T1[k + q * j], a);
                bd = fma(sD[i + q * k], T1[k + q * j], bd);
                c = fma(sE[i + q * k], T1d[k + q * j], c);
            }
            out[offo + i + (size_t)ldo * j] += sD[el] * a + sE[el] * (bd + c);
        }
        __syncthreads();
    }
}

__global__ void k_mask_live(int N, int q, int live, double* __restrict__ A, int lda) {
    const size_t tot = (size_t)N * N;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e % N), c = (int)(e / N);
        if (r / q >= live || c / q >= live) A[r + (size_t)lda * c] = 0.0;
    }
}

__global__ void k_tangent_coupling(int bt, int n, const double* __restrict__ H, int ldh,
                                   const double* __restrict__ theta, double tol, double* __restrict__ K,
                                   double* __restrict__ lam_dot) {
    const double a0 = fabs(theta[0]);
    const int tot = bt * n;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x) {
        const int jj = e % bt, ii = e / bt;
        const double hs = 0.5 * (H[jj + (size_t)ldh * ii] + H[ii + (size_t)ldh * jj]);
        const double gap = theta[ii] - theta[jj];
        K[e] = (fabs(gap) <= tol * a0) ? 0.0 : hs / gap;
        if (jj == ii) lam_dot[ii] = hs;
    }
}

__global__ void k_deflate_update(int N, int n, const double* __restrict__ Rhs, const double* __restrict__ T,
                                 const double* __restrict__ theta, double* __restrict__ Y,
                                 double* __restrict__ part) {
    __shared__ double rc[32], ry[32];
    double mc = 0.0, my = 0.0;
    const size_t tot = (size_t)N * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / N);
        const double v = (Rhs[e] + (T ? T[e] : 0.0)) / theta[i];
        mc = fmax(mc, fabs(v - Y[e]));
        my = fmax(my, fabs(v));
        Y[e] = v;
    }
    for (int o = 16; o > 0; o >>= 1) {
        mc = fmax(mc, __shfl_xor_sync(0xffffffffu, mc, o));
        my = fmax(my, __shfl_xor_sync(0xffffffffu, my, o));
    }
    if ((threadIdx.x & 31) == 0) {
        rc[threadIdx.x >> 5] = mc;
        ry[threadIdx.x >> 5] = my;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a = fmax(a, rc[w]);
            b = fmax(b, ry[w]);
        }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

__global__ void k_dot_partial(size_t n, const double* __restrict__ x, const double* __restrict__ y,
                              double* __restrict__ part) {
    __shared__ double red[32];
    double s = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        s = fma(x[e], y[e], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += red[w];
        part[blockIdx.x] = a;
    }
}

__global__ void k_add_inplace(size_t n, const double* __restrict__ x, double* __restrict__ y) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        y[e] += x[e];
}

__global__ void k_tangent_normalise(size_t n, const double* __restrict__ R, const double* __restrict__ Rdot,
                                    double inv_k, double c, double* __restrict__ out) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        out[e] = Rdot[e] * inv_k - R[e] * c;
}

// out[i] = sum_t A[t, i] B[t, i] (w[t % q] when w is given: the spin of
// row t = s + q gamma), one CTA per column.
__global__ void k_column_dots(int N, int n, const double* __restrict__ A, int lda, const double* __restrict__ B,
                              int ldb, const double* __restrict__ w, int q, double* __restrict__ out) {
    __shared__ double red[32];
    const int i = blockIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
        const double v = A[t + (size_t)lda * i] * B[t + (size_t)ldb * i];
        s = fma(v, w ? w[t % q] : 1.0, s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) a += red[k];
        out[i] = a;
    }
}

}  // namespace

cudaError_t wcontract_dbeta(cudaStream_t st, int q, int live, const double* X, int ldx, const double* E,
                            const double* Eh, double* out, int ldo, bool inner_h) {
    const int q2 = q * q;
    if (q2 > 1024 || live < 1) return cudaErrorInvalidValue;
    const int threads = ((q2 + 31) / 32) * 32;
    const size_t smem = (size_t)8 * q2 * sizeof(double);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_wcontract_dbeta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const long nblk = (long)live * live;
    const int grid = (int)(nblk < 152 * 4 ? nblk : 152 * 4);
    k_wcontract_dbeta<<<grid, threads, smem, st>>>(q, live, X, ldx, E, Eh, inner_h ? 1 : 0, out, ldo);
    return cudaGetLastError();
}

void column_dots(cudaStream_t st, int N, int n, const double* A, int lda, const double* B, int ldb,
                 const double* wspin, int q, double* out) {
    k_column_dots<<<n, 256, 0, st>>>(N, n, A, lda, B, ldb, wspin, q, out);
}

void mask_live(cudaStream_t st, int N, int q, int live, double* A, int lda) {
    k_mask_live<<<grid_of((size_t)N * N), 256, 0, st>>>(N, q, live, A, lda);
}

void tangent_coupling(cudaStream_t st, int bt, int n, const double* H, int ldh, const double* theta, double tol,
                      double* K, double* lam_dot) {
    k_tangent_coupling<<<grid_of((size_t)bt * n), 256, 0, st>>>(bt, n, H, ldh, theta, tol, K, lam_dot);
}

void deflate_update(cudaStream_t st, int N, int n, const double* Rhs, const double* T, const double* theta,
                    double* Y, double* part) {
    k_deflate_update<<<kTanParts, 256, 0, st>>>(N, n, Rhs, T, theta, Y, part);
}

void dot_partial(cudaStream_t st, size_t n, const double* x, const double* y, double* part) {
    k_dot_partial<<<kTanParts, 256, 0, st>>>(n, x, y, part);
}

void add_inplace(cudaStream_t st, size_t n, const double* x, double* y) {
    k_add_inplace<<<grid_of(n), 256, 0, st>>>(n, x, y);
}

void tangent_normalise(cudaStream_t st, size_t n, const double* R, const double* Rdot, double inv_k, double c,
                       double* out) {
    k_tangent_normalise<<<grid_of(n), 256, 0, st>>>(n, R, Rdot, inv_k, c, out);
}

}  // namespace ctm
