// xi.cu -- kernels of the effective correlation length (Sec. II of
// arXiv:2004.08669): the renormalised row-to-row transfer matrix built from
// the fixed-point half-row tensor P, applied implicitly, and the vector
// operations of a Lanczos iteration on it.
//
// The row through the centre is the left half-row P, the centre vertex W and
// the right half-row P:
//   T[(a, t, a'), (g, u, g')] = sum_{s, s'} P(a, g, s) W(s, t, s', u) P(a', g', s'),
// W(a, b, c, d) = E_ab E_bc E_cd E_da (Eq. 1, cyclic corner order, E the
// bond weight).  T is symmetric (P(a, g, s) = P(g, a, s)) and of order m^2 q.
// In the device layout P(a, g, s) = P[a + m (s + q g)]; a vector of T's
// domain is X[g + m u + m q g'].  y = T x takes three steps (ctm.cu):
//   A1 (mq x qm) = Phat X, Phat = P read as (m q) x m with leading dim m q;
//   A2 = the centre-vertex contraction below;
//   Y  (mq x m)  = A2 P^t.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "xi.cuh"

namespace ctm {

namespace {

inline int blocks_for(size_t n, int per = 256, int cap = 152 * 8) {
    size_t b = (n + per - 1) / per;
    if (b < 1) b = 1;
    if (b > (size_t)cap) b = cap;
    return (int)b;
}

// A2[(a + m t) + mq (s' + q g')] = sum_{s,u} W(s, t, s', u) A1[(a + m s) + mq (u + q g')]
// for one g' (blockIdx.y) and a tile of `ta` values of a (blockIdx.x), using
//   W(s, t, s', u) = E(s, t) E(t, s') E(s', u) E(u, s):
//   G(s, s') = sum_u E(s', u) E(u, s) A1(s, u);  A2(t, s') = E(t, s') sum_s E(s, t) G(s, s').
// Shared memory: the slab X[s][u][i] (q^2 ta doubles) and E (q^2).
__global__ void __launch_bounds__(256) k_xi_w(int m, int q, int ta, const double* __restrict__ A1,
                                              const double* __restrict__ E, double* __restrict__ A2) {
    extern __shared__ double xsh[];
    double* X = xsh;                      // [s][u][i]
    double* Es = xsh + (size_t)q * q * ta;  // E[a + q b]
    const int a0 = blockIdx.x * ta, g2 = blockIdx.y;
    const size_t mq = (size_t)m * q;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < q * q; e += nt) Es[e] = E[e];
    const int tot = q * q * ta;
    for (int e = tid; e < tot; e += nt) {
        const int i = e % ta, su = e / ta;
        const int s = su % q, u = su / q;
        const int a = a0 + i;
        X[(s * q + u) * ta + i] = a < m ? A1[(a + (size_t)m * s) + mq * (u + (size_t)q * g2)] : 0.0;
    }
    __syncthreads();
    // G, one row s at a time, in place
    const int per_row = q * ta;
    for (int s = 0; s < q; ++s) {
        double g[4];
        int cnt = 0;
        for (int e = tid; e < per_row; e += nt, ++cnt) {
            const int i = e % ta, s2 = e / ta;
            double acc = 0.0;
            for (int u = 0; u < q; ++u) acc = fma(Es[s2 + q * u] * Es[u + q * s], X[(s * q + u) * ta + i], acc);
            g[cnt] = acc;
        }
        __syncthreads();
        cnt = 0;
        for (int e = tid; e < per_row; e += nt, ++cnt) {
            const int i = e % ta, s2 = e / ta;
            X[(s * q + s2) * ta + i] = g[cnt];
        }
        __syncthreads();
    }
    // A2(t, s') = E(t, s') sum_s E(s, t) G(s, s')
    for (int e = tid; e < tot; e += nt) {
        const int i = e % ta, ts = e / ta;
        const int t = ts % q, s2 = ts / q;
        const int a = a0 + i;
        double acc = 0.0;
        for (int s = 0; s < q; ++s) acc = fma(Es[s + q * t], X[(s * q + s2) * ta + i], acc);
        if (a < m) A2[(a + (size_t)m * t) + mq * (s2 + (size_t)q * g2)] = Es[t + q * s2] * acc;
    }
}

// part[j * nb + blk] = partial sum over this block's rows of V[:, j] . w
__global__ void k_dots_partial(size_t n, const double* __restrict__ V, size_t ldv, const double* __restrict__ w,
                               double* __restrict__ part) {
    const int j = blockIdx.y;
    const double* v = V + ldv * j;
    double acc = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        acc = fma(v[e], w[e], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
        part[(size_t)j * gridDim.x + blockIdx.x] = s;
    }
}

// out[j] = sum over blocks of part[j * nb + blk], in block order
__global__ void k_dots_final(int k, int nb, const double* __restrict__ part, double* __restrict__ out) {
    const int j = blockIdx.x;
    if (j >= k) return;
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += part[(size_t)j * nb + b];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        out[j] = s;
    }
}

// w -= sum_{j < k} V[:, j] c[j]
__global__ void k_sub_multi(size_t n, int k, const double* __restrict__ V, size_t ldv, const double* __restrict__ c,
                            double* __restrict__ w) {
    __shared__ double cs[128];
    for (int j = threadIdx.x; j < k; j += blockDim.x) cs[j] = c[j];
    __syncthreads();
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        double acc = w[e];
        for (int j = 0; j < k; ++j) acc = fma(-V[e + ldv * j], cs[j], acc);
        w[e] = acc;
    }
}

// beta_j = ||w|| (from dot[0] = w . w); v_next = w / beta_j; records beta
__global__ void k_normalise(size_t n, const double* __restrict__ w, const double* __restrict__ dot,
                            double* __restrict__ vnext, double* __restrict__ beta_out) {
    const double b = sqrt(fmax(dot[0], 0.0));
    if (blockIdx.x == 0 && threadIdx.x == 0) *beta_out = b;
    const double inv = b > 0.0 ? 1.0 / b : 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        vnext[e] = w[e] * inv;
}

// Tridiagonal Lanczos matrix (k x k, column-major): alpha on the diagonal,
// beta[0..k-2] beside it.
__global__ void k_tridiag(int k, const double* __restrict__ alpha, const double* __restrict__ beta,
                          double* __restrict__ Tk) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < k * k; e += gridDim.x * blockDim.x) {
        const int i = e % k, j = e / k;
        double v = 0.0;
        if (i == j) v = alpha[i];
        else if (i == j + 1) v = beta[j];
        else if (j == i + 1) v = beta[i];
        Tk[e] = v;
    }
}

}  // namespace

size_t xi_w_smem(int q, int* ta) {
    const int t = (q <= 24) ? 32 : 16;
    if (ta) *ta = t;
    return ((size_t)q * q * t + (size_t)q * q) * sizeof(double);
}

cudaError_t xi_wcontract(cudaStream_t st, int m, int q, const double* A1, const double* E, double* A2) {
    int ta = 0;
    const size_t smem = xi_w_smem(q, &ta);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_xi_w, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((m + ta - 1) / ta, m);
    k_xi_w<<<grid, 256, smem, st>>>(m, q, ta, A1, E, A2);
    return cudaGetLastError();
}

int xi_dots_blocks(size_t n) { return blocks_for(n, 256, 152 * 2); }

void xi_dots(cudaStream_t st, size_t n, int k, const double* V, size_t ldv, const double* w, double* part,
             double* out) {
    const int nb = xi_dots_blocks(n);
    k_dots_partial<<<dim3(nb, k), 256, 0, st>>>(n, V, ldv, w, part);
    k_dots_final<<<k, 256, 0, st>>>(k, nb, part, out);
}

void xi_sub_multi(cudaStream_t st, size_t n, int k, const double* V, size_t ldv, const double* c, double* w) {
    k_sub_multi<<<blocks_for(n), 256, 0, st>>>(n, k, V, ldv, c, w);
}

void xi_normalise(cudaStream_t st, size_t n, const double* w, const double* dot, double* vnext, double* beta_out) {
    k_normalise<<<blocks_for(n), 256, 0, st>>>(n, w, dot, vnext, beta_out);
}

void xi_tridiag(cudaStream_t st, int k, const double* alpha, const double* beta, double* Tk) {
    k_tridiag<<<blocks_for((size_t)k * k), 256, 0, st>>>(k, alpha, beta, Tk);
}

}  // namespace ctm
