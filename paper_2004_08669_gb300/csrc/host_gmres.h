// host_gmres.h -- GMRES without restarts on host vectors, for the linear
// fixed-point equation (I - J) x = b of the implicit derivative, where each
// application of the operator is one tangent step on the device.
//
// Arnoldi with modified Gram-Schmidt applied twice, Givens rotations for the
// small least-squares problem, back substitution at the end (Saad and
// Schultz's method).  Plain C++: no CUDA, so it is tested on the host alone.
#pragma once

#include <cmath>
#include <cstddef>
#include <vector>

namespace ctm {

enum { kGmresOk = 0, kGmresNotConverged = 1, kGmresOpFailed = 2 };

// op(v, w) writes w = A v and returns false on failure.  Solves A x = rhs to
// a relative residual tol in at most max_iter iterations; x is overwritten.
template <class Op>
int host_gmres(Op op, const std::vector<double>& rhs, std::vector<double>& x, double tol, int max_iter,
               int* iters, double* rel_res) {
    const size_t n = rhs.size();
    double b0 = 0.0;
    for (double v : rhs) b0 += v * v;
    b0 = std::sqrt(b0);
    x.assign(n, 0.0);
    *iters = 0;
    *rel_res = 0.0;
    if (b0 == 0.0) return kGmresOk;
    std::vector<std::vector<double>> V(1, std::vector<double>(n));
    for (size_t i = 0; i < n; ++i) V[0][i] = rhs[i] / b0;
    std::vector<std::vector<double>> H;  // columns of the rotated Hessenberg matrix
    std::vector<double> cs, sn, g(1, b0), w(n);
    int k = 0;
    double res = 1.0;
    for (k = 0; k < max_iter; ++k) {
        if (!op(V[k], w)) return kGmresOpFailed;
        std::vector<double> hk(k + 2, 0.0);
        for (int pass = 0; pass < 2; ++pass)
            for (int j = 0; j <= k; ++j) {
                double hj = 0.0;
                for (size_t i = 0; i < n; ++i) hj += V[j][i] * w[i];
                hk[j] += hj;
                for (size_t i = 0; i < n; ++i) w[i] -= hj * V[j][i];
            }
        double nw = 0.0;
        for (double v : w) nw += v * v;
        nw = std::sqrt(nw);
        hk[k + 1] = nw;
        for (int j = 0; j < k; ++j) {  // the earlier rotations
            const double t = cs[j] * hk[j] + sn[j] * hk[j + 1];
            hk[j + 1] = -sn[j] * hk[j] + cs[j] * hk[j + 1];
            hk[j] = t;
        }
        const double r = std::hypot(hk[k], hk[k + 1]);
        const double ck = r > 0.0 ? hk[k] / r : 1.0, sk = r > 0.0 ? hk[k + 1] / r : 0.0;
        cs.push_back(ck);
        sn.push_back(sk);
        hk[k] = r;
        hk[k + 1] = 0.0;
        g.push_back(-sk * g[k]);
        g[k] = ck * g[k];
        H.push_back(hk);
        res = std::fabs(g[k + 1]) / b0;
        if (res <= tol || nw == 0.0) {
            ++k;
            break;
        }
        V.emplace_back(n);
        for (size_t i = 0; i < n; ++i) V[k + 1][i] = w[i] / nw;
    }
    *rel_res = res;
    if (res > tol) return kGmresNotConverged;
    std::vector<double> y(k, 0.0);
    for (int i = k - 1; i >= 0; --i) {
        double acc = g[i];
        for (int j = i + 1; j < k; ++j) acc -= H[j][i] * y[j];
        y[i] = acc / H[i][i];
    }
    for (int j = 0; j < k; ++j)
        for (size_t i = 0; i < n; ++i) x[i] += y[j] * V[j][i];
    *iters = k;
    return kGmresOk;
}

}  // namespace ctm
