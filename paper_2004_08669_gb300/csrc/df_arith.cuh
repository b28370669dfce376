// df_arith.cuh -- rotation arithmetic shared by the small dense solvers of
// the eigen stage: the Jacobi rotation of a 2 x 2 symmetric problem (FP64
// with an FP32 tangent) and the two arithmetic policies of the solvers, J64
// (FP64) and JDF (double-float pairs of FP32 words on the FP32 pipe).
#pragma once

#include <cuda_runtime.h>
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
    double c, s;
    bool on;
};

// A pair is rotated while its coupling exceeds eps relative to the geometric
// mean of its diagonal entries (the criterion that keeps relative accuracy for
// graded matrices) and an absolute floor.  The comparison is made on squares
// when they are safely representable, so that no FP64 square root (slow on
// this part) is taken per pair.
__device__ __forceinline__ bool jac_above(double app, double aqq, double apq, double eps, double floor_abs) {
    if (apq == 0.0) return false;
    const double a = fabs(apq);
    if (!(a > floor_abs)) return false;
    const double pr = fabs(app * aqq), a2 = apq * apq;
    if (pr > 1e-290 && pr < 1e290 && a2 > 1e-290 && a2 < 1e290) return a2 > (eps * eps) * pr;
    return a > eps * sqrt(pr);
}

// Rotation of the pair (p, q) (Golub & Van Loan 8.5.2): tau = (a_qq - a_pp) /
// (2 a_pq), t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1 + t^2),
// s = t c.  The tangent is taken in FP32: an approximate angle leaves ~1e-7
// of a_pq instead of zero, which the next sweep removes, so convergence is
// unaffected.  c must be FP64-accurate for the rotation to be orthogonal to
// FP64 rounding: an FP32 reciprocal square root y0 of x = 1 + t^2 is refined
// by one Newton-Raphson step y <- y + y (1 - x y^2) / 2 in double-float
// arithmetic on the FP32 pipe (x and y0^2 split exactly by FMA), and then by
// one step in FP64; s = t c.  This keeps the dependent FP64 chain, slow on
// this part, to a few operations.
__device__ __forceinline__ Rot rot_fast(double app, double aqq, double apq, double eps, double floor_abs) {
    Rot R{1.0, 0.0, false};
    if (!jac_above(app, aqq, apq, eps, floor_abs)) return R;
    const double d = aqq - app;
    const double aa = fabs(apq), ad = fabs(d);
    double t;
    if (aa > 1e-30 && aa < 1e30 && ad < 1e30 && ad < 1e18 * aa) {
        const float tau = (float)d / (float)(2.0 * apq);
        t = (double)(copysignf(1.0f, tau) / (fabsf(tau) + sqrtf(1.0f + tau * tau)));
    } else {  // extreme scales or |tau| beyond 5e17: the FP64 formula
        const double tau = d / (2.0 * apq);
        t = fabs(tau) > 1e150 ? 0.5 / tau : copysign(1.0, tau) / (fabs(tau) + sqrt(1.0 + tau * tau));
    }
    const double x = fma(t, t, 1.0);
    double y;
    const float tf = (float)t;
    if ((double)tf == t && fabsf(tf) <= 1.0f) {
        // x = 1 + t^2 as xh + xl (exact: |t| <= 1, t^2 split by FMA)
        const float t2 = tf * tf, t2e = fmaf(tf, tf, -t2);
        const float xh = 1.0f + t2, xl = ((1.0f - xh) + t2) + t2e;
        const float y0 = rsqrtf(xh);
        // r = 1 - x y0^2 to ~2^-46 (y0^2 and xh y0^2 split by FMA)
        const float p = y0 * y0, pe = fmaf(y0, y0, -p);
        const float q = xh * p, qe = fmaf(xh, p, -q) + fmaf(xh, pe, xl * p);
        const float r = (1.0f - q) - qe;
        y = (double)y0 + (double)(0.5f * y0 * r);
    } else {
        y = (double)rsqrtf((float)x);
        y = y * (1.5 - 0.5 * x * y * y);
    }
    y = y * (1.5 - 0.5 * x * y * y);
    R.c = y;
    R.s = t * y;
    R.on = true;
    return R;
}

// Arithmetic of the Jacobi solver.  J64: FP64 throughout.  JDF: A and S held
// as double-float pairs (hi + lo floats, ~48 significant bits) and all
// arithmetic on the FP32 pipe (FP64 on this part is 64x slower in throughput
// and 14x in latency); used by the mixed-precision forms, whose contractions
// carry errors of the same order.
struct J64 {
    using T = double;
    static constexpr int kMinBlocks = 3;  // blocks per SM of the one-round-per-barrier solver
    struct R {
        T c, s;
        bool on;
    };
    __device__ static T ld(const T* p) { return __ldcg(p); }
    __device__ static T from(double x) { return x; }
    __device__ static double to(T a) { return a; }
    __device__ static T zero() { return 0.0; }
    __device__ static T one() { return 1.0; }
    __device__ static T neg(T a) { return -a; }
    __device__ static T half(T a) { return 0.5 * a; }
    __device__ static T add(T a, T b) { return a + b; }
    __device__ static T lin(T a, T x, T b, T y) { return a * x - b * y; }  // a x - b y
    __device__ static bool nz(T a) { return a != 0.0; }
    __device__ static bool above(T app, T aqq, T apq, double eps, double floor_abs) {
        return jac_above(app, aqq, apq, eps, floor_abs);
    }
    __device__ static R rot(T app, T aqq, T apq, double eps, double floor_abs) {
        const Rot r = rot_fast(app, aqq, apq, eps, floor_abs);
        return R{r.c, r.s, r.on};
    }
};

struct JDF {
    using T = float2;  // x = hi, y = lo
    static constexpr int kMinBlocks = 4;  // blocks per SM of the one-round-per-barrier solver
    struct R {
        T c, s;
        bool on;
    };
    __device__ static T quick(float s, float e) {
        const float h = s + e;
        return make_float2(h, e - (h - s));
    }
    __device__ static T ld(const T* p) { return __ldcg(p); }
    __device__ static T from(double x) {
        const float h = (float)x;
        return make_float2(h, (float)(x - (double)h));
    }
    __device__ static double to(T a) { return (double)a.x + (double)a.y; }
    __device__ static T zero() { return make_float2(0.f, 0.f); }
    __device__ static T one() { return make_float2(1.f, 0.f); }
    __device__ static T neg(T a) { return make_float2(-a.x, -a.y); }
    __device__ static T half(T a) { return make_float2(0.5f * a.x, 0.5f * a.y); }
    __device__ static T add(T a, T b) {  // Knuth's two-sum on the high parts
        const float s = a.x + b.x, bb = s - a.x;
        const float e = (a.x - (s - bb)) + (b.x - bb);
        return quick(s, e + (a.y + b.y));
    }
    // a x - b y with both products' rounding errors kept (two-product by FMA)
    // and the high parts summed by a two-sum, normalised once
    __device__ static T lin(T a, T x, T b, T y) {
        const float p1 = a.x * x.x, e1 = fmaf(a.x, x.x, -p1);
        const float p2 = -b.x * y.x, e2 = fmaf(-b.x, y.x, -p2);
        const float s = p1 + p2, bb = s - p1;
        const float e = (p1 - (s - bb)) + (p2 - bb);
        const float lo = ((e + e1) + e2) + (fmaf(a.x, x.y, a.y * x.x) - fmaf(b.x, y.y, b.y * y.x));
        return quick(s, lo);
    }
    __device__ static bool nz(T a) { return a.x != 0.f; }
    __device__ static T mul(T a, T b) {
        const float p = a.x * b.x;
        return quick(p, fmaf(a.x, b.x, -p) + fmaf(a.x, b.y, a.y * b.x));
    }
    __device__ static bool above(T app, T aqq, T apq, double eps, double floor_abs) {
        if (apq.x == 0.f) return false;
        const float a = fabsf(apq.x);
        if (!(a > (float)floor_abs)) return false;
        return a > (float)eps * sqrtf(fabsf(app.x)) * sqrtf(fabsf(aqq.x));
    }
    // The rotation of rot_fast in double-float: FP32 tangent, then c = 1/sqrt(1
    // + t^2) from an FP32 seed by two double-float Newton steps, s = t c.
    __device__ static R rot(T app, T aqq, T apq, double eps, double floor_abs) {
        R out{one(), zero(), false};
        if (!above(app, aqq, apq, eps, floor_abs)) return out;
        const T d = add(aqq, neg(app));
        const float tau = d.x / (2.0f * apq.x);
        const float t = fabsf(tau) > 1e18f ? 0.5f / tau
                                           : copysignf(1.0f, tau) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.0f)));
        // x = 1 + t^2 exactly as a pair (|t| <= 1)
        const float t2 = t * t, t2e = fmaf(t, t, -t2);
        const float xh = 1.0f + t2;
        const T x = quick(xh, ((1.0f - xh) + t2) + t2e);
        T y = make_float2(rsqrtf(xh), 0.f);
#pragma unroll
        for (int it = 0; it < 2; ++it) {
            const T r = add(one(), neg(mul(x, mul(y, y))));  // 1 - x y^2, small
            y = add(y, make_float2(0.5f * y.x * r.x, 0.f));
        }
        out.c = y;
        const float sh = t * y.x;
        out.s = quick(sh, fmaf(t, y.x, -sh) + t * y.y);
        out.on = true;
        return out;
    }
};

}  // namespace
}  // namespace ctm
