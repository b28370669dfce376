// ctm.cu -- host orchestration of the CTMRG step and the C-ABI of include/ctm.h.
//
// One handle = one temperature of Algorithm 3 (Symmetric-CTMRG) of
// arXiv:2004.08669 on one GPU.  A step is
//   a2  extension   C~ = Sub-CTMRG(P, Omega P, W)      (GEMM of the form + W contraction)
//   a3  eigenpairs  leading b Ritz pairs of C~           (subspace iteration,
//                   Jacobi Rayleigh-Ritz, CholQR2, multiplet-aware cut,
//                   gauge alignment to the previous step)
//   a4  renormalise P <- U^t Sub-CTMRG(P, U', W)          (GEMMs + W contraction)
//   a5  normalise   P <- P / ||P||_F, Omega <- Omega / (sum w^4)^{1/4}
//   a6  S_E (Eq. 6) and the convergence measure delta on the device.
// The GEMMs run on the FP64 cores (CTM_FP64), on tcgen05 in TF32 / BF16, or
// as FP64 emulated by bf16 digit slices on tcgen05 (CTM_OZAKI64); the small
// solves are FP64 (CTM_FP64) or double-float on the FP32 pipe (the others).
// The host only sequences launches and reads back one small control block per
// subspace iteration.  Also here: the autotuner of the tensor-core GEMMs, the
// temperature scan (ctm_scan_*, one handle per beta, a native worker pool)
// and the effective correlation length (ctm_xi, Lanczos on the row-to-row
// transfer matrix).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <string>
#include <vector>

#include "../../include/ctm.h"
#include "ctm_internal.cuh"
#include "eig_f64.cuh"
#include "oz_gemm.cuh"
#include "host_gmres.h"
#include "tangent.cuh"
#include "tc_gemm.cuh"
#include "xi.cuh"

namespace {

thread_local std::string g_err;

ctm_status fail(ctm_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

#define CTM_CUDA(call)                                                                       \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(CTM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));      \
    } while (0)

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    int q, dim, m, N, b, npad, splits;
    size_t off_spins, off_E, off_Eh, off_mag, off_P, off_Pn, off_omega, off_prev, off_C, off_V, off_Y,
        off_Z, off_T, off_Zprev, off_U, off_Up, off_H, off_Sb, off_G, off_Linv, off_theta, off_res,
        off_part, off_red, off_A0, off_A1, off_S, off_diag, off_rank, off_gd, off_gQ, off_gk, off_ctl,
        off_S1, off_mfull, off_colv, off_opP, off_opPw, off_opC, off_opV, off_opUp, off_opU, off_tcerr, off_ozP, off_ozBig,
        off_ozSA, off_ozSB, off_ozeP, off_ozeBig, off_ozeSA, off_ozeSB, off_oaX, off_oaW1, off_oaS, off_oaR, off_oaE,
        off_oapart, off_oaclus, off_tcpart, off_rrc, total;
    size_t tcpart_cap;  // doubles of the split-K partial buffer of the tensor-core GEMM
    int slices;     // digit planes of the FP64-emulating form
    size_t part_cap;  // doubles of the split-K partial buffer
    int prec;       // ctm_precision
    int esz;        // operand element bytes (2 bf16, 4 tf32; 0 in FP64 form)
    int ldm, ldN;   // operand leading dimensions for K = m and K = N
};

Layout make_layout(const ctm_config& c) {
    Layout L{};
    L.q = c.q;
    L.dim = c.dim;
    L.m = c.m;
    L.N = c.m * c.q;
    int extra = c.block_extra > 0 ? c.block_extra : std::max(8, c.m / 8);
    L.b = std::min(L.N, c.m + extra);
    L.npad = L.b + (L.b & 1);
    if (L.npad < 2) L.npad = 2;
    L.splits = 16;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t r = o;
        o = align256(o + bytes);
        return r;
    };
    const size_t d = sizeof(double);
    const size_t N = L.N, b = L.b, m = L.m, q = L.q, np = L.npad;
    L.off_spins = take(q * L.dim * d);
    L.off_E = take(q * q * d);
    L.off_Eh = take(q * q * d);
    L.off_mag = take(q * d);
    L.off_P = take(m * N * d);
    L.off_Pn = take(m * N * d);
    L.off_omega = take(m * d);
    L.off_prev = take(m * d);
    L.off_C = take(N * N * d);
    L.off_V = take(N * b * d);
    L.off_Y = take(N * b * d);
    L.off_Z = take(N * b * d);
    L.off_T = take(N * b * d);
    L.off_Zprev = take(N * b * d);
    L.off_U = take(N * m * d);
    L.off_Up = take(m * N * d);
    L.off_H = take(b * b * d);
    L.off_Sb = take(b * b * d);
    L.off_G = take(b * b * d);
    L.off_Linv = take(b * b * d);
    L.off_theta = take(np * d);
    L.off_res = take(np * d);
    // split-K partials: the b x b Gram products (up to 16 slices) and, in the
    // FP64-emulating forms, up to 6 slices of the N x b and m x N products
    L.part_cap = (size_t)L.splits * b * b;
    if (c.prec != CTM_FP64) L.part_cap = std::max(L.part_cap, (size_t)6 * N * b);
    L.off_part = take(L.part_cap * d);
    L.off_red = take(4096 * d);
    L.off_A0 = take(np * np * d);
    L.off_A1 = take(np * np * d);
    L.off_S = take(np * np * d);
    L.off_S1 = take(np * np * d);
    L.off_diag = take(np * d);
    L.off_rank = take(np * sizeof(int));
    L.off_gd = take(3 * np * d);
    L.off_gQ = take(4 * np * d);
    L.off_gk = take(np * sizeof(int));
    L.off_ctl = take(sizeof(ctm::DevCtl));
    L.off_mfull = take(sizeof(int));
    L.off_colv = take(2 * np * d);
    L.off_oaX = take(b * b * d);
    L.off_oaW1 = take(std::max<size_t>((size_t)b * b, (size_t)((b + 31) / 32) * 1024) * d);  // also trinv scratch
    L.off_oaS = take(b * b * d);
    L.off_oaR = take(b * b * d);
    L.off_oaE = take(b * b * d);
    L.off_oapart = take(1024 * d);
    L.off_oaclus = take(np * sizeof(int));
    // cluster-aware refinement of the Rayleigh-Ritz solve (mixed forms)
    L.off_rrc = (c.prec != CTM_FP64 && ctm::rrc_supported(L.b)) ? take(ctm::rrc_workspace_bytes(L.b)) : 0;
    L.prec = c.prec;
    L.slices = c.ozaki_slices > 0 ? c.ozaki_slices : 7;
    L.esz = (c.prec == CTM_BF16) ? 2 : (c.prec == CTM_TF32 ? 4 : 0);
    L.ldm = ((L.m + 63) / 64) * 64;
    L.ldN = ((L.N + 63) / 64) * 64;
    if (L.esz) {
        const size_t e = L.esz;
        L.off_opP = take(N * L.ldm * e);
        L.off_opPw = take(N * L.ldm * e);
        L.off_opC = take(N * L.ldN * e);
        L.off_opV = take(b * L.ldN * e);
        L.off_opUp = take(N * L.ldm * e);
        L.off_opU = take(m * L.ldN * e);
        L.off_tcerr = take(sizeof(int));
        // split-K partial tiles: up to 4 slices of the N x b product
        L.tcpart_cap = 4 * N * b;
        L.off_tcpart = take(L.tcpart_cap * d);
        // digit-plane slots of the FP64-emulated small products (N x b x b,
        // b x b x N) of the Rayleigh-Ritz and Cholesky QR steps
        const int S = L.slices, Ni = L.N, bi = L.b;
        auto opA = [&](int R, int K) { return ctm::oz_operand_bytes(R, K, S, true); };
        auto opB = [&](int R, int K) { return ctm::oz_operand_bytes(R, K, S, false); };
        L.off_ozSA = take(std::max(opA(Ni, bi), opA(bi, Ni)));
        L.off_ozSB = take(std::max(opB(bi, Ni), opB(bi, bi)));
        L.off_ozeSA = take(N * sizeof(int));
        L.off_ozeSB = take(N * sizeof(int));
    }
    if (c.prec == CTM_OZAKI64) {
        // digit-plane slots: P (A role, kept from the extension to the P
        // update), BIG (C~ or X, N x N), SA / SB (the small operands)
        const int S = L.slices, Ni = L.N, bi = L.b, mi = L.m;
        auto opA = [&](int R, int K) { return ctm::oz_operand_bytes(R, K, S, true); };
        auto opB = [&](int R, int K) { return ctm::oz_operand_bytes(R, K, S, false); };
        L.off_ozP = take(opA(Ni, mi));
        L.off_ozBig = take(std::max(opA(Ni, Ni), opB(Ni, Ni)));
        L.off_ozSA = take(std::max({opA(Ni, bi), opA(bi, Ni), opA(mi, Ni)}));
        L.off_ozSB = take(std::max({opB(Ni, mi), opB(bi, Ni), opB(bi, bi)}));
        L.off_ozeP = take(N * sizeof(int));
        L.off_ozeBig = take(N * sizeof(int));
        L.off_ozeSA = take(N * sizeof(int));
        L.off_ozeSB = take(N * sizeof(int));
        L.off_tcerr = take(sizeof(int));
    }
    L.total = o;
    return L;
}

}  // namespace

struct ctm_handle {
    ctm_config cfg;
    Layout lay;
    cudaStream_t st = nullptr;
    bool own_ws = false;
    char* ws = nullptr;
    // device views
    double *spins, *E, *Eh, *mag, *P, *Pn, *omega, *prev, *C, *V, *Y, *Z, *T, *Zprev, *U, *Up, *H, *Sb, *G,
        *Linv, *theta, *res, *part, *red, *colv;
    int* mfull;
    void *opP = nullptr, *opPw = nullptr, *opC = nullptr, *opV = nullptr, *opUp = nullptr, *opU = nullptr;
    int* tcerr = nullptr;
    double* tcpart = nullptr;
    void *ozP = nullptr, *ozBig = nullptr, *ozSA = nullptr, *ozSB = nullptr;
    int *ozeP = nullptr, *ozeBig = nullptr, *ozeSA = nullptr, *ozeSB = nullptr;
    ctm::EigWork ew;
    ctm::OaWork oa;
    ctm::RrcWork rrc{};
    bool have_rrc = false;
    long long rrc_solves = 0, rrc_fails = 0;  // cluster refinement attempts that failed
    long long rr_refined = 0, rr_jacobi = 0;  // Rayleigh-Ritz solves by path
    int last_backward_iters = 0;              // GMRES iterations of the last ctm_step_backward
    double last_backward_residual = 0.0;
    double last_resid = 0.0;                  // last Ritz residual / |w_1|
    int rr_fail_streak = 0;                   // consecutive failed refinements
    long long rr_fail_counts[5] = {0, 0, 0, 0, 0};  // fallbacks to Jacobi by reason
    double resid_rate = 0.5;                  // measured Ritz residual reduction per iteration
    int jac_rec = -1;                         // profile record of the last Jacobi solve
    ctm::DevCtl* ctl;
    ctm::DevCtl* hctl = nullptr;  // pinned mirror
    // host-side iteration state
    int live = 1;
    int steps = 0;
    bool warm = false;
    int warm_live = -1;
    uint64_t seed = 2004086690ull;
    ctm_step_info last{};
    std::vector<double> spins_h;
    // profiling (kernel classes timed with events on st) and launch counting
    struct Rec {
        int cls;
        cudaEvent_t a, b;
        double flops, bytes;
        int nk;
    };
    bool prof_on = false;
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> evpool;
    size_t evnext = 0;
    long long launches = 0;
    long long launches_prof = 0;
};

namespace {

ctm_status validate(const ctm_config* c) {
    if (!c) return fail(CTM_EINVAL, "config is NULL");
    if (c->q < 2 || c->q > 32) return fail(CTM_EINVAL, "q must be in [2, 32]");
    if (c->dim < 1 || c->dim > 4) return fail(CTM_EINVAL, "dim must be in [1, 4]");
    if (!c->spins) return fail(CTM_EINVAL, "spins is NULL");
    if (c->m < 1) return fail(CTM_EINVAL, "m must be >= 1");
    if ((long)c->m * c->q > 65536) return fail(CTM_EINVAL, "m q must be <= 65536");
    if (!(c->beta >= 0.0) || !isfinite(c->beta)) return fail(CTM_EINVAL, "beta must be finite and >= 0");
    if (c->boundary_spin < 0 || c->boundary_spin >= c->q) return fail(CTM_EINVAL, "boundary_spin out of range");
    for (int s = 0; s < c->q; ++s) {
        double n2 = 0.0;
        for (int k = 0; k < c->dim; ++k) n2 += c->spins[s * c->dim + k] * c->spins[s * c->dim + k];
        if (!(fabs(sqrt(n2) - 1.0) <= 1e-12)) return fail(CTM_EINVAL, "spins must be unit vectors");
    }
    if (c->prec != CTM_FP64 && c->prec != CTM_TF32 && c->prec != CTM_BF16 && c->prec != CTM_OZAKI64)
        return fail(CTM_EUNSUPPORTED, "precision mode not built in this library");
    if (c->prec == CTM_OZAKI64 && c->ozaki_slices != 0 && (c->ozaki_slices < 3 || c->ozaki_slices > 7))
        return fail(CTM_EINVAL, "ozaki_slices must be 0 (default 7) or in [3, 7]");
    return CTM_OK;
}

// Defaults.  The residual and the step-to-step change cannot fall below the
// rounding of the contraction operands, so the reduced-precision forms get
// tolerances at their floor (TF32: 10 explicit mantissa bits, BF16: 7).
ctm_config with_defaults(const ctm_config& c) {
    ctm_config r = c;
    double floor_tol = (c.prec == CTM_BF16) ? 3e-3 : (c.prec == CTM_TF32 ? 3e-5 : 0.0);
    if (c.prec == CTM_OZAKI64) {
        // s digit planes of 7 bits: products carry about 2^(-7s) relative error
        const int S = c.ozaki_slices > 0 ? c.ozaki_slices : 7;
        floor_tol = std::max(1e-13, ldexp(1.0, -7 * S + 3));
    }
    if (r.tol_spectrum <= 0.0) r.tol_spectrum = floor_tol > 0.0 ? floor_tol : 1e-12;
    if (r.max_steps <= 0) r.max_steps = 5000;
    if (r.max_subspace_iters <= 0) r.max_subspace_iters = 50;
    if (r.subspace_tol <= 0.0) r.subspace_tol = floor_tol > 0.0 ? floor_tol : 1e-13;
    // Multiplets must still be recognised when rounding splits them: in the
    // reduced-precision forms the cluster tolerance sits above the noise.
    if (r.tol_cluster <= 0.0) {
        r.tol_cluster = (c.prec == CTM_BF16) ? 3e-2 : (c.prec == CTM_TF32 ? 3e-4 : 1e-10);
        // the digit expansion is relative to each row's largest entry, so the
        // small eigenvalues of C~ carry errors near 2^(-7s) K times |w_1|
        // with converged Ritz pairs (residual ~1e-11 |w_1|) seven slices resolve
        // multiplets as the FP64 form does
        if (c.prec == CTM_OZAKI64) r.tol_cluster = (c.ozaki_slices == 0 || c.ozaki_slices == 7) ? 1e-10 : 1e-8;
    }
    return r;
}

// ------------------------------------------------------------ small kernels
__global__ void k_weights(int q, int dim, const double* __restrict__ v, double beta, int bspin,
                          double* __restrict__ E, double* __restrict__ Eh, double* __restrict__ mag) {
    for (int e = threadIdx.x; e < q * q; e += blockDim.x) {
        int a = e % q, b = e / q;
        double d = 0.0;
        for (int k = 0; k < dim; ++k) d += v[a * dim + k] * v[b * dim + k];
        double w = exp(beta * d);  // Eq. (2): one bond's share exp(-h/T), h = -v.v
        E[e] = w;
        Eh[e] = -d * w;            // the same bond with its energy h inserted
    }
    for (int s = threadIdx.x; s < q; s += blockDim.x) {
        double d = 0.0;
        for (int k = 0; k < dim; ++k) d += v[bspin * dim + k] * v[s * dim + k];
        mag[s] = d;
    }
}

// U (N x m) = Z[:, :m] with columns >= meff zeroed; U' (m x N) with
// U'[alpha + m (sigma + q alpha')] = U[(sigma + q alpha) + N alpha'] (P-Index2).
__global__ void k_make_U(int N, int m, int q, const double* __restrict__ Z, int ldz,
                         const ctm::DevCtl* __restrict__ ctl, double* __restrict__ U, double* __restrict__ Up) {
    const int meff = ctl->meff_new;
    size_t tot = (size_t)N * m;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot;
         e += (size_t)gridDim.x * blockDim.x) {
        int t = (int)(e % N), ap = (int)(e / N);
        double v = (ap < meff) ? Z[t + (size_t)ldz * ap] : 0.0;
        U[e] = v;
        int sigma = t % q, alpha = t / q;
        Up[alpha + (size_t)m * (sigma + (size_t)q * ap)] = v;
    }
}

// Deterministic partial sums of squares.
__global__ void k_sumsq_partial(size_t n, const double* __restrict__ x, double* __restrict__ part) {
    __shared__ double red[32];
    double s = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        s += x[i] * x[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) part[blockIdx.x] = s;
    }
}

// a5/a6: kappa, Omega normalisation, S_E of the kept spectrum, delta.
// Block-wide sum / max over 256 threads (result valid in every thread).
__device__ double block_sum256(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    return t;
}

__device__ double block_max256(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = red[0];
    for (int w = 1; w < 8; ++w) t = fmax(t, red[w]);
    return t;
}

// a5/a6 of a step, one block of 256 threads: kappa = ||P_new||_F from the
// partial sums, the kept spectrum omega = theta / (sum theta^4)^(1/4), S_E
// (Eq. 6) and the convergence measure delta (reading R6).
__global__ void __launch_bounds__(256) k_step_finalize(int m, int nparts, const double* __restrict__ part,
                                                       const double* __restrict__ theta,
                                                       double* __restrict__ omega, double* __restrict__ prev,
                                                       ctm::DevCtl* ctl) {
    __shared__ double red[8];
    const int t = threadIdx.x;
    double ss = 0.0;
    for (int i = t; i < nparts; i += 256) ss += part[i];
    const double kappa = sqrt(block_sum256(ss, red));
    const int meff = ctl->meff_new;
    double z = 0.0;
    for (int i = t; i < meff; i += 256) {
        const double x = theta[i] * theta[i];
        z += x * x;
    }
    const double z4 = block_sum256(z, red);
    const double sc = 1.0 / sqrt(sqrt(z4));
    double se = 0.0;
    for (int i = t; i < meff; i += 256) {
        const double x = theta[i] * theta[i];
        const double p = x * x / z4;
        if (p > 0.0) se -= p * log(p);
    }
    const double SE = block_sum256(se, red);
    const double a1 = fabs(theta[0]);
    const int have_prev = ctl->have_prev;
    double dl = 0.0;
    for (int i = t; i < m; i += 256) {
        const double w = (i < meff) ? theta[i] * sc : 0.0;
        omega[i] = w;
        const double r = (i < meff) ? fabs(theta[i]) / a1 : 0.0;
        if (have_prev) dl = fmax(dl, fabs(r - prev[i]));
        prev[i] = r;
    }
    double delta = block_max256(dl, red);
    if (t == 0) {
        if (have_prev) delta = fmax(delta, fabs(kappa / ctl->prev_kappa - 1.0));
        else delta = INFINITY;
        if (!isfinite(kappa) || kappa == 0.0 || !isfinite(SE)) ctl->numeric_bad = 1;
        ctl->have_prev = 1;
        ctl->prev_kappa = kappa;
        ctl->kappa = kappa;
        ctl->delta = delta;
        ctl->SE = SE;
        ctl->live = meff;
    }
}

__global__ void k_scale(size_t n, const double* __restrict__ x, const ctm::DevCtl* __restrict__ ctl,
                        double* __restrict__ y) {
    double inv = 1.0 / ctl->kappa;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = x[i] * inv;
}

// Observables: per kept column, col[i] = sum_t Z_ti^2 mag(t mod q) and
// col[b + i] = z_i . Yh_i.
__global__ void k_obs_cols(int N, int q, int b, const double* __restrict__ Z, const double* __restrict__ Yh,
                           const double* __restrict__ mag, double* __restrict__ col) {
    __shared__ double red[2][32];
    int i = blockIdx.x;
    double s0 = 0.0, s1 = 0.0;
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
        double z = Z[t + (size_t)N * i];
        s0 += z * z * mag[t % q];
        s1 += z * Yh[t + (size_t)N * i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = s0;
        red[1][threadIdx.x >> 5] = s1;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        int nw = blockDim.x >> 5;
        s0 = threadIdx.x < nw ? red[0][threadIdx.x] : 0.0;
        s1 = threadIdx.x < nw ? red[1][threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        }
        if (threadIdx.x == 0) {
            col[i] = s0;
            col[b + i] = s1;
        }
    }
}

__global__ void k_obs_finalize(int b, const double* __restrict__ theta, const double* __restrict__ col,
                               ctm::DevCtl* ctl) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int meff = ctl->meff_new;
    double z4 = 0, mn = 0, un = 0;
    for (int i = 0; i < meff; ++i) {
        double w = theta[i], w3 = w * w * w, w4 = w3 * w;
        z4 += w4;
        mn += w4 * col[i];
        un += w3 * col[b + i];
    }
    double SE = 0.0;
    for (int i = 0; i < meff; ++i) {
        double p = pow(theta[i], 4) / z4;
        if (p > 0.0) SE -= p * log(p);
    }
    ctl->obs_M_num = mn;
    ctl->obs_u_num = un;
    ctl->obs_z4 = z4;
    ctl->obs_SE = SE;
}

__global__ void k_gather(int count, const long long* __restrict__ idx, const double* __restrict__ C,
                         double* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        out[i] = C[idx[i]];
}

__global__ void k_set_int(int* p, int v) { *p = v; }

inline int grid_for(size_t work, int cap = 152 * 8) {
    size_t g = (work + 255) / 256;
    if (g < 1) g = 1;
    if (g > (size_t)cap) g = cap;
    return (int)g;
}

// --------------------------------------------------------------- profiling
enum ProfClass {
    PC_GEMM = 0, PC_WCONTRACT, PC_JACOBI, PC_CHOLQR, PC_TCGEMM, PC_CONVERT, PC_OZGEMM, PC_OZSPLIT, PC_SMALL,
    PC_XI_W, PC_XI_VEC, PC_RRC, PC_COUNT
};
const char* const kProfNames[PC_COUNT + 1] = {"gemm_f64", "wcontract_f64", "jacobi_f64", "cholqr_f64", "tc_gemm",
                                              "to_operand", "oz_gemm",  "oz_split",    "small",      "xi_wcontract",
                                              "xi_lanczos", "rr_refine", "all"};

cudaEvent_t take_event(ctm_handle* h) {
    if (h->evnext == h->evpool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        h->evpool.push_back(e);
    }
    return h->evpool[h->evnext++];
}

// Bracket one kernel class: begin returns an event (or null when off).
cudaEvent_t prof_begin(ctm_handle* h) {
    if (!h->prof_on) return nullptr;
    cudaEvent_t a = take_event(h);
    cudaEventRecord(a, h->st);
    return a;
}

void prof_end(ctm_handle* h, cudaEvent_t a, int cls, int nk, double flops = 0.0, double bytes = 0.0) {
    h->launches += nk;
    if (!h->prof_on) return;
    h->launches_prof += nk;
    if (!a) return;
    cudaEvent_t b = take_event(h);
    cudaEventRecord(b, h->st);
    h->recs.push_back({cls, a, b, flops, bytes, nk});
}

// Small bookkeeping kernels: counted, not timed.
void count_small(ctm_handle* h, int nk) {
    h->launches += nk;
    if (h->prof_on) h->launches_prof += nk;
}

// Profiled FP64 GEMM with its algorithmic FLOPs and minimum bytes.
// Outputs of an M x N product: all of them, or (lowq > 0) the q x q blocks
// on and below the block diagonal.
double outputs_of(int M, int N, int lowq) {
    if (lowq <= 0) return (double)M * N;
    const double nb = (double)(M / lowq);
    return nb * (nb + 1) / 2.0 * lowq * lowq;
}

void pgemm(ctm_handle* h, bool tA, bool tB, int M, int N, int K, const double* A, int lda, const double* B,
           int ldb, double* C, int ldc, const double* scaleK = nullptr, int splits = 1, int lowq = 0) {
    cudaEvent_t a = prof_begin(h);
    int nk = ctm::gemm_f64(h->st, tA, tB, M, N, K, 1.0, A, lda, B, ldb, 0.0, C, ldc, scaleK, splits, h->part,
                           lowq);
    const double outs = outputs_of(M, N, splits > 1 ? 0 : lowq);
    double fl = 2.0 * outs * K;
    double by = 8.0 * ((double)M * K + (double)K * N + outs);
    prof_end(h, a, PC_GEMM, nk, fl, by);
}

// Profiled conversion of R rows (each a column of a column-major FP64 matrix,
// K long) into the tensor-core operand precision.
void pconvert(ctm_handle* h, int R, int K, const double* src, int lds, const double* scale, void* dst, int ldo) {
    cudaEvent_t a = prof_begin(h);
    ctm::to_operand(h->st, h->lay.esz == 2, R, K, src, lds, scale, dst, ldo);
    prof_end(h, a, PC_CONVERT, 1, 0.0, (double)R * K * 8.0 + (double)R * ldo * h->lay.esz);
}

// Launch shapes picked by ctm_tune, per (operand bytes, M, N, K); shared by
// every handle of the process (the best shape depends on the GEMM, not on
// the data).
struct TcKey {
    int esz, M, N, K;
    bool operator<(const TcKey& o) const {
        if (esz != o.esz) return esz < o.esz;
        if (M != o.M) return M < o.M;
        if (N != o.N) return N < o.N;
        return K < o.K;
    }
};
std::mutex g_tc_mu;
std::map<TcKey, ctm::TcPlan> g_tc_plans;

// Ozaki GEMM K slices picked by ctm_tune, per (digit planes, M, N, K); 0 = the
// kernel's own rule.
std::map<TcKey, int> g_oz_plans;

int oz_plan_for(int S, int M, int N, int K) {
    std::lock_guard<std::mutex> g(g_tc_mu);
    auto it = g_oz_plans.find(TcKey{S, M, N, K});
    return it != g_oz_plans.end() ? it->second : 0;
}

ctm::TcPlan tc_plan_for(int esz, int M, int N, int K) {
    std::lock_guard<std::mutex> g(g_tc_mu);
    auto it = g_tc_plans.find(TcKey{esz, M, N, K});
    if (it != g_tc_plans.end()) return it->second;
    return ctm::tc_default_plan(M, N, K, esz == 2);
}

// Profiled tensor-core GEMM D = A B^t (operands already converted).
ctm_status ptc(ctm_handle* h, int M, int N, int K, const void* A, int lda, const void* B, int ldb, double* D,
               int ldd, int lowq = 0) {
    cudaEvent_t a = prof_begin(h);
    const ctm::TcPlan plan = tc_plan_for(h->lay.esz, M, N, K);
    cudaError_t e = ctm::tc_gemm(h->st, h->lay.esz == 2, M, N, K, 1.0, A, lda, B, ldb, 0.0, D, ldd, h->tcerr, &plan,
                                 h->tcpart, h->lay.tcpart_cap, lowq);
    if (e != cudaSuccess) return fail(CTM_ECUDA, std::string("tc_gemm: ") + cudaGetErrorString(e));
    const double outs = outputs_of(M, N, ctm::tc_plan_slices(plan, K, h->lay.esz == 2, nullptr) > 1 ? 0 : lowq);
    double fl = 2.0 * outs * K;
    double by = (double)h->lay.esz * ((double)M * K + (double)K * N) + 8.0 * outs;
    prof_end(h, a, PC_TCGEMM, ctm::tc_plan_slices(plan, K, h->lay.esz == 2, nullptr) > 1 ? 2 : 1, fl, by);
    return CTM_OK;
}

// Operand of a contraction D(i, j) = sum_k A(i, k) B(j, k): element (r, k) is
// p[r rs + k ks], times scale[k] when scale is given.
struct Opnd {
    const double* p;
    long rs, ks;
    const double* scale;
};
enum OzSlot { OZ_P = 0, OZ_BIG, OZ_SA, OZ_SB };

void oz_slot(ctm_handle* h, OzSlot sl, void** planes, int** e) {
    switch (sl) {
        case OZ_P: *planes = h->ozP; *e = h->ozeP; break;
        case OZ_BIG: *planes = h->ozBig; *e = h->ozeBig; break;
        case OZ_SA: *planes = h->ozSA; *e = h->ozeSA; break;
        default: *planes = h->ozSB; *e = h->ozeSB; break;
    }
}

// FP64-emulating contraction on the tensor cores: split A and B (unless the
// slot already holds that operand) and multiply the digit planes.
ctm_status ozmm(ctm_handle* h, int M, int N, int K, Opnd A, OzSlot sa, bool splitA, Opnd B, OzSlot sb, bool splitB,
                double* D, int ldd, int lowq = 0) {
    const int S = h->lay.slices;
    void *pa, *pb;
    int *ea, *eb;
    oz_slot(h, sa, &pa, &ea);
    oz_slot(h, sb, &pb, &eb);
    if (splitA || splitB) {
        cudaEvent_t a = prof_begin(h);
        int nk = 0;
        if (splitA) {
            ctm::oz_split_strided(h->st, M, K, S, A.p, A.rs, A.ks, A.scale, pa, true, ea);
            ++nk;
        }
        if (splitB) {
            ctm::oz_split_strided(h->st, N, K, S, B.p, B.rs, B.ks, B.scale, pb, false, eb);
            ++nk;
        }
        prof_end(h, a, PC_OZSPLIT, nk, 0.0, 8.0 * ((splitA ? (double)M * K : 0.0) + (splitB ? (double)N * K : 0.0)));
    }
    cudaEvent_t a = prof_begin(h);
    const int req = oz_plan_for(S, M, N, K);
    cudaError_t e =
        ctm::oz_gemm(h->st, S, M, N, K, pa, ea, pb, eb, D, ldd, h->tcerr, h->part, h->lay.part_cap, req, lowq);
    if (e != cudaSuccess) return fail(CTM_ECUDA, std::string("oz_gemm: ") + cudaGetErrorString(e));
    const double pairs = S * (S + 1) / 2.0;
    // outputs computed: all of D, or its q x q blocks on and below the block diagonal
    const double outs = outputs_of(M, N, lowq);
    prof_end(h, a, PC_OZGEMM, 1, pairs * 2.0 * outs * K, 2.0 * S * ((double)M * K + (double)N * K) + 8.0 * outs);
    return CTM_OK;
}

inline bool is_oz(const ctm_handle* h) { return h->lay.prec == CTM_OZAKI64; }

// The N x b x b and b x b x N products of the Rayleigh-Ritz and Cholesky QR
// steps must be FP64-accurate in every form: the mixed-precision forms run
// them as FP64 emulated on the tensor cores (their slots SA / SB exist in
// every form but FP64), the FP64 form on the FP64 cores.
inline bool oz_small(const ctm_handle* h) { return h->lay.prec != CTM_FP64; }

void pwcontract(ctm_handle* h, double* X, const double* E1, const int* live_dev, int live_host, bool sym = false) {
    const Layout& L = h->lay;
    cudaEvent_t a = prof_begin(h);
    // FP64 form: FP64; Ozaki form: double-float (its products carry ~2^-42);
    // TF32 / BF16 forms: FP32 (far below their operand rounding)
    const int arith = (L.prec == CTM_FP64) ? 0 : (L.prec == CTM_OZAKI64 ? 2 : 1);
    // the symmetric variant needs a symmetric X and E1 = E
    ctm::wcontract_ar(h->st, arith, L.m, L.q, X, L.N, h->E, E1, live_dev, sym && E1 == h->E);
    double nb = (double)live_host * live_host, q = L.q;
    prof_end(h, a, PC_WCONTRACT, 1, nb * 4.0 * q * q * q, nb * 2.0 * 8.0 * q * q);
}

// --------------------------------------------------------------- stages
ctm_status sync_ctl(ctm_handle* h) {
    CTM_CUDA(cudaMemcpyAsync(h->hctl, h->ctl, sizeof(ctm::DevCtl), cudaMemcpyDeviceToHost, h->st));
    CTM_CUDA(cudaStreamSynchronize(h->st));
    return CTM_OK;
}

// Split-K factor: enough CTAs to fill the GPU, at least 128 of K per split,
// and never more partial sums than the partial buffer (splits_max b^2) holds.
int gemm_splits(const Layout& L, int M, int Nn, int K) {
    long tiles = (long)((M + 63) / 64) * ((Nn + 63) / 64);
    long want = (2L * 152 + tiles - 1) / tiles;
    long maxs = std::max(1, K / 128);
    long cap = ((long)L.splits * L.b * L.b) / ((long)M * Nn);
    long s = std::min<long>(std::min<long>(want, maxs), std::min<long>(L.splits, cap));
    return (int)std::max<long>(1, s);
}

// C = P^t diag(omega) P, then the vertex-weight contraction (E1 = E or Eh).
void stage_extend(ctm_handle* h, const double* E1) {
    const Layout& L = h->lay;
    if (is_oz(h)) {
        // with the plain weight the contraction below reads only the blocks
        // on and below the block diagonal of the symmetric X1
        ozmm(h, L.N, L.N, L.m, {h->P, L.m, 1, nullptr}, OZ_P, true, {h->P, L.m, 1, h->omega}, OZ_SB, true, h->C,
             L.N, E1 == h->E ? L.q : 0);
    } else if (L.esz) {
        // X1 = P^t diag(omega) P on the tensor cores: operand rows are the
        // columns of P (K = m), the second one scaled by omega along K.
        pconvert(h, L.N, L.m, h->P, L.m, nullptr, h->opP, L.ldm);
        pconvert(h, L.N, L.m, h->P, L.m, h->omega, h->opPw, L.ldm);
        ptc(h, L.N, L.N, L.m, h->opP, L.ldm, h->opPw, L.ldm, h->C, L.N, E1 == h->E ? L.q : 0);
    } else {
        pgemm(h, true, false, L.N, L.N, L.m, h->P, L.m, h->P, L.m, h->C, L.N, h->omega, 1, E1 == h->E ? L.q : 0);
    }
    pwcontract(h, h->C, E1, &h->ctl->live, h->live, true);  // X1 is symmetric
}

// Orthonormalise src (N x b) into dst by Cholesky QR; `passes` 2 (CholQR,
// then one Newton-Schulz correction) or 3 (shifted CholQR, CholQR, then the
// correction), each factorisation replaced by a Newton-Schulz correction when
// the block's defect is already below 1e-4 (decided on the device).  (Fixed
// Newton-Schulz passes in place of the factorisations were measured: some
// warm blocks leave a defect near 1, where they do not converge.)  tmp is
// clobbered.
ctm_status stage_orth(ctm_handle* h, double* src, double* dst, double* tmp, int passes) {
    const Layout& L = h->lay;
    const int N = L.N, b = L.b;
    double* bufs[2] = {dst, tmp};
    double* cur = src;
    for (int i = 0; i < passes; ++i) {
        double* out = bufs[(passes - 1 - i) % 2];
        if (oz_small(h)) {
            // G = cur^t cur: one split serves both operands
            ctm_status s0 = ozmm(h, b, b, N, {cur, N, 1, nullptr}, OZ_SA, true, {cur, N, 1, nullptr}, OZ_SA, false,
                                 h->G, b);
            if (s0 != CTM_OK) return s0;
        } else {
            pgemm(h, true, false, b, b, N, cur, N, cur, N, h->G, b, nullptr, gemm_splits(L, b, b, N));
        }
        cudaEvent_t a = prof_begin(h);
        if (i + 1 == passes && passes >= 2) {
            // The last pass starts from a block orthonormal to ~eps cond^2
            // (G = I + E, |E| far below 1e-8): Q = Y (3I - G)/2 is
            // orthonormal to O(|E|^2) and needs no factorisation.
            ctm::ns_coeff_f64(h->st, b, h->G, b, h->Linv, b);
            prof_end(h, a, PC_CHOLQR, 1, 0.0, 8.0 * 2.0 * b * b);
        } else {
            // Every earlier pass checks the defect G - I on the device first.
            // A warm block is often close to orthonormal already (the scaled
            // C~ V of a nearly converged block; the shifted factor's output,
            // whose defect is about the shift over the smallest eigenvalue of
            // the first Gram matrix): at a defect d <= 1e-4 the remaining
            // passes as Newton-Schulz corrections reach FP64 orthonormality
            // (each squares the defect, 0.42 d^4 < 1e-16) and the
            // factorisation kernels return at once; otherwise (a defect near
            // 1, where the corrections do not converge) the block is
            // factorised, with a shift in the first of three passes.
            double shift_rel =
                (passes == 3 && i == 0) ? 11.0 * ((double)N * b + (double)b * (b + 1)) * 2.22e-16 : 0.0;
            ctm::orth_check(h->st, b, h->G, b, 1e-4, h->Linv, b, h->ctl, i);
            CTM_CUDA(ctm::cholesky_f64(h->st, b, h->G, b, shift_rel, h->ctl, h->lay.prec != CTM_FP64,
                                       &h->ctl->orth_ns));
            ctm::trinv_f64(h->st, b, h->G, b, h->Linv, b, h->oa.W1, &h->ctl->orth_ns, h->lay.prec != CTM_FP64);
            prof_end(h, a, PC_CHOLQR, 5, (double)b * b * b / 3.0 + (double)b * b * b / 3.0, 8.0 * 2.0 * b * b);
        }
        if (oz_small(h)) {
            ctm_status s0 = ozmm(h, N, b, b, {cur, 1, N, nullptr}, OZ_SA, true, {h->Linv, 1, b, nullptr}, OZ_SB, true,
                                 out, N);
            if (s0 != CTM_OK) return s0;
        } else {
            pgemm(h, false, true, N, b, b, cur, N, h->Linv, b, out, N);
        }
        cur = out;
    }
    CTM_CUDA(cudaGetLastError());
    return CTM_OK;
}

// Leading b eigenpairs of C (a3).  On return theta/Z hold the sorted Ritz
// pairs, h->hctl the decision (meff_new, residual, convergence).
ctm_status stage_eigen(ctm_handle* h, int max_iters, bool* sub_converged, int* iters_used) {
    const Layout& L = h->lay;
    const int N = L.N, b = L.b, m = L.m;
    const int Ldim = L.q * h->live;
    bool cold = true;
    int passes = 3;
    CTM_CUDA(cudaMemsetAsync(&h->ctl->chol_status, 0, sizeof(int), h->st));
    if (Ldim <= b) {
        ctm::identity_block(h->st, N, b, h->V, N);
        count_small(h, 1);
        max_iters = 1;
        passes = 2;
    } else if (h->warm && 2 * h->live >= h->warm_live && h->live <= 2 * h->warm_live) {
        // the renormalised basis is the same one up to states near the cut
        CTM_CUDA(cudaMemcpyAsync(h->V, h->Zprev, sizeof(double) * N * b, cudaMemcpyDeviceToDevice, h->st));
        cold = false;
        passes = 2;
    } else {
        ctm::randn_block(h->st, N, b, h->Y, N, h->seed + (uint64_t)h->steps);
        count_small(h, 1);
        ctm_status s = stage_orth(h, h->Y, h->V, h->T, 3);
        if (s != CTM_OK) return s;
        max_iters = std::max(max_iters, 200);
    }
    bool conv = false;
    int it = 0;
    // last measured Ritz residual (the previous stage's final one to start)
    // A warm block starts from the previous step's Ritz pairs, whose C~ has
    // since changed by about the step's convergence measure delta: the
    // residual is predicted from the larger of the two.
    double r_meas = h->last_resid > 0.0 ? h->last_resid : 1.0;
    if (!cold && h->steps > 0) {
        const double dprev = h->last.delta;
        r_meas = std::max(r_meas, std::isfinite(dprev) ? std::min(dprev, 1.0) : 1.0);
    }
    int it_meas = -1;
    bool meas_here = false;
    if (L.esz) pconvert(h, N, N, h->C, N, nullptr, h->opC, L.ldN);  // C~ rows (symmetric)
    // dst = C~ src (N x b) after the first iteration (C~'s operand is ready)
    auto cmul = [&](const double* src, double* dst) -> ctm_status {
        if (is_oz(h))
            return ozmm(h, N, b, N, {h->C, N, 1, nullptr}, OZ_BIG, false, {src, N, 1, nullptr}, OZ_SB, true, dst, N);
        if (L.esz) {
            pconvert(h, b, N, src, N, nullptr, h->opV, L.ldN);
            return ptc(h, N, b, N, h->opC, L.ldN, h->opV, L.ldN, dst, N);
        }
        pgemm(h, false, false, N, b, N, h->C, N, src, N, dst, N);
        return CTM_OK;
    };
    for (it = 0; it < max_iters; ++it) {
        // A warm block is advanced without a Rayleigh-Ritz solve while the
        // residual cannot yet meet the tolerance: span(C~ V) does not depend
        // on the rotation within span(V), so a later solve extracts the same
        // Ritz pairs.  The residual is predicted from the last measured one
        // and the measured rate per iteration; a solve is taken at the last
        // allowed iteration, when the prediction reaches 10x the tolerance
        // (or the tolerance itself once the residual has stalled: a rate
        // above 1/2 means it sits near the rounding floor of the operands),
        // and at least every 16 iterations.  Skipped blocks are scaled by the
        // previous Ritz values (their columns are last Ritz vectors) and
        // re-orthonormalised by shifted Cholesky QR.
        bool skip_rr = false;
        if (!cold && it + 1 < max_iters && it - it_meas < 16) {
            const double pred = r_meas * std::pow(h->resid_rate, (double)(it - it_meas));
            const double tol = h->cfg.subspace_tol;
            skip_rr = pred > 10.0 * tol || (h->resid_rate > 0.5 && pred > tol);
        }
        if (is_oz(h)) {
            // C~ is split once per eigen stage (first iteration), V every iteration
            ctm_status s0 = ozmm(h, N, b, N, {h->C, N, 1, nullptr}, OZ_BIG, it == 0, {h->V, N, 1, nullptr}, OZ_SB,
                                 true, h->Y, N);
            if (s0 != CTM_OK) return s0;
            if (!skip_rr) {
                s0 = ozmm(h, b, b, N, {h->V, N, 1, nullptr}, OZ_SA, true, {h->Y, N, 1, nullptr}, OZ_SB, true, h->H,
                          b);
                if (s0 != CTM_OK) return s0;
            }
        } else if (L.esz) {
            pconvert(h, b, N, h->V, N, nullptr, h->opV, L.ldN);
            ctm_status s0 = ptc(h, N, b, N, h->opC, L.ldN, h->opV, L.ldN, h->Y, N);
            if (s0 != CTM_OK) return s0;
            if (!skip_rr) {
                s0 = ozmm(h, b, b, N, {h->V, N, 1, nullptr}, OZ_SA, true, {h->Y, N, 1, nullptr}, OZ_SB, true, h->H,
                          b);
                if (s0 != CTM_OK) return s0;
            }
        } else {
            pgemm(h, false, false, N, b, N, h->C, N, h->V, N, h->Y, N);
            if (!skip_rr)
                pgemm(h, true, false, b, b, N, h->V, N, h->Y, N, h->H, b, nullptr, gemm_splits(L, b, b, N));
        }
        if (skip_rr) {
            ctm::next_block(h->st, N, b, h->Y, h->V, N, h->theta, 1e-12, h->T);
            count_small(h, 1);
            // When the next iteration (or the next two) would skip its solve
            // too, its power step is taken now and one orthonormalisation
            // serves both (or all three): span(C~^k V) is what the
            // iterations produce either way.  The group is filtered by the
            // degree-k Chebyshev polynomial on [-|theta_{b-1}|,
            // |theta_{b-1}|] (k = 2, 3), which damps the unwanted spectrum
            // more than C~^k does.
            // Not in a stage's first two iterations, whose blocks still carry
            // the step's change of C~ (their scaled blocks are the least
            // orthonormal: defects up to ~1), and only while the Ritz values
            // the block is scaled by span at most four decades (a column's
            // components along the leading eigenvectors grow by up to the
            // inverse of that range per power step; a corner with a steep
            // spectrum, e.g. Ising's, left the shifted Cholesky QR a
            // non-positive pivot after two steps).  FP64-accurate products
            // only: the TF32 / BF16 products' rounding (~1e-4, ~1e-2 of each
            // column) grows the same way.
            bool twice = false;
            if (!L.esz && it >= 2 && it + 2 < max_iters && it + 1 - it_meas < 16 &&
                h->hctl->theta_range >= 1e-4) {
                const double pred = r_meas * std::pow(h->resid_rate, (double)(it + 1 - it_meas));
                const double tol = h->cfg.subspace_tol;
                twice = pred > 10.0 * tol || (h->resid_rate > 0.5 && pred > tol);
            }
            // measured at q = 20, m = 256 (Ritz values within three
            // decades): groups of three, 27.9 ms per exact Ozaki step, of
            // two, 30.3 ms, single steps, 33.4 ms
            bool thrice = false;
            if (twice && it + 3 < max_iters && it + 2 - it_meas < 16) {
                const double pred = r_meas * std::pow(h->resid_rate, (double)(it + 2 - it_meas));
                const double tol = h->cfg.subspace_tol;
                thrice = pred > 10.0 * tol || (h->resid_rate > 0.5 && pred > tol);
            }
            double* src = h->T;
            if (thrice) {
                ctm_status s1 = cmul(h->T, h->Y);
                if (s1 != CTM_OK) return s1;
                ctm::next_block(h->st, N, b, h->Y, h->T, N, h->theta, 1e-12, h->Z);
                s1 = cmul(h->Z, h->Y);
                if (s1 != CTM_OK) return s1;
                ctm::cheb3_block(h->st, N, b, h->Y, h->T, h->V, N, h->theta, 1e-12);
                count_small(h, 2);
                src = h->V;
                it += 2;
            } else if (twice) {
                ctm_status s1 = cmul(h->T, h->Y);
                if (s1 != CTM_OK) return s1;
                // the pair as the degree-2 Chebyshev filter on the unwanted
                // spectrum's interval (V still holds the block before the pair)
                ctm::cheb2_block(h->st, N, b, h->Y, h->V, N, h->theta, 1e-12);
                count_small(h, 1);
                src = h->V;
                ++it;
            }
            ctm_status s = twice ? stage_orth(h, src, h->T, h->Y, 3) : stage_orth(h, src, h->V, h->Y, 3);
            if (s != CTM_OK) return s;
            if (twice) CTM_CUDA(cudaMemcpyAsync(h->V, h->T, sizeof(double) * N * b, cudaMemcpyDeviceToDevice, h->st));
            continue;
        }
        // Rayleigh-Ritz: simultaneous Jacobi rotations when the block is warm
        // (H nearly diagonal), the cooperative Jacobi solver otherwise or as a
        // fallback.
        int rrc_rec = -1;
        bool rrc_tried = false;
        if (h->have_rrc) {
            // Mixed-precision forms: the cluster-aware refinement in one
            // cooperative launch; the double-float Jacobi solver behind it
            // runs only if the refinement gave up (a device-side flag), so
            // the host does not wait for the outcome.  A cold block (H far
            // from diagonal) goes to Jacobi directly.  A warm block whose
            // strongly coupled pairs form a cluster above 32 states is
            // recognised at the refinement's first check (no product is
            // formed there), so it is tried at every warm solve.
            // Not in the TF32 / BF16 forms: their products leave couplings
            // near their rounding (~1e-4, ~1e-2 of the Ritz values), which
            // the refinement cannot bring to its double-float threshold, so
            // it only ran to its iteration cap before the Jacobi fallback
            // (measured at m = 256: 8 ms of a 17 ms TF32 step).
            rrc_tried = !L.esz && (!cold || it > 0);
            CTM_CUDA(cudaMemsetAsync(&h->ctl->rrc_ok, 0, sizeof(int), h->st));
            if (rrc_tried) {
                cudaEvent_t ra = prof_begin(h);
                // the kept states and the multiplet test at the cut need the
                // leading m + 1 pairs; 16 more keep a multiplet straddling
                // the cut inside the head.  Up to 20 iterations: the first
                // solve of an exact step converges in 10-14 (linearly at
                // first, while the couplings are ~1e-3), and a fallback to
                // Jacobi costs several times an iteration (~230 us at b = 416).
                CTM_CUDA(ctm::rr_cluster_refine(h->st, b, h->H, b, h->rrc, h->ew, h->ctl, 20, std::min(b, m + 16)));
                prof_end(h, ra, PC_RRC, 1);
                rrc_rec = (h->prof_on && ra) ? (int)h->recs.size() - 1 : -1;
                ++h->rrc_solves;
            }
            cudaEvent_t ja2 = prof_begin(h);
            // TF32 / BF16: rotate while a coupling exceeds 1e-9 of the
            // diagonal scale, far below their products' rounding (the
            // double-float threshold 2^-46 only adds sweeps there)
            CTM_CUDA(ctm::jacobi_f64(h->st, b, h->H, b, h->ew, h->theta, h->Sb, b, 40, h->ctl,
                                     L.esz ? 1e-9 : 0.0, 0.0, true,
                                     rrc_tried ? &h->ctl->rrc_ok : nullptr, cold ? 0 : std::min(b, m + 16)));
            prof_end(h, ja2, PC_JACOBI, 4);
            h->jac_rec = (h->prof_on && ja2) ? (int)h->recs.size() - 1 : -1;
        }
        cudaEvent_t ja = h->have_rrc ? nullptr : prof_begin(h);
        int nk_rr = 0, used = -1;
        // After repeated failures (a dense spectrum whose near-degenerate
        // Ritz values are not yet separated) the refinement is only retried
        // every 16th solve, so a failing attempt does not tax every step.
        const bool try_refine =
            !h->have_rrc && (!cold || it > 0) && (h->rr_fail_streak < 3 || (h->rr_jacobi % 16) == 0);
        if (h->have_rrc) {
            // outcome known after the next synchronisation
        } else if (try_refine) {
            used = ctm::rr_refine_f64(h->st, b, std::min(b, m + 2), h->H, b, h->oa, h->ew, h->theta, h->Sb, b, 1e-13,
                                      8, h->ctl, h->hctl, &nk_rr);
            h->rr_fail_streak = used < 0 ? h->rr_fail_streak + 1 : 0;
            if (used < 0 && h->oa.fail_reason >= 1 && h->oa.fail_reason <= 4) ++h->rr_fail_counts[h->oa.fail_reason];
        }
        if (h->have_rrc) {
            // recorded above
        } else if (used < 0) {
            // Full FP64 accuracy: the corner is stored diagonal in the Ritz
            // basis, so any coupling left unrotated enters the next extension
            // at first order.
            // the mixed-precision forms solve in double-float (FP32 pipe); the
            // FP64 form in FP64
            CTM_CUDA(ctm::jacobi_f64(h->st, b, h->H, b, h->ew, h->theta, h->Sb, b, 40, h->ctl, 0.0, 0.0,
                                     h->lay.prec != CTM_FP64, nullptr, cold ? 0 : std::min(b, m + 16)));
            nk_rr += 4;
            ++h->rr_jacobi;
        } else {
            ++h->rr_refined;
        }
        if (!h->have_rrc) {
            prof_end(h, ja, PC_JACOBI, nk_rr);
            // the solve's algorithmic FLOPs are known after the next sync
            h->jac_rec = (used < 0 && h->prof_on && ja) ? (int)h->recs.size() - 1 : -1;
        }
        if (oz_small(h)) {
            ctm_status s0 = ozmm(h, N, b, b, {h->V, 1, N, nullptr}, OZ_SA, true, {h->Sb, b, 1, nullptr}, OZ_SB, true,
                                 h->Z, N);
            if (s0 != CTM_OK) return s0;
            s0 = ozmm(h, N, b, b, {h->Y, 1, N, nullptr}, OZ_SA, true, {h->Sb, b, 1, nullptr}, OZ_SB, false, h->T, N);
            if (s0 != CTM_OK) return s0;
        } else {
            pgemm(h, false, false, N, b, b, h->V, N, h->Sb, b, h->Z, N);
            pgemm(h, false, false, N, b, b, h->Y, N, h->Sb, b, h->T, N);
        }
        int nchk = std::min(m + 1, std::min(b, Ldim));
        ctm::resid_f64(h->st, N, nchk, h->T, h->Z, N, h->theta, h->res);
        ctm::decide(h->st, b, Ldim, m, h->cfg.subspace_tol, h->cfg.tol_cluster, h->theta, h->res, h->ctl);
        count_small(h, (nchk > 0 ? 1 : 0) + 1);
        CTM_CUDA(cudaGetLastError());
        ctm_status s = sync_ctl(h);
        if (s != CTM_OK) return s;
        h->last_resid = h->hctl->resid;
        if (h->have_rrc) {
            const bool ok = rrc_tried && h->hctl->rrc_ok == 1;
            if (ok) {
                ++h->rr_refined;
                h->rr_fail_streak = 0;
            } else {
                ++h->rr_jacobi;
                if (rrc_tried) {
                    ++h->rrc_fails;
                    ++h->rr_fail_streak;
                }
            }
            h->oa.fail_reason = rrc_tried ? h->hctl->rrc_fail : 0;
            if (rrc_tried && !ok && h->oa.fail_reason >= 1 && h->oa.fail_reason <= 4)
                ++h->rr_fail_counts[h->oa.fail_reason];
            h->oa.last_iter = h->hctl->rrc_iters;
            float mc;
            memcpy(&mc, &h->hctl->rrc_maxc, sizeof(float));
            h->oa.last_max = (double)mc;
            if (rrc_rec >= 0 && rrc_rec < (int)h->recs.size()) {
                // per measured iteration H X, X^t X (half) and X^t (H X)
                // (half); per update X (I + E) Q: 2 b^3 FLOP per full product
                const double b3 = (double)b * b * b;
                const int iters = h->hctl->rrc_iters;
                h->recs[rrc_rec].flops = 2.0 * b3 * (2.0 * iters + (iters > 0 ? iters - 1 : 0));
            }
        }
        if (h->jac_rec >= 0 && h->jac_rec < (int)h->recs.size()) {
            // a rotation of (p, q) updates rows p, q and columns p, q of A and
            // columns p, q of S: 3 x 2 x npad elements at 3 FLOP each
            long long nrot = 0;
            for (int k = 0; k < 64; ++k) nrot += h->hctl->rot_count[k];
            const int np = b + (b & 1);
            h->recs[h->jac_rec].flops = 18.0 * np * (double)nrot;
            h->jac_rec = -1;
        }
        if (meas_here && r_meas > 0.0 && h->last_resid > 0.0 && it > it_meas) {
            const double rate = std::pow(h->last_resid / r_meas, 1.0 / (double)(it - it_meas));
            if (std::isfinite(rate)) h->resid_rate = std::min(0.999, std::max(1e-3, rate));
        }
        r_meas = h->last_resid;
        it_meas = it;
        meas_here = true;
        if (h->hctl->jac_status == 2 || h->hctl->chol_status == 2)
            return fail(CTM_ETIMEOUT, "a device-side barrier timed out");
        if (h->hctl->chol_status == 1) return fail(CTM_ENUMERIC, "Cholesky QR met a non-positive pivot");
        if (h->hctl->numeric_bad) return fail(CTM_ENUMERIC, "non-finite values in the eigen stage");
        if (h->hctl->sub_converged) {
            conv = true;
            ++it;
            break;
        }
        if (it + 1 == max_iters) {
            ++it;
            break;
        }
        ctm::next_block(h->st, N, b, h->T, h->Z, N, h->theta, 1e-12, h->Y);
        count_small(h, 1);
        s = stage_orth(h, h->Y, h->V, h->T, passes);
        if (s != CTM_OK) return s;
        // the Cholesky status is sticky and read at the next iteration's sync
    }
    if (!cold) {
        ctm::gauge_align(h->st, N, b, h->Z, h->Zprev, N, h->theta, h->cfg.tol_cluster, h->ew);
        count_small(h, 3);
    }
    CTM_CUDA(cudaGetLastError());
    *sub_converged = conv;
    *iters_used = it;
    return CTM_OK;
}

ctm_status step_once(ctm_handle* h) {
    const Layout& L = h->lay;
    const int N = L.N, m = L.m;
    const int live_in = h->live;  // basis of this step's C~
    stage_extend(h, h->E);
    bool conv = false;
    int iters = 0;
    ctm_status s = stage_eigen(h, h->cfg.max_subspace_iters, &conv, &iters);
    if (s != CTM_OK) return s;
    const int meff = h->hctl->meff_new;
    if (meff < 1) return fail(CTM_ENUMERIC, "no state kept");
    // a4: U, U' and P <- U^t Sub-CTMRG(P, U', W)
    k_make_U<<<grid_for((size_t)N * m), 256, 0, h->st>>>(N, m, L.q, h->Z, N, h->ctl, h->U, h->Up);
    count_small(h, 1);
    if (is_oz(h)) {
        // X1' = P^t U' (the P planes of the extension are still current)
        s = ozmm(h, N, N, m, {h->P, m, 1, nullptr}, OZ_P, false, {h->Up, m, 1, nullptr}, OZ_SB, true, h->C, N);
        if (s != CTM_OK) return s;
    } else if (L.esz) {
        // X1' = P^t U' (the P operand of the extension is still current)
        pconvert(h, N, m, h->Up, m, nullptr, h->opUp, L.ldm);
        s = ptc(h, N, N, m, h->opP, L.ldm, h->opUp, L.ldm, h->C, N);
        if (s != CTM_OK) return s;
    } else {
        pgemm(h, true, false, N, N, m, h->P, m, h->Up, m, h->C, N);
    }
    pwcontract(h, h->C, h->E, h->mfull, m);
    if (is_oz(h)) {
        s = ozmm(h, m, N, N, {h->U, N, 1, nullptr}, OZ_SA, true, {h->C, N, 1, nullptr}, OZ_BIG, true, h->Pn, m);
        if (s != CTM_OK) return s;
    } else if (L.esz) {
        // P_new = U^t X: operand rows are the columns of U and of X (K = N)
        pconvert(h, m, N, h->U, N, nullptr, h->opU, L.ldN);
        pconvert(h, N, N, h->C, N, nullptr, h->opC, L.ldN);
        s = ptc(h, m, N, N, h->opU, L.ldN, h->opC, L.ldN, h->Pn, m);
        if (s != CTM_OK) return s;
    } else {
        pgemm(h, true, false, m, N, N, h->U, N, h->C, N, h->Pn, m, nullptr, gemm_splits(L, m, N, N));
    }
    // a5/a6
    const int nparts = 512;
    k_sumsq_partial<<<nparts, 256, 0, h->st>>>((size_t)m * N, h->Pn, h->red);
    k_step_finalize<<<1, 256, 0, h->st>>>(m, nparts, h->red, h->theta, h->omega, h->prev, h->ctl);
    k_scale<<<grid_for((size_t)m * N), 256, 0, h->st>>>((size_t)m * N, h->Pn, h->ctl, h->P);
    count_small(h, 3);
    CTM_CUDA(cudaGetLastError());
    s = sync_ctl(h);
    if (s != CTM_OK) return s;
    if (h->hctl->numeric_bad) return fail(CTM_ENUMERIC, "non-finite values in the renormalisation");
    if (h->tcerr) {
        int e = 0;
        CTM_CUDA(cudaMemcpyAsync(&e, h->tcerr, sizeof(int), cudaMemcpyDeviceToHost, h->st));
        CTM_CUDA(cudaStreamSynchronize(h->st));
        if (e) return fail(CTM_ETIMEOUT, "a bounded wait of the tensor-core GEMM gave up");
    }
    // the warm start for the next step is this step's aligned Ritz block
    std::swap(h->Z, h->Zprev);
    h->warm = true;
    h->warm_live = live_in;  // valid for the next step only if its live dim is unchanged
    h->live = meff;
    h->steps += 1;
    ctm_step_info& I = h->last;
    I.kappa = h->hctl->kappa;
    I.delta = h->hctl->delta;
    I.S_E = h->hctl->SE;
    I.residual = h->hctl->resid;
    I.m_eff = meff;
    I.live_dim = L.q * meff;
    I.subspace_iters = iters;
    I.jacobi_sweeps = h->hctl->jac_sweeps;
    I.steps = h->steps;
    I.converged = (h->hctl->delta < h->cfg.tol_spectrum) ? 1 : 0;
    I.rr_refined = h->rr_refined;
    I.rr_jacobi = h->rr_jacobi;
    I.rr_fail_reason = h->oa.fail_reason;
    for (int k = 0; k < 5; ++k) I.rr_fail_counts[k] = h->rr_fail_counts[k];
    I.rr_last_iter = h->oa.last_iter;
    I.rr_last_max = h->oa.last_max;
    for (int k = 0; k < 8; ++k) I.jacobi_rotations[k] = h->hctl->rot_count[k];
    return conv ? CTM_OK : CTM_ENOTCONVERGED;
}

// ------------------------------------------------- beta tangent of a step
// Paper layout P[a + m (g + m s)] <-> device layout P[a + m (s + q g)].
void to_device_layout(const Layout& L, const double* src, double* dst) {
    for (int g = 0; g < L.m; ++g)
        for (int s = 0; s < L.q; ++s)
            for (int a = 0; a < L.m; ++a)
                dst[a + (size_t)L.m * (s + (size_t)L.q * g)] = src[a + (size_t)L.m * (g + (size_t)L.m * s)];
}

void from_device_layout(const Layout& L, const double* src, double* dst) {
    for (int g = 0; g < L.m; ++g)
        for (int s = 0; s < L.q; ++s)
            for (int a = 0; a < L.m; ++a)
                dst[a + (size_t)L.m * (g + (size_t)L.m * s)] = src[a + (size_t)L.m * (s + (size_t)L.q * g)];
}

// Scratch and the primal pieces of one step, kept for any number of tangents.
struct TanCtx {
    char* scratch = nullptr;
    double *X1s = nullptr, *Cs = nullptr, *Cd = nullptr, *X1p = nullptr, *Xd = nullptr, *Pd = nullptr,
           *Pnd = nullptr, *Zd = nullptr, *Ud = nullptr, *Upd = nullptr, *W1 = nullptr, *HH = nullptr,
           *Kc = nullptr, *lamd = nullptr, *omd = nullptr, *Rhs = nullptr, *Y = nullptr, *T = nullptr,
           *Tz = nullptr, *res = nullptr, *part = nullptr;
    // for the observables' tangents: dX1 before its contraction, C~_h, its
    // tangent, C~_h Z and dC~_h Z, the column sums
    double *X1d = nullptr, *Ch = nullptr, *Chd = nullptr, *Bh = nullptr, *Bd = nullptr, *cols = nullptr;
    int meff = 0, bt = 0, iters = 0, live = 0, deflate_iters = 0;
    double kap = 0.0, sc = 0.0, z4 = 0.0;
    std::vector<double> th;
};

ctm_status tan_alloc(ctm_handle* h, TanCtx& c, bool with_obs = false) {
    const Layout& L = h->lay;
    const int m = L.m, N = L.N, b = L.b;
    if (L.q * L.q > 1024) return fail(CTM_EINVAL, "the tangent step needs q <= 32");
    const size_t d = sizeof(double), mN = (size_t)m * N, NN = (size_t)N * N;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t r = off;
        off = align256(off + bytes);
        return r;
    };
    const size_t o_X1 = take(NN * d), o_Cs = take(NN * d), o_Cd = take(NN * d), o_X1p = take(NN * d),
                 o_Xd = take(NN * d), o_Pd = take(mN * d), o_Pnd = take(mN * d), o_Zd = take((size_t)N * m * d),
                 o_Ud = take((size_t)N * m * d), o_Upd = take(mN * d), o_W1 = take((size_t)N * b * d),
                 o_HH = take((size_t)b * b * d), o_K = take((size_t)b * m * d), o_ld = take((size_t)m * d),
                 o_od = take((size_t)m * d), o_Rhs = take((size_t)N * m * d), o_Y = take((size_t)N * m * d),
                 o_T = take((size_t)N * m * d), o_Tz = take((size_t)b * m * d), o_res = take((size_t)b * d),
                 o_part = take((size_t)2 * ctm::kTanParts * d);
    size_t o_X1d = 0, o_Ch = 0, o_Chd = 0, o_Bh = 0, o_Bd = 0, o_cols = 0;
    if (with_obs) {
        o_X1d = take(NN * d);
        o_Ch = take(NN * d);
        o_Chd = take(NN * d);
        o_Bh = take((size_t)N * m * d);
        o_Bd = take((size_t)N * m * d);
        o_cols = take((size_t)5 * m * d);
    }
    if (cudaMalloc(&c.scratch, off) != cudaSuccess) {
        c.scratch = nullptr;
        return fail(CTM_ENOMEM, "cudaMalloc of the tangent scratch failed");
    }
    auto Dp = [&](size_t o) { return (double*)(c.scratch + o); };
    c.X1s = Dp(o_X1);
    c.Cs = Dp(o_Cs);
    c.Cd = Dp(o_Cd);
    c.X1p = Dp(o_X1p);
    c.Xd = Dp(o_Xd);
    c.Pd = Dp(o_Pd);
    c.Pnd = Dp(o_Pnd);
    c.Zd = Dp(o_Zd);
    c.Ud = Dp(o_Ud);
    c.Upd = Dp(o_Upd);
    c.W1 = Dp(o_W1);
    c.HH = Dp(o_HH);
    c.Kc = Dp(o_K);
    c.lamd = Dp(o_ld);
    c.omd = Dp(o_od);
    c.Rhs = Dp(o_Rhs);
    c.Y = Dp(o_Y);
    c.T = Dp(o_T);
    c.Tz = Dp(o_Tz);
    c.res = Dp(o_res);
    c.part = Dp(o_part);
    if (with_obs) {
        c.X1d = Dp(o_X1d);
        c.Ch = Dp(o_Ch);
        c.Chd = Dp(o_Chd);
        c.Bh = Dp(o_Bh);
        c.Bd = Dp(o_Bd);
        c.cols = Dp(o_cols);
    }
    return CTM_OK;
}

void tan_free(ctm_handle* h, TanCtx& c) {
    cudaStreamSynchronize(h->st);
    if (c.scratch) cudaFree(c.scratch);
    c.scratch = nullptr;
}

void tan_gemm(ctm_handle* h, bool tA, bool tB, int M, int Nn, int K, double alpha, const double* A, int lda,
              const double* B, int ldb, double beta, double* C, int ldc, const double* scaleK) {
    int nk = ctm::gemm_f64(h->st, tA, tB, M, Nn, K, alpha, A, lda, B, ldb, beta, C, ldc, scaleK, 1, h->part, 0);
    count_small(h, nk);
}

ctm_status tan_sum(ctm_handle* h, TanCtx& c, size_t n, const double* x, const double* y, double* outv) {
    ctm::dot_partial(h->st, n, x, y, c.part);
    count_small(h, 1);
    std::vector<double> hp(ctm::kTanParts);
    CTM_CUDA(cudaMemcpyAsync(hp.data(), c.part, sizeof(double) * ctm::kTanParts, cudaMemcpyDeviceToHost, h->st));
    CTM_CUDA(cudaStreamSynchronize(h->st));
    double acc = 0.0;
    for (double v : hp) acc += v;
    *outv = acc;
    return CTM_OK;
}

// The primal pieces of one step of Algorithm 3 at the handle's (P, omega):
// X1 (before its contraction), C~ (live block), the Ritz block (warm and
// rotated onto the last step's if the handle is warm), U, U', X1', X (left
// in h->C), P_raw (h->Pn) and kappa = ||P_raw||.
ctm_status tan_prepare(ctm_handle* h, TanCtx& c) {
    const Layout& L = h->lay;
    const int m = L.m, q = L.q, N = L.N, b = L.b;
    const size_t d = sizeof(double), mN = (size_t)m * N, NN = (size_t)N * N;
    cudaStream_t st = h->st;
    c.live = h->live;
    tan_gemm(h, true, false, N, N, m, 1.0, h->P, m, h->P, m, 0.0, h->C, N, h->omega);
    CTM_CUDA(cudaMemcpyAsync(c.X1s, h->C, d * NN, cudaMemcpyDeviceToDevice, st));
    pwcontract(h, h->C, h->E, &h->ctl->live, c.live, false);
    ctm::mask_live(st, N, q, c.live, h->C, N);
    CTM_CUDA(cudaMemcpyAsync(c.Cs, h->C, d * NN, cudaMemcpyDeviceToDevice, st));
    count_small(h, 1);
    bool conv = false;
    ctm_status s = stage_eigen(h, 400, &conv, &c.iters);
    if (s != CTM_OK) return s;
    if (!conv) return fail(CTM_ENOTCONVERGED, "tangent step: the subspace iteration did not converge");
    c.meff = h->hctl->meff_new;
    if (c.meff < 1 || c.meff > m) return fail(CTM_ENUMERIC, "tangent step: no state kept");
    k_make_U<<<grid_for(mN), 256, 0, st>>>(N, m, q, h->Z, N, h->ctl, h->U, h->Up);
    count_small(h, 1);
    tan_gemm(h, true, false, N, N, m, 1.0, h->P, m, h->Up, m, 0.0, h->C, N, nullptr);
    CTM_CUDA(cudaMemcpyAsync(c.X1p, h->C, d * NN, cudaMemcpyDeviceToDevice, st));
    pwcontract(h, h->C, h->E, h->mfull, m);
    tan_gemm(h, true, false, m, N, N, 1.0, h->U, N, h->C, N, 0.0, h->Pn, m, nullptr);
    double nrm2 = 0.0;
    s = tan_sum(h, c, mN, h->Pn, h->Pn, &nrm2);
    if (s != CTM_OK) return s;
    c.kap = sqrt(nrm2);
    if (!(c.kap > 0.0) || !std::isfinite(c.kap)) return fail(CTM_ENUMERIC, "tangent step: zero or non-finite P");
    // Ritz values and residuals of the whole block: the eigen tangent couples
    // the leading pairs that are eigenpairs to 1e-11 |theta_0|
    tan_gemm(h, false, false, N, b, N, 1.0, c.Cs, N, h->Z, N, 0.0, c.W1, N, nullptr);
    ctm::resid_f64(st, N, b, c.W1, h->Z, N, h->theta, c.res);
    count_small(h, 1);
    c.th.assign(b, 0.0);
    std::vector<double> rs(b);
    CTM_CUDA(cudaMemcpyAsync(c.th.data(), h->theta, d * b, cudaMemcpyDeviceToHost, st));
    CTM_CUDA(cudaMemcpyAsync(rs.data(), c.res, d * b, cudaMemcpyDeviceToHost, st));
    CTM_CUDA(cudaStreamSynchronize(st));
    const double a0 = fabs(c.th[0]), tolc = h->cfg.tol_cluster;
    int bt = 0;
    while (bt < b && bt < q * c.live && rs[bt] <= 1e-11 * a0) ++bt;
    while (bt > c.meff && bt < b && fabs(c.th[bt - 1] - c.th[bt]) <= tolc * a0) --bt;
    if (bt < c.meff) return fail(CTM_ENOTCONVERGED, "tangent step: kept Ritz pairs not converged");
    c.bt = bt;
    c.z4 = 0.0;
    for (int i = 0; i < c.meff; ++i) c.z4 += c.th[i] * c.th[i] * c.th[i] * c.th[i];
    c.sc = pow(c.z4, -0.25);
    return CTM_OK;
}

// Input tangent (device layout P_dot, m entries of omega_dot) from the host.
ctm_status tan_upload(ctm_handle* h, TanCtx& c, const double* P_dot_dev_layout, const double* omega_dot) {
    const Layout& L = h->lay;
    CTM_CUDA(cudaMemcpyAsync(c.Pd, P_dot_dev_layout, sizeof(double) * L.m * L.N, cudaMemcpyHostToDevice, h->st));
    CTM_CUDA(cudaMemcpyAsync(c.omd, omega_dot, sizeof(double) * L.m, cudaMemcpyHostToDevice, h->st));
    return CTM_OK;
}

// One tangent of the prepared step along (c.Pd, c.omd) and, with source, W's
// own beta dependence.  Leaves the new P tangent in c.Pd (device layout),
// the new omega tangent in omega_dot_new (m entries) and kappa's in kdot.
ctm_status tan_apply(ctm_handle* h, TanCtx& c, bool source, double* kdot, std::vector<double>* omega_dot_new) {
    const Layout& L = h->lay;
    const int m = L.m, q = L.q, N = L.N, b = L.b, meff = c.meff, bt = c.bt;
    const size_t d = sizeof(double), mN = (size_t)m * N;
    cudaStream_t st = h->st;
    const double tolc = h->cfg.tol_cluster;
    // dX1 = dP^t W P + P^t W dP + P^t dW P (W = diag(omega)), contracted,
    // plus the contraction's own beta-derivative on X1
    tan_gemm(h, true, false, N, N, m, 1.0, c.Pd, m, h->P, m, 0.0, c.Cd, N, h->omega);
    tan_gemm(h, true, false, N, N, m, 1.0, h->P, m, c.Pd, m, 1.0, c.Cd, N, h->omega);
    tan_gemm(h, true, false, N, N, m, 1.0, h->P, m, h->P, m, 1.0, c.Cd, N, c.omd);
    if (c.X1d) CTM_CUDA(cudaMemcpyAsync(c.X1d, c.Cd, sizeof(double) * (size_t)N * N, cudaMemcpyDeviceToDevice, st));
    pwcontract(h, c.Cd, h->E, &h->ctl->live, c.live, false);
    if (source) CTM_CUDA(ctm::wcontract_dbeta(st, q, c.live, c.X1s, N, h->E, h->Eh, c.Cd, N));
    ctm::mask_live(st, N, q, c.live, c.Cd, N);
    count_small(h, source ? 2 : 1);
    // eigen tangent: in-block coupling over the bt pairs, the rest by the
    // deflated iteration Y <- (Rhs + (I - Z Z^t) C~ Y) diag(theta)^-1
    tan_gemm(h, false, false, N, bt, N, 1.0, c.Cd, N, h->Z, N, 0.0, c.W1, N, nullptr);
    tan_gemm(h, true, false, bt, bt, N, 1.0, h->Z, N, c.W1, N, 0.0, c.HH, b, nullptr);
    ctm::tangent_coupling(st, bt, meff, c.HH, b, h->theta, tolc, c.Kc, c.lamd);
    tan_gemm(h, false, false, N, meff, bt, 1.0, h->Z, N, c.Kc, bt, 0.0, c.Zd, N, nullptr);
    CTM_CUDA(cudaMemcpyAsync(c.Rhs, c.W1, d * (size_t)N * meff, cudaMemcpyDeviceToDevice, st));
    tan_gemm(h, false, false, N, meff, bt, -1.0, h->Z, N, c.HH, b, 1.0, c.Rhs, N, nullptr);
    CTM_CUDA(cudaMemsetAsync(c.Y, 0, d * (size_t)N * meff, st));
    ctm::deflate_update(st, N, meff, c.Rhs, nullptr, h->theta, c.Y, c.part);
    count_small(h, 2);
    int dit = 0;
    bool dconv = false;
    std::vector<double> hp(2 * ctm::kTanParts);
    for (dit = 1; dit <= 4000; ++dit) {
        tan_gemm(h, false, false, N, meff, N, 1.0, c.Cs, N, c.Y, N, 0.0, c.T, N, nullptr);
        tan_gemm(h, true, false, bt, meff, N, 1.0, h->Z, N, c.T, N, 0.0, c.Tz, bt, nullptr);
        tan_gemm(h, false, false, N, meff, bt, -1.0, h->Z, N, c.Tz, bt, 1.0, c.T, N, nullptr);
        ctm::deflate_update(st, N, meff, c.Rhs, c.T, h->theta, c.Y, c.part);
        count_small(h, 1);
        if (dit % 4 == 0) {
            CTM_CUDA(cudaMemcpyAsync(hp.data(), c.part, d * hp.size(), cudaMemcpyDeviceToHost, st));
            CTM_CUDA(cudaStreamSynchronize(st));
            double ch = 0.0, my = 0.0;
            for (int k = 0; k < ctm::kTanParts; ++k) {
                ch = std::max(ch, hp[2 * k]);
                my = std::max(my, hp[2 * k + 1]);
            }
            if (!std::isfinite(ch) || !std::isfinite(my))
                return fail(CTM_ENUMERIC, "tangent step: non-finite deflated iterate");
            if (ch <= 1e-14 * std::max(my, 1e-300)) {
                dconv = true;
                break;
            }
        }
    }
    if (!dconv) return fail(CTM_ENOTCONVERGED, "tangent step: the deflated iteration did not converge");
    c.deflate_iters = dit;
    ctm::add_inplace(st, (size_t)N * meff, c.Y, c.Zd);
    CTM_CUDA(cudaMemsetAsync(c.Zd + (size_t)N * meff, 0, d * (size_t)N * (m - meff), st));
    k_make_U<<<grid_for(mN), 256, 0, st>>>(N, m, q, c.Zd, N, h->ctl, c.Ud, c.Upd);
    count_small(h, 2);
    // dX1' = dP^t U' + P^t dU', contracted, plus the contraction's beta-derivative on X1'
    tan_gemm(h, true, false, N, N, m, 1.0, c.Pd, m, h->Up, m, 0.0, c.Xd, N, nullptr);
    tan_gemm(h, true, false, N, N, m, 1.0, h->P, m, c.Upd, m, 1.0, c.Xd, N, nullptr);
    pwcontract(h, c.Xd, h->E, h->mfull, m);
    if (source) {
        CTM_CUDA(ctm::wcontract_dbeta(st, q, m, c.X1p, N, h->E, h->Eh, c.Xd, N));
        count_small(h, 1);
    }
    // dP_raw = dU^t X + U^t dX; dkappa = <P_raw, dP_raw> / kappa
    tan_gemm(h, true, false, m, N, N, 1.0, c.Ud, N, h->C, N, 0.0, c.Pnd, m, nullptr);
    tan_gemm(h, true, false, m, N, N, 1.0, h->U, N, c.Xd, N, 1.0, c.Pnd, m, nullptr);
    double pdot = 0.0;
    ctm_status s = tan_sum(h, c, mN, h->Pn, c.Pnd, &pdot);
    if (s != CTM_OK) return s;
    *kdot = pdot / c.kap;
    ctm::tangent_normalise(st, mN, h->Pn, c.Pnd, 1.0 / c.kap, *kdot / (c.kap * c.kap), c.Pd);
    count_small(h, 1);
    // omega_new = theta (sum theta^4)^(-1/4) on the kept states, and its tangent
    std::vector<double> ld(meff);
    CTM_CUDA(cudaMemcpyAsync(ld.data(), c.lamd, d * meff, cudaMemcpyDeviceToHost, st));
    CTM_CUDA(cudaStreamSynchronize(st));
    double z4d = 0.0;
    for (int i = 0; i < meff; ++i) z4d += 4.0 * c.th[i] * c.th[i] * c.th[i] * ld[i];
    const double scd = -0.25 * pow(c.z4, -1.25) * z4d;
    omega_dot_new->assign(m, 0.0);
    for (int i = 0; i < meff; ++i) (*omega_dot_new)[i] = ld[i] * c.sc + c.th[i] * scd;
    return CTM_OK;
}

// The observables of the prepared state (Eq. 5-6 and the bond energy, over
// the kept states, as ctm_observables) and their tangents along the last
// tan_apply (which must have kept dX1: a context allocated with_obs):
//   M = sum w^4 m_i / sum w^4, m_i = sum_t z_ti^2 mag_t;
//   u = 2 sum w^3 h_i / sum w^4, h_i = z_i^t C~_h z_i, C~_h the extension
//   with the bond energy inserted (inner factor Eh);
//   S_E = -sum p ln p, p = w^4 / sum w^4;
// with w the Ritz values, dw = lambda_dot, dz the eigen tangent, and dC~_h
// the contraction of dX1 with Eh plus its own beta-derivative.
ctm_status tan_observables(ctm_handle* h, TanCtx& c, double val[3], double dval[3]) {
    const Layout& L = h->lay;
    const int m = L.m, q = L.q, N = L.N, meff = c.meff;
    const size_t d = sizeof(double), NN = (size_t)N * N;
    cudaStream_t st = h->st;
    if (!c.X1d) return fail(CTM_EINVAL, "tangent context without the observables' buffers");
    CTM_CUDA(cudaMemcpyAsync(c.Ch, c.X1s, d * NN, cudaMemcpyDeviceToDevice, st));
    pwcontract(h, c.Ch, h->Eh, &h->ctl->live, c.live, false);
    ctm::mask_live(st, N, q, c.live, c.Ch, N);
    CTM_CUDA(cudaMemcpyAsync(c.Chd, c.X1d, d * NN, cudaMemcpyDeviceToDevice, st));
    pwcontract(h, c.Chd, h->Eh, &h->ctl->live, c.live, false);
    CTM_CUDA(ctm::wcontract_dbeta(st, q, c.live, c.X1s, N, h->E, h->Eh, c.Chd, N, true));
    ctm::mask_live(st, N, q, c.live, c.Chd, N);
    count_small(h, 3);
    tan_gemm(h, false, false, N, meff, N, 1.0, c.Ch, N, h->Z, N, 0.0, c.Bh, N, nullptr);
    tan_gemm(h, false, false, N, meff, N, 1.0, c.Chd, N, h->Z, N, 0.0, c.Bd, N, nullptr);
    ctm::column_dots(st, N, meff, h->Z, N, h->Z, N, h->mag, q, c.cols);
    ctm::column_dots(st, N, meff, h->Z, N, c.Zd, N, h->mag, q, c.cols + m);
    ctm::column_dots(st, N, meff, h->Z, N, c.Bh, N, nullptr, q, c.cols + 2 * m);
    ctm::column_dots(st, N, meff, c.Zd, N, c.Bh, N, nullptr, q, c.cols + 3 * m);
    ctm::column_dots(st, N, meff, h->Z, N, c.Bd, N, nullptr, q, c.cols + 4 * m);
    count_small(h, 5);
    std::vector<double> cl((size_t)5 * m), ld(meff);
    CTM_CUDA(cudaMemcpyAsync(cl.data(), c.cols, d * cl.size(), cudaMemcpyDeviceToHost, st));
    CTM_CUDA(cudaMemcpyAsync(ld.data(), c.lamd, d * meff, cudaMemcpyDeviceToHost, st));
    CTM_CUDA(cudaStreamSynchronize(st));
    double z4 = 0.0, z4d = 0.0, Mn = 0.0, Mnd = 0.0, Hn = 0.0, Hnd = 0.0;
    for (int i = 0; i < meff; ++i) {
        const double w = c.th[i], wd = ld[i], w2 = w * w, w3 = w2 * w, w4 = w3 * w;
        const double mi = cl[i], mid = 2.0 * cl[m + i];
        const double hi = cl[2 * m + i], hid = 2.0 * cl[3 * m + i] + cl[4 * m + i];
        z4 += w4;
        z4d += 4.0 * w3 * wd;
        Mn += w4 * mi;
        Mnd += 4.0 * w3 * wd * mi + w4 * mid;
        Hn += w3 * hi;
        Hnd += 3.0 * w2 * wd * hi + w3 * hid;
    }
    const double M = Mn / z4, hb = Hn / z4;
    double S = 0.0, Sd = 0.0;
    for (int i = 0; i < meff; ++i) {
        const double w = c.th[i], w3 = w * w * w, w4 = w3 * w;
        const double p = w4 / z4, pd = 4.0 * w3 * ld[i] / z4 - w4 * z4d / (z4 * z4);
        if (p > 0.0) {
            S -= p * std::log(p);
            Sd -= pd * std::log(p);
        }
    }
    val[0] = M;
    val[1] = 2.0 * hb;
    val[2] = S;
    dval[0] = (Mnd - M * z4d) / z4;
    dval[1] = 2.0 * (Hnd - hb * z4d) / z4;
    dval[2] = Sd;
    return CTM_OK;
}

}  // namespace

// ================================================================ C-ABI
extern "C" {

const char* ctm_last_error(void) { return g_err.c_str(); }

ctm_status ctm_workspace_size(const ctm_config* cfg, size_t* bytes) {
    ctm_status s = validate(cfg);
    if (s != CTM_OK) return s;
    if (!bytes) return fail(CTM_EINVAL, "bytes is NULL");
    *bytes = make_layout(with_defaults(*cfg)).total;
    return CTM_OK;
}

ctm_status ctm_init(ctm_handle** out, const ctm_config* cfg, void* cuda_stream) {
    if (!out) return fail(CTM_EINVAL, "handle pointer is NULL");
    *out = nullptr;
    ctm_status s = validate(cfg);
    if (s != CTM_OK) return s;
    ctm_handle* h = new ctm_handle();
    h->cfg = with_defaults(*cfg);
    h->lay = make_layout(h->cfg);
    const Layout& L = h->lay;
    h->st = (cudaStream_t)cuda_stream;
    if (cfg->workspace) {
        if (cfg->workspace_bytes < L.total) {
            delete h;
            return fail(CTM_ENOMEM, "workspace too small");
        }
        h->ws = (char*)cfg->workspace;
    } else {
        if (cudaMalloc(&h->ws, L.total) != cudaSuccess) {
            delete h;
            return fail(CTM_ENOMEM, "cudaMalloc of the workspace failed");
        }
        h->own_ws = true;
    }
    if (cudaMallocHost(&h->hctl, sizeof(ctm::DevCtl)) != cudaSuccess) {
        ctm_destroy(h);
        return fail(CTM_ENOMEM, "pinned host allocation failed");
    }
    auto D = [&](size_t off) { return (double*)(h->ws + off); };
    h->spins = D(L.off_spins);
    h->E = D(L.off_E);
    h->Eh = D(L.off_Eh);
    h->mag = D(L.off_mag);
    h->P = D(L.off_P);
    h->Pn = D(L.off_Pn);
    h->omega = D(L.off_omega);
    h->prev = D(L.off_prev);
    h->C = D(L.off_C);
    h->V = D(L.off_V);
    h->Y = D(L.off_Y);
    h->Z = D(L.off_Z);
    h->T = D(L.off_T);
    h->Zprev = D(L.off_Zprev);
    h->U = D(L.off_U);
    h->Up = D(L.off_Up);
    h->H = D(L.off_H);
    h->Sb = D(L.off_Sb);
    h->G = D(L.off_G);
    h->Linv = D(L.off_Linv);
    h->theta = D(L.off_theta);
    h->res = D(L.off_res);
    h->part = D(L.off_part);
    h->red = D(L.off_red);
    h->colv = D(L.off_colv);
    if (L.esz) {
        h->opP = h->ws + L.off_opP;
        h->opPw = h->ws + L.off_opPw;
        h->opC = h->ws + L.off_opC;
        h->opV = h->ws + L.off_opV;
        h->opUp = h->ws + L.off_opUp;
        h->opU = h->ws + L.off_opU;
        h->tcerr = (int*)(h->ws + L.off_tcerr);
        h->tcpart = D(L.off_tcpart);
        h->ozSA = h->ws + L.off_ozSA;
        h->ozSB = h->ws + L.off_ozSB;
        h->ozeSA = (int*)(h->ws + L.off_ozeSA);
        h->ozeSB = (int*)(h->ws + L.off_ozeSB);
    }
    if (L.prec == CTM_OZAKI64) {
        h->ozP = h->ws + L.off_ozP;
        h->ozBig = h->ws + L.off_ozBig;
        h->ozSA = h->ws + L.off_ozSA;
        h->ozSB = h->ws + L.off_ozSB;
        h->ozeP = (int*)(h->ws + L.off_ozeP);
        h->ozeBig = (int*)(h->ws + L.off_ozeBig);
        h->ozeSA = (int*)(h->ws + L.off_ozeSA);
        h->ozeSB = (int*)(h->ws + L.off_ozeSB);
        h->tcerr = (int*)(h->ws + L.off_tcerr);
    }
    h->ew.A0 = D(L.off_A0);
    h->ew.A1 = D(L.off_A1);
    h->ew.S = D(L.off_S);
    h->ew.S1 = D(L.off_S1);  // double-buffered S: two Jacobi rounds per grid barrier
    h->ew.diag = D(L.off_diag);
    h->ew.rank = (int*)(h->ws + L.off_rank);
    h->ew.gdots = D(L.off_gd);
    h->ew.gQ = D(L.off_gQ);
    h->ew.gkind = (int*)(h->ws + L.off_gk);
    h->ctl = (ctm::DevCtl*)(h->ws + L.off_ctl);
    h->oa.X = D(L.off_oaX);
    h->oa.W1 = D(L.off_oaW1);
    h->oa.S = D(L.off_oaS);
    h->oa.R = D(L.off_oaR);
    h->oa.E = D(L.off_oaE);
    h->oa.part = D(L.off_oapart);
    h->oa.clus = (int*)(h->ws + L.off_oaclus);
    h->oa.gpart = D(L.off_part);
    h->oa.max_splits = L.splits;
    if (L.off_rrc) {
        ctm::rrc_carve(h->ws + L.off_rrc, L.b, h->rrc);
        h->have_rrc = true;
    }
    h->mfull = (int*)(h->ws + L.off_mfull);
    h->spins_h.assign(cfg->spins, cfg->spins + (size_t)cfg->q * cfg->dim);

    cudaStream_t st = h->st;
    auto bail = [&](cudaError_t e, const char* what) {
        ctm_destroy(h);
        return fail(CTM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    };
    cudaError_t e;
    if ((e = cudaMemsetAsync(h->ws, 0, L.total, st)) != cudaSuccess) return bail(e, "memset");
    if ((e = cudaMemcpyAsync(h->spins, cfg->spins, sizeof(double) * L.q * L.dim, cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
        return bail(e, "spins upload");
    k_weights<<<1, 256, 0, st>>>(L.q, L.dim, h->spins, cfg->beta, cfg->boundary_spin, h->E, h->Eh, h->mag);
    // Algorithm 3 initialisation: p = 1 at alpha = 1, (gamma = 1, s = boundary); omega = e_1.
    const double one = 1.0;
    size_t p0 = 0 + (size_t)L.m * (cfg->boundary_spin + (size_t)L.q * 0);
    if ((e = cudaMemcpyAsync(h->P + p0, &one, sizeof(double), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return bail(e, "P init");
    if ((e = cudaMemcpyAsync(h->omega, &one, sizeof(double), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return bail(e, "omega init");
    k_set_int<<<1, 1, 0, st>>>(&h->ctl->live, 1);
    k_set_int<<<1, 1, 0, st>>>(h->mfull, L.m);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return bail(e, "init sync");
    if ((e = cudaGetLastError()) != cudaSuccess) return bail(e, "init kernels");
    h->live = 1;
    *out = h;
    return CTM_OK;
}

void ctm_destroy(ctm_handle* h) {
    if (!h) return;
    if (h->st) cudaStreamSynchronize(h->st);
    else cudaDeviceSynchronize();
    if (h->own_ws && h->ws) cudaFree(h->ws);
    if (h->hctl) cudaFreeHost(h->hctl);
    for (cudaEvent_t e : h->evpool) cudaEventDestroy(e);
    delete h;
}

ctm_status ctm_profile(ctm_handle* h, int enable) {
    if (!h) return fail(CTM_EINVAL, "handle is NULL");
    CTM_CUDA(cudaStreamSynchronize(h->st));
    h->prof_on = enable != 0;
    h->recs.clear();
    h->evnext = 0;
    h->launches_prof = 0;
    return CTM_OK;
}

ctm_status ctm_profile_read(ctm_handle* h, ctm_prof_entry* out, int max_entries, int* n_entries) {
    if (!h || !out || !n_entries) return fail(CTM_EINVAL, "NULL argument");
    CTM_CUDA(cudaStreamSynchronize(h->st));
    ctm_prof_entry agg[PC_COUNT + 1];
    for (int c = 0; c <= PC_COUNT; ++c) agg[c] = {kProfNames[c], 0, 0.0, 0.0, 0.0};
    for (const auto& r : h->recs) {
        float ms = 0.f;
        CTM_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
        agg[r.cls].launches += r.nk;
        agg[r.cls].ms += ms;
        agg[r.cls].flops += r.flops;
        agg[r.cls].bytes += r.bytes;
    }
    agg[PC_COUNT].launches = h->launches_prof;
    int n = std::min(max_entries, PC_COUNT + 1);
    for (int c = 0; c < n; ++c) out[c] = agg[c];
    *n_entries = n;
    h->recs.clear();
    h->evnext = 0;
    h->launches_prof = 0;
    return CTM_OK;
}

// ---- standalone dense symmetric eigensolver
namespace {
struct SymeigLayout {
    size_t A0, A1, S, diag, rank, ctl, total;
};
SymeigLayout symeig_layout(int n) {
    const size_t np = (size_t)(n + (n & 1) < 2 ? 2 : n + (n & 1));
    SymeigLayout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t r = o;
        o = align256(o + bytes);
        return r;
    };
    L.A0 = take(np * np * sizeof(double));
    L.A1 = take(np * np * sizeof(double));
    L.S = take(np * np * sizeof(double));
    L.diag = take(np * sizeof(double));
    L.rank = take(np * sizeof(int));
    L.ctl = take(sizeof(ctm::DevCtl));
    L.total = o;
    return L;
}
}  // namespace

ctm_status ctm_symeig_workspace_size(int n, size_t* bytes) {
    if (n < 1 || n > 4096 || !bytes) return fail(CTM_EINVAL, "n must be in [1, 4096] and bytes non-NULL");
    *bytes = symeig_layout(n).total;
    return CTM_OK;
}

ctm_status ctm_symeig(int n, const double* A, int lda, double* evals, double* vecs, int ldv, int max_sweeps,
                      void* workspace, size_t workspace_bytes, void* cuda_stream) {
    if (n < 1 || n > 4096) return fail(CTM_EINVAL, "n must be in [1, 4096]");
    if (!A || !evals || !vecs || !workspace) return fail(CTM_EINVAL, "NULL argument");
    if (lda < n || ldv < n) return fail(CTM_EINVAL, "leading dimension smaller than n");
    SymeigLayout L = symeig_layout(n);
    if (workspace_bytes < L.total) return fail(CTM_EINVAL, "workspace too small");
    if (max_sweeps <= 0) max_sweeps = 40;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    char* ws = (char*)workspace;
    ctm::EigWork w{};
    w.A0 = (double*)(ws + L.A0);
    w.A1 = (double*)(ws + L.A1);
    w.S = (double*)(ws + L.S);
    w.diag = (double*)(ws + L.diag);
    w.rank = (int*)(ws + L.rank);
    ctm::DevCtl* ctl = (ctm::DevCtl*)(ws + L.ctl);
    CTM_CUDA(cudaMemsetAsync(ctl, 0, sizeof(ctm::DevCtl), st));
    CTM_CUDA(ctm::jacobi_f64(st, n, A, lda, w, evals, vecs, ldv, max_sweeps, ctl));
    int jst = 0;
    CTM_CUDA(cudaMemcpyAsync(&jst, &ctl->jac_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CTM_CUDA(cudaStreamSynchronize(st));
    if (jst == 2) return fail(CTM_ETIMEOUT, "a device-side barrier of the Jacobi solver gave up");
    if (jst == 1) return fail(CTM_ENOTCONVERGED, "Jacobi reached its sweep cap");
    return CTM_OK;
}

// ---- one contraction in a chosen precision
namespace {
size_t contract_ws(ctm_precision prec, int slices, int M, int N, int K) {
    if (prec == CTM_FP64) return 256;
    if (prec == CTM_OZAKI64)
        return align256(ctm::oz_operand_bytes(M, K, slices, true)) + align256(ctm::oz_operand_bytes(N, K, slices, false)) +
               align256((size_t)M * sizeof(int)) + align256((size_t)N * sizeof(int)) + 256;
    size_t esz = (prec == CTM_BF16) ? 2 : 4;
    size_t ld = (size_t)ctm::tc_ld(K);
    // the split-K partial tiles of the launch shape in force for this GEMM
    const ctm::TcPlan p = tc_plan_for((int)esz, M, N, K);
    const int sl = ctm::tc_plan_slices(p, K, esz == 2, nullptr);
    const size_t part = sl > 1 ? align256((size_t)sl * M * N * sizeof(double)) : 0;
    return align256((size_t)M * ld * esz) + align256((size_t)N * ld * esz) + 256 + part;
}
bool contract_prec_ok(ctm_precision p) {
    return p == CTM_FP64 || p == CTM_TF32 || p == CTM_BF16 || p == CTM_OZAKI64;
}
}  // namespace

ctm_status ctm_contract_workspace_size(ctm_precision prec, int ozaki_slices, int M, int N, int K, size_t* bytes) {
    if (!bytes || M < 1 || N < 1 || K < 1) return fail(CTM_EINVAL, "bad sizes");
    if (!contract_prec_ok(prec)) return fail(CTM_EUNSUPPORTED, "precision not built for ctm_contract");
    if (ozaki_slices == 0) ozaki_slices = 6;
    if (prec == CTM_OZAKI64 && (ozaki_slices < 3 || ozaki_slices > 7))
        return fail(CTM_EINVAL, "ozaki_slices must be in [3, 7]");
    *bytes = contract_ws(prec, ozaki_slices, M, N, K);
    return CTM_OK;
}

ctm_status ctm_contract(ctm_precision prec, int ozaki_slices, int M, int N, int K, const double* A, int lda,
                        const double* B, int ldb, double* D, int ldd, void* workspace, size_t workspace_bytes,
                        void* cuda_stream) {
    if (M < 1 || N < 1 || K < 1) return fail(CTM_EINVAL, "bad sizes");
    if (!A || !B || !D || !workspace) return fail(CTM_EINVAL, "NULL argument");
    if (lda < K || ldb < K || ldd < M) return fail(CTM_EINVAL, "leading dimension too small");
    if (!contract_prec_ok(prec)) return fail(CTM_EUNSUPPORTED, "precision not built for ctm_contract");
    if (ozaki_slices == 0) ozaki_slices = 6;
    if (prec == CTM_OZAKI64 && (ozaki_slices < 3 || ozaki_slices > 7))
        return fail(CTM_EINVAL, "ozaki_slices must be in [3, 7]");
    if (workspace_bytes < contract_ws(prec, ozaki_slices, M, N, K)) return fail(CTM_EINVAL, "workspace too small");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    char* ws = (char*)workspace;
    if (prec == CTM_FP64) {
        ctm::gemm_f64(st, true, false, M, N, K, 1.0, A, lda, B, ldb, 0.0, D, ldd, nullptr, 1, nullptr);
        CTM_CUDA(cudaGetLastError());
        CTM_CUDA(cudaStreamSynchronize(st));
        return CTM_OK;
    }
    int* err = nullptr;
    if (prec == CTM_OZAKI64) {
        size_t oa = align256(ctm::oz_operand_bytes(M, K, ozaki_slices, true));
        size_t ob = align256(ctm::oz_operand_bytes(N, K, ozaki_slices, false));
        void* Ap = ws;
        void* Bp = ws + oa;
        int* eA = (int*)(ws + oa + ob);
        int* eB = (int*)(ws + oa + ob + align256((size_t)M * sizeof(int)));
        err = (int*)(ws + oa + ob + align256((size_t)M * sizeof(int)) + align256((size_t)N * sizeof(int)));
        CTM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
        ctm::oz_split(st, M, K, ozaki_slices, A, lda, nullptr, Ap, true, eA);
        ctm::oz_split(st, N, K, ozaki_slices, B, ldb, nullptr, Bp, false, eB);
        CTM_CUDA(ctm::oz_gemm(st, ozaki_slices, M, N, K, Ap, eA, Bp, eB, D, ldd, err));
    } else {
        const bool bf16 = prec == CTM_BF16;
        const size_t esz = bf16 ? 2 : 4;
        const int ld = ctm::tc_ld(K);
        void* Aop = ws;
        void* Bop = ws + align256((size_t)M * ld * esz);
        err = (int*)(ws + align256((size_t)M * ld * esz) + align256((size_t)N * ld * esz));
        double* part = (double*)((char*)err + 256);
        const size_t cap = (workspace_bytes - ((char*)part - ws)) / sizeof(double);
        const ctm::TcPlan plan = tc_plan_for((int)esz, M, N, K);
        CTM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
        ctm::to_operand(st, bf16, M, K, A, lda, nullptr, Aop, ld);
        ctm::to_operand(st, bf16, N, K, B, ldb, nullptr, Bop, ld);
        CTM_CUDA(ctm::tc_gemm(st, bf16, M, N, K, 1.0, Aop, ld, Bop, ld, 0.0, D, ldd, err, &plan, part, cap));
    }
    int herr = 0;
    CTM_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CTM_CUDA(cudaStreamSynchronize(st));
    if (herr) return fail(CTM_ETIMEOUT, "a bounded wait of the tensor-core GEMM gave up");
    return CTM_OK;
}

// Effective correlation length (Sec. II): Lanczos with full
// reorthogonalisation on the row-to-row transfer matrix T of the current P,
// applied as Phat X (GEMM), the centre-vertex contraction, and A2 P^t (GEMM).
ctm_status ctm_xi(ctm_handle* h, int max_iters, double tol, ctm_xi_result* out) {
    if (!h || !out) return fail(CTM_EINVAL, "NULL argument");
    const Layout& L = h->lay;
    const int m = L.m, q = L.q;
    const size_t mq = (size_t)m * q, n = mq * m;
    int K = max_iters <= 0 ? 64 : max_iters;
    if (K > 120) return fail(CTM_EINVAL, "max_iters must be <= 120");
    if ((size_t)K > n) K = (int)n;
    if (!(tol > 0.0)) tol = 1e-12;
    size_t smem_ta = ctm::xi_w_smem(q, nullptr);
    if (smem_ta > 200 * 1024) return fail(CTM_EINVAL, "q too large for the centre-vertex contraction");
    const int npad = (K + 1) + ((K + 1) & 1);
    const int nb = ctm::xi_dots_blocks(n);
    // scratch (A1 reuses the N x N corner buffer, scratch between steps)
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t r = off;
        off = align256(off + bytes);
        return r;
    };
    const size_t d = sizeof(double);
    const size_t o_A2 = take(mq * mq * d), o_V = take(n * (size_t)(K + 1) * d), o_w = take(n * d),
                 o_part = take((size_t)(K + 1) * nb * d), o_c = take((size_t)(K + 1) * d),
                 o_alpha = take((size_t)(K + 1) * d), o_beta = take((size_t)(K + 1) * d),
                 o_nrm = take(d), o_Tk = take((size_t)K * K * d), o_Sk = take((size_t)K * K * d),
                 o_th = take((size_t)npad * d), o_A0 = take((size_t)npad * npad * d),
                 o_B1 = take((size_t)npad * npad * d), o_S = take((size_t)npad * npad * d),
                 o_dg = take((size_t)npad * d), o_rk = take((size_t)npad * sizeof(int));
    char* scratch = nullptr;
    if (cudaMalloc(&scratch, off) != cudaSuccess) return fail(CTM_ENOMEM, "cudaMalloc of the Lanczos scratch failed");
    auto Dp = [&](size_t o) { return (double*)(scratch + o); };
    double *A1 = h->C, *A2 = Dp(o_A2), *V = Dp(o_V), *w = Dp(o_w), *part = Dp(o_part), *c = Dp(o_c),
           *alpha = Dp(o_alpha), *beta = Dp(o_beta), *nrm = Dp(o_nrm), *Tk = Dp(o_Tk), *Sk = Dp(o_Sk),
           *theta = Dp(o_th);
    ctm::EigWork ew{};
    ew.A0 = Dp(o_A0);
    ew.A1 = Dp(o_B1);
    ew.S = Dp(o_S);
    ew.diag = Dp(o_dg);
    ew.rank = (int*)(scratch + o_rk);
    auto done = [&](ctm_status st) {
        cudaStreamSynchronize(h->st);
        cudaFree(scratch);
        return st;
    };
    cudaStream_t st = h->st;
    auto vec = [&](int j) { return V + n * (size_t)j; };
    // seeded Gaussian start vector, normalised
    ctm::randn_block(st, (int)n, 1, vec(0), (int)n, h->seed ^ 0x5851f42d4c957f2dull);
    ctm::xi_dots(st, n, 1, vec(0), n, vec(0), part, nrm);
    ctm::xi_normalise(st, n, vec(0), nrm, vec(0), c);
    count_small(h, 4);
    double lam[4] = {0, 0, 0, 0}, res[4] = {0, 0, 0, 0};
    int it = 0, conv = 0;
    for (int j = 0; j < K; ++j) {
        // w = T v_j
        pgemm(h, false, false, (int)mq, (int)mq, m, h->P, (int)mq, vec(j), m, A1, (int)mq);
        cudaEvent_t a = prof_begin(h);
        cudaError_t ce = ctm::xi_wcontract(st, m, q, A1, h->E, A2);
        if (ce != cudaSuccess) return done(fail(CTM_ECUDA, std::string("xi_wcontract: ") + cudaGetErrorString(ce)));
        prof_end(h, a, PC_XI_W, 1, 4.0 * q * q * (double)q * m * m, 2.0 * d * mq * mq);
        pgemm(h, false, true, (int)mq, m, (int)mq, A2, (int)mq, h->P, m, w, (int)mq);
        // alpha_j = v_j . w (first pass), then two passes of classical
        // Gram-Schmidt against v_0..v_j, then beta_j = ||w||, v_{j+1} = w / beta_j
        a = prof_begin(h);
        ctm::xi_dots(st, n, j + 1, V, n, w, part, c);
        CTM_CUDA(cudaMemcpyAsync(alpha + j, c + j, d, cudaMemcpyDeviceToDevice, st));
        ctm::xi_sub_multi(st, n, j + 1, V, n, c, w);
        ctm::xi_dots(st, n, j + 1, V, n, w, part, c);
        ctm::xi_sub_multi(st, n, j + 1, V, n, c, w);
        ctm::xi_dots(st, n, 1, w, n, w, part, nrm);
        ctm::xi_normalise(st, n, w, nrm, vec(j + 1), beta + j);
        prof_end(h, a, PC_XI_VEC, 9, 0.0, d * n * (4.0 * (j + 1) + 6.0));
        it = j + 1;
        if (it % 4 != 0 && it != K) continue;
        // Ritz values of the tridiagonal matrix, sorted by |theta|
        ctm::xi_tridiag(st, it, alpha, beta, Tk);
        ce = ctm::jacobi_f64(st, it, Tk, it, ew, theta, Sk, it, 40, h->ctl);
        count_small(h, 5);
        if (ce != cudaSuccess) return done(fail(CTM_ECUDA, std::string("jacobi_f64: ") + cudaGetErrorString(ce)));
        double hb[8];
        const int nr = std::min(4, it);
        std::vector<double> last(nr);
        CTM_CUDA(cudaMemcpyAsync(hb, theta, sizeof(double) * nr, cudaMemcpyDeviceToHost, st));
        for (int i = 0; i < nr; ++i)
            CTM_CUDA(cudaMemcpyAsync(&last[i], Sk + (it - 1) + (size_t)it * i, d, cudaMemcpyDeviceToHost, st));
        double bj = 0.0;
        CTM_CUDA(cudaMemcpyAsync(&bj, beta + j, d, cudaMemcpyDeviceToHost, st));
        ctm_status s0 = sync_ctl(h);
        if (s0 != CTM_OK) return done(s0);
        if (h->hctl->jac_status == 2) return done(fail(CTM_ETIMEOUT, "a device-side barrier timed out"));
        for (int i = 0; i < 4; ++i) {
            lam[i] = i < nr ? hb[i] : 0.0;
            res[i] = i < nr ? fabs(bj * last[i]) : 0.0;
        }
        const double scale = fabs(lam[0]) > 0.0 ? fabs(lam[0]) : 1.0;
        for (int i = 0; i < 4; ++i) res[i] /= scale;
        const bool invariant = bj <= 1e-14 * scale;
        if (invariant || (res[0] <= tol && (nr < 2 || res[1] <= tol))) {
            conv = 1;
            break;
        }
    }
    out->iterations = it;
    out->converged = conv;
    for (int i = 0; i < 4; ++i) {
        out->lambda[i] = lam[i];
        out->residual[i] = res[i];
    }
    out->xi = (lam[1] != 0.0) ? 1.0 / log(fabs(lam[0] / lam[1])) : 0.0;
    return done(conv ? CTM_OK : fail(CTM_ENOTCONVERGED, "Lanczos reached max_iters"));
}

ctm_status ctm_tc_plan_set(ctm_precision prec, int M, int N, int K, int bn, int splits) {
    if (prec != CTM_TF32 && prec != CTM_BF16) return fail(CTM_EINVAL, "launch shapes exist for TF32 / BF16 only");
    if (M < 1 || N < 1 || K < 1) return fail(CTM_EINVAL, "bad sizes");
    const int esz = prec == CTM_BF16 ? 2 : 4;
    std::lock_guard<std::mutex> g(g_tc_mu);
    if (splits == 0) {
        g_tc_plans.erase(TcKey{esz, M, N, K});
        return CTM_OK;
    }
    if (bn != 64 && bn != 128 && bn != 256) return fail(CTM_EINVAL, "bn must be 64, 128 or 256");
    if (splits < 1 || splits > 16) return fail(CTM_EINVAL, "splits must be in [1, 16] (0 clears)");
    g_tc_plans[TcKey{esz, M, N, K}] = ctm::TcPlan{bn, splits};
    return CTM_OK;
}

ctm_status ctm_tc_plan_get(ctm_precision prec, int M, int N, int K, int* bn, int* splits) {
    if (prec != CTM_TF32 && prec != CTM_BF16) return fail(CTM_EINVAL, "launch shapes exist for TF32 / BF16 only");
    if (!bn || !splits) return fail(CTM_EINVAL, "NULL argument");
    const ctm::TcPlan p = tc_plan_for(prec == CTM_BF16 ? 2 : 4, M, N, K);
    *bn = p.bn;
    *splits = ctm::tc_plan_slices(p, K, prec == CTM_BF16, nullptr);
    return CTM_OK;
}

ctm_status ctm_launch_count(ctm_handle* h, long long* launches) {
    if (!h || !launches) return fail(CTM_EINVAL, "NULL argument");
    *launches = h->launches;
    return CTM_OK;
}

ctm_status ctm_step(ctm_handle* h, int nsteps, int* steps_done, ctm_step_info* info) {
    if (!h) return fail(CTM_EINVAL, "handle is NULL");
    if (nsteps < 0) return fail(CTM_EINVAL, "nsteps < 0");
    int done = 0;
    ctm_status worst = CTM_OK;
    for (int k = 0; k < nsteps; ++k) {
        ctm_status s = step_once(h);
        if (s != CTM_OK && s != CTM_ENOTCONVERGED) {
            if (steps_done) *steps_done = done;
            return s;
        }
        if (s == CTM_ENOTCONVERGED) worst = s;
        ++done;
        if (h->last.converged) break;
    }
    if (steps_done) *steps_done = done;
    if (info) *info = h->last;
    if (worst != CTM_OK) fail(worst, "a subspace iteration reached its cap");
    return worst;
}

ctm_status ctm_observables(ctm_handle* h, ctm_obs* out) {
    if (!h || !out) return fail(CTM_EINVAL, "NULL argument");
    const Layout& L = h->lay;
    const int N = L.N, b = L.b;
    stage_extend(h, h->E);
    bool conv = false;
    int iters = 0;
    ctm_status s = stage_eigen(h, h->cfg.max_subspace_iters, &conv, &iters);
    if (s != CTM_OK) return s;
    // the eigen stage aligned Z to Zprev; keep it as the warm start
    std::swap(h->Z, h->Zprev);
    h->warm = true;
    h->warm_live = h->live;
    // impurity corner C~_h (bond energy inserted), then Yh = C~_h Z
    stage_extend(h, h->Eh);
    if (is_oz(h)) {
        s = ozmm(h, N, b, N, {h->C, N, 1, nullptr}, OZ_BIG, true, {h->Zprev, N, 1, nullptr}, OZ_SB, true, h->Y, N);
        if (s != CTM_OK) return s;
    } else {
        pgemm(h, false, false, N, b, N, h->C, N, h->Zprev, N, h->Y, N);
    }
    k_obs_cols<<<b, 256, 0, h->st>>>(N, L.q, b, h->Zprev, h->Y, h->mag, h->colv);
    k_obs_finalize<<<1, 32, 0, h->st>>>(b, h->theta, h->colv, h->ctl);
    count_small(h, 2);
    CTM_CUDA(cudaGetLastError());
    s = sync_ctl(h);
    if (s != CTM_OK) return s;
    const ctm::DevCtl& c = *h->hctl;
    double kappa = h->last.kappa > 0.0 ? h->last.kappa : c.kappa;
    out->f = (h->cfg.beta > 0.0 && kappa > 0.0) ? -0.5 / h->cfg.beta * log(kappa) : NAN;
    out->M = c.obs_M_num / c.obs_z4;
    out->u = 2.0 * c.obs_u_num / c.obs_z4;
    out->S_E = c.obs_SE;
    out->delta = h->last.delta;
    out->steps = h->steps;
    out->converged = h->last.converged;
    return conv ? CTM_OK : fail(CTM_ENOTCONVERGED, "observables: subspace iteration reached its cap");
}

ctm_status ctm_tangent_step(ctm_handle* h, const double* P_dot, const double* omega_dot, int source,
                            ctm_tangent_out* out) {
    if (!h || !P_dot || !omega_dot || !out) return fail(CTM_EINVAL, "NULL argument");
    if (h->lay.prec != CTM_FP64) return fail(CTM_EUNSUPPORTED, "the tangent step is built for the FP64 form");
    if (!out->P_new || !out->omega_new || !out->P_dot_new || !out->omega_dot_new)
        return fail(CTM_EINVAL, "NULL output array");
    const Layout& L = h->lay;
    const int m = L.m, q = L.q;
    TanCtx c;
    ctm_status s = tan_alloc(h, c);
    if (s != CTM_OK) return s;
    auto done = [&](ctm_status st) {
        tan_free(h, c);
        h->warm = false;  // the Ritz block left behind is not aligned to anything
        h->warm_live = -1;
        return st;
    };
    h->warm = false;  // a cold subspace iteration: the output basis is the eigensolver's own
    s = tan_prepare(h, c);
    if (s != CTM_OK) return done(s);
    std::vector<double> pin((size_t)m * L.N);
    to_device_layout(L, P_dot, pin.data());
    s = tan_upload(h, c, pin.data(), omega_dot);
    if (s != CTM_OK) return done(s);
    double kdot = 0.0;
    std::vector<double> odn;
    s = tan_apply(h, c, source != 0, &kdot, &odn);
    if (s != CTM_OK) return done(s);
    std::vector<double> pn((size_t)m * L.N), pdn((size_t)m * L.N);
    {
        cudaError_t e = cudaMemcpyAsync(pn.data(), h->Pn, sizeof(double) * pn.size(), cudaMemcpyDeviceToHost, h->st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(pdn.data(), c.Pd, sizeof(double) * pdn.size(), cudaMemcpyDeviceToHost, h->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
        if (e != cudaSuccess) return done(fail(CTM_ECUDA, std::string("ctm_tangent_step: ") + cudaGetErrorString(e)));
    }
    for (double& v : pn) v /= c.kap;
    from_device_layout(L, pn.data(), out->P_new);
    from_device_layout(L, pdn.data(), out->P_dot_new);
    for (int i = 0; i < m; ++i) {
        out->omega_new[i] = i < c.meff ? c.th[i] * c.sc : 0.0;
        out->omega_dot_new[i] = odn[i];
    }
    (void)q;
    out->kappa = c.kap;
    out->kappa_dot = kdot;
    out->m_eff = c.meff;
    out->ritz_pairs = c.bt;
    out->deflate_iterations = c.deflate_iters;
    out->subspace_iterations = c.iters;
    return done(CTM_OK);
}

ctm_status ctm_step_backward(ctm_handle* h, const ctm_obs* grad_obs, double* grad_beta) {
    if (!h || !grad_obs || !grad_beta) return fail(CTM_EINVAL, "NULL argument");
    if (h->lay.prec != CTM_FP64) return fail(CTM_EUNSUPPORTED, "the backward step is built for the FP64 form");
    if (!h->warm || h->steps < 1) return fail(CTM_EINVAL, "ctm_step_backward needs a state reached by ctm_step");
    const bool need_obs = grad_obs->M != 0.0 || grad_obs->u != 0.0 || grad_obs->S_E != 0.0;
    const Layout& L = h->lay;
    const int m = L.m, N = L.N;
    TanCtx c;
    ctm_status s = tan_alloc(h, c, need_obs);
    if (s != CTM_OK) return s;
    auto done = [&](ctm_status st) {
        tan_free(h, c);
        return st;
    };
    // the gauge-fixed step at the state: its Ritz block rotated onto the last
    // step's, so that at a fixed point P_new repeats P entry by entry
    s = tan_prepare(h, c);
    if (s != CTM_OK) return done(s);
    const size_t mN = (size_t)m * N;
    std::vector<double> pn(mN), p0(mN), om0(m);
    {
        cudaError_t e = cudaMemcpyAsync(pn.data(), h->Pn, sizeof(double) * mN, cudaMemcpyDeviceToHost, h->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(p0.data(), h->P, sizeof(double) * mN, cudaMemcpyDeviceToHost, h->st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(om0.data(), h->omega, sizeof(double) * m, cudaMemcpyDeviceToHost, h->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
        if (e != cudaSuccess) return done(fail(CTM_ECUDA, std::string("ctm_step_backward: ") + cudaGetErrorString(e)));
    }
    {
        // entries weighted by |omega| of both block legs (device layout
        // a + m (s + q g)): states deep in the spectrum with nearly equal
        // eigenvalues are fixed only to rounding over their gap
        double change = 0.0;
        const double a1 = std::fabs(om0[0]) > 0.0 ? std::fabs(om0[0]) : 1.0;
        for (size_t e = 0; e < mN; ++e) {
            const int a = (int)(e % m), g = (int)((e / m) / L.q);
            const double wgt = std::fabs(om0[a]) * std::fabs(om0[g]) / (a1 * a1);
            change = std::max(change, wgt * std::fabs(pn[e] / c.kap - p0[e]));
        }
        if (!(change < 1e-8))
            return done(fail(CTM_ENOTCONVERGED, "ctm_step_backward: the state is not a fixed point of the step"));
    }
    // right side: the tangent of the step along W's own beta dependence
    const int meff = c.meff;
    const size_t n = mN + (size_t)meff;
    std::vector<double> zeroP(mN, 0.0), zeroO(m, 0.0), rhs(n), x(n, 0.0);
    double kd_b = 0.0;
    std::vector<double> odn;
    auto apply = [&](const double* Pin, const double* Oin, bool source, double* out_vec, double* kdot) -> ctm_status {
        std::vector<double> oin(m, 0.0);
        for (int i = 0; i < meff; ++i) oin[i] = Oin[i];
        ctm_status st = tan_upload(h, c, Pin, oin.data());
        if (st != CTM_OK) return st;
        st = tan_apply(h, c, source, kdot, &odn);
        if (st != CTM_OK) return st;
        if (out_vec) {
            CTM_CUDA(cudaMemcpyAsync(out_vec, c.Pd, sizeof(double) * mN, cudaMemcpyDeviceToHost, h->st));
            CTM_CUDA(cudaStreamSynchronize(h->st));
            for (int i = 0; i < meff; ++i) out_vec[mN + i] = odn[i];
        }
        return CTM_OK;
    };
    s = apply(zeroP.data(), zeroO.data(), true, rhs.data(), &kd_b);
    if (s != CTM_OK) return done(s);
    // GMRES on (I - J) x = rhs, J x = one tangent step without the source
    std::vector<double> Jv(n);
    auto op = [&](const std::vector<double>& v, std::vector<double>& w) -> ctm_status {
        double kd = 0.0;
        ctm_status st = apply(v.data(), v.data() + mN, false, Jv.data(), &kd);
        if (st != CTM_OK) return st;
        for (size_t i = 0; i < n; ++i) w[i] = v[i] - Jv[i];
        return CTM_OK;
    };
    int gm_iters = 0;
    double gm_res = 0.0;
    ctm_status op_status = CTM_OK;
    auto op_host = [&](const std::vector<double>& v, std::vector<double>& w) -> bool {
        op_status = op(v, w);
        return op_status == CTM_OK;
    };
    const int gst = ctm::host_gmres(op_host, rhs, x, 1e-12, 300, &gm_iters, &gm_res);
    if (gst == ctm::kGmresOpFailed) return done(op_status);
    if (gst != ctm::kGmresOk) return done(fail(CTM_ENOTCONVERGED, "ctm_step_backward: GMRES did not converge"));
    // d kappa / d beta at the fixed point: the step's kappa tangent along x
    // with the source
    double kdot = 0.0;
    s = apply(x.data(), x.data() + mN, true, nullptr, &kdot);
    if (s != CTM_OK) return done(s);
    const double beta = h->cfg.beta, lk = std::log(c.kap);
    // f = -ln kappa / (2 beta)
    const double df = 0.5 * lk / (beta * beta) - 0.5 * kdot / (beta * c.kap);
    double g = grad_obs->f * df;
    if (need_obs) {
        // M, u, S_E of the fixed point and their tangents along x (the last
        // tan_apply above, with the source)
        double val[3], dval[3];
        s = tan_observables(h, c, val, dval);
        if (s != CTM_OK) return done(s);
        g += grad_obs->M * dval[0] + grad_obs->u * dval[1] + grad_obs->S_E * dval[2];
    }
    *grad_beta = g;
    h->last_backward_iters = gm_iters;
    h->last_backward_residual = gm_res;
    return done(CTM_OK);
}

ctm_status ctm_get_spectrum(ctm_handle* h, double* omega) {
    if (!h || !omega) return fail(CTM_EINVAL, "NULL argument");
    CTM_CUDA(cudaMemcpyAsync(omega, h->omega, sizeof(double) * h->lay.m, cudaMemcpyDeviceToHost, h->st));
    CTM_CUDA(cudaStreamSynchronize(h->st));
    return CTM_OK;
}

ctm_status ctm_get_state(ctm_handle* h, double* P, double* omega, int* live) {
    if (!h) return fail(CTM_EINVAL, "handle is NULL");
    const Layout& L = h->lay;
    if (P) {
        std::vector<double> tmp((size_t)L.m * L.N);
        CTM_CUDA(cudaMemcpyAsync(tmp.data(), h->P, sizeof(double) * tmp.size(), cudaMemcpyDeviceToHost, h->st));
        CTM_CUDA(cudaStreamSynchronize(h->st));
        for (int g = 0; g < L.m; ++g)
            for (int s = 0; s < L.q; ++s)
                for (int a = 0; a < L.m; ++a)
                    P[a + (size_t)L.m * (g + (size_t)L.m * s)] = tmp[a + (size_t)L.m * (s + (size_t)L.q * g)];
    }
    if (omega) {
        CTM_CUDA(cudaMemcpyAsync(omega, h->omega, sizeof(double) * L.m, cudaMemcpyDeviceToHost, h->st));
        CTM_CUDA(cudaStreamSynchronize(h->st));
    }
    if (live) *live = h->live;
    return CTM_OK;
}

ctm_status ctm_set_state(ctm_handle* h, const double* P, const double* omega, int live) {
    if (!h || !P || !omega) return fail(CTM_EINVAL, "NULL argument");
    const Layout& L = h->lay;
    if (live < 1 || live > L.m) return fail(CTM_EINVAL, "live out of range");
    std::vector<double> tmp((size_t)L.m * L.N);
    for (int g = 0; g < L.m; ++g)
        for (int s = 0; s < L.q; ++s)
            for (int a = 0; a < L.m; ++a)
                tmp[a + (size_t)L.m * (s + (size_t)L.q * g)] = P[a + (size_t)L.m * (g + (size_t)L.m * s)];
    CTM_CUDA(cudaMemcpyAsync(h->P, tmp.data(), sizeof(double) * tmp.size(), cudaMemcpyHostToDevice, h->st));
    CTM_CUDA(cudaMemcpyAsync(h->omega, omega, sizeof(double) * L.m, cudaMemcpyHostToDevice, h->st));
    k_set_int<<<1, 1, 0, h->st>>>(&h->ctl->live, live);
    k_set_int<<<1, 1, 0, h->st>>>(&h->ctl->have_prev, 0);
    CTM_CUDA(cudaStreamSynchronize(h->st));
    h->live = live;
    h->warm = false;
    h->warm_live = -1;
    h->last_resid = 0.0;
    h->resid_rate = 0.5;
    h->rr_fail_streak = 0;
    return CTM_OK;
}

namespace {
struct SaveHeader {
    uint64_t magic;
    int q, m, b, N;
    int live, steps, warm, warm_live;
    uint64_t seed;
    ctm_step_info last;
    // host-side state of the subspace iteration's schedule (Rayleigh-Ritz
    // timing), so that a resumed run repeats the uninterrupted one
    double last_resid, resid_rate;
    int rr_fail_streak, pad;
};
const uint64_t kMagic = 0x43544d5247423330ull;  // "CTMRGB30"
}  // namespace

ctm_status ctm_save(ctm_handle* h, void* buf, size_t* len) {
    if (!h || !len) return fail(CTM_EINVAL, "NULL argument");
    const Layout& L = h->lay;
    size_t need = sizeof(SaveHeader) +
                  sizeof(double) * ((size_t)L.m * L.N + 2 * (size_t)L.m + (size_t)L.N * L.b + (size_t)L.npad) +
                  sizeof(ctm::DevCtl);
    if (!buf) {
        *len = need;
        return CTM_OK;
    }
    if (*len < need) return fail(CTM_EINVAL, "buffer too small");
    SaveHeader hd{kMagic,      L.q,       L.m,           L.b,           L.N,     h->live,
                  h->steps,    h->warm ? 1 : 0, h->warm_live, h->seed,    h->last, h->last_resid,
                  h->resid_rate, h->rr_fail_streak, 0};
    char* p = (char*)buf;
    memcpy(p, &hd, sizeof(hd));
    p += sizeof(hd);
    CTM_CUDA(cudaMemcpyAsync(p, h->P, sizeof(double) * L.m * L.N, cudaMemcpyDeviceToHost, h->st));
    p += sizeof(double) * L.m * L.N;
    CTM_CUDA(cudaMemcpyAsync(p, h->omega, sizeof(double) * L.m, cudaMemcpyDeviceToHost, h->st));
    p += sizeof(double) * L.m;
    CTM_CUDA(cudaMemcpyAsync(p, h->prev, sizeof(double) * L.m, cudaMemcpyDeviceToHost, h->st));
    p += sizeof(double) * L.m;
    CTM_CUDA(cudaMemcpyAsync(p, h->Zprev, sizeof(double) * L.N * L.b, cudaMemcpyDeviceToHost, h->st));
    p += sizeof(double) * L.N * L.b;
    // the last Ritz values scale the next step's first block
    CTM_CUDA(cudaMemcpyAsync(p, h->theta, sizeof(double) * L.npad, cudaMemcpyDeviceToHost, h->st));
    p += sizeof(double) * L.npad;
    CTM_CUDA(cudaMemcpyAsync(p, h->ctl, sizeof(ctm::DevCtl), cudaMemcpyDeviceToHost, h->st));
    CTM_CUDA(cudaStreamSynchronize(h->st));
    *len = need;
    return CTM_OK;
}

ctm_status ctm_load(ctm_handle* h, const void* buf, size_t len) {
    if (!h || !buf) return fail(CTM_EINVAL, "NULL argument");
    const Layout& L = h->lay;
    size_t need = sizeof(SaveHeader) +
                  sizeof(double) * ((size_t)L.m * L.N + 2 * (size_t)L.m + (size_t)L.N * L.b + (size_t)L.npad) +
                  sizeof(ctm::DevCtl);
    if (len < need) return fail(CTM_EINVAL, "buffer too small");
    SaveHeader hd;
    memcpy(&hd, buf, sizeof(hd));
    if (hd.magic != kMagic || hd.q != L.q || hd.m != L.m || hd.b != L.b || hd.N != L.N)
        return fail(CTM_EINVAL, "checkpoint does not match this configuration");
    const char* p = (const char*)buf + sizeof(hd);
    CTM_CUDA(cudaMemcpyAsync(h->P, p, sizeof(double) * L.m * L.N, cudaMemcpyHostToDevice, h->st));
    p += sizeof(double) * L.m * L.N;
    CTM_CUDA(cudaMemcpyAsync(h->omega, p, sizeof(double) * L.m, cudaMemcpyHostToDevice, h->st));
    p += sizeof(double) * L.m;
    CTM_CUDA(cudaMemcpyAsync(h->prev, p, sizeof(double) * L.m, cudaMemcpyHostToDevice, h->st));
    p += sizeof(double) * L.m;
    CTM_CUDA(cudaMemcpyAsync(h->Zprev, p, sizeof(double) * L.N * L.b, cudaMemcpyHostToDevice, h->st));
    p += sizeof(double) * L.N * L.b;
    CTM_CUDA(cudaMemcpyAsync(h->theta, p, sizeof(double) * L.npad, cudaMemcpyHostToDevice, h->st));
    p += sizeof(double) * L.npad;
    CTM_CUDA(cudaMemcpyAsync(h->ctl, p, sizeof(ctm::DevCtl), cudaMemcpyHostToDevice, h->st));
    CTM_CUDA(cudaStreamSynchronize(h->st));
    h->live = hd.live;
    h->steps = hd.steps;
    h->warm = hd.warm != 0;
    h->warm_live = hd.warm_live;
    h->seed = hd.seed;
    h->last = hd.last;
    h->last_resid = hd.last_resid;
    h->resid_rate = hd.resid_rate;
    h->rr_fail_streak = hd.rr_fail_streak;
    return CTM_OK;
}

ctm_status ctm_extend(ctm_handle* h) {
    if (!h) return fail(CTM_EINVAL, "handle is NULL");
    stage_extend(h, h->E);
    CTM_CUDA(cudaGetLastError());
    CTM_CUDA(cudaStreamSynchronize(h->st));
    return CTM_OK;
}

ctm_status ctm_get_ctilde(ctm_handle* h, const int* rows, const int* cols, int count, double* out) {
    if (!h || (count > 0 && (!rows || !cols || !out))) return fail(CTM_EINVAL, "NULL argument");
    if (count <= 0) return CTM_OK;
    const Layout& L = h->lay;
    std::vector<long long> idx((size_t)count);
    for (int i = 0; i < count; ++i) {
        int r = rows[i], c = cols[i];
        if (r < 0 || r >= L.N || c < 0 || c >= L.N) return fail(CTM_EINVAL, "index out of range");
        long long tr = (r / L.m) + (long long)L.q * (r % L.m);  // paper gamma + m s -> device s + q gamma
        long long tc = (c / L.m) + (long long)L.q * (c % L.m);
        idx[i] = tr + (long long)L.N * tc;
    }
    long long* d_idx = nullptr;
    double* d_out = nullptr;
    CTM_CUDA(cudaMallocAsync(&d_idx, sizeof(long long) * idx.size(), h->st));
    CTM_CUDA(cudaMallocAsync(&d_out, sizeof(double) * count, h->st));
    CTM_CUDA(cudaMemcpyAsync(d_idx, idx.data(), sizeof(long long) * idx.size(), cudaMemcpyHostToDevice, h->st));
    k_gather<<<grid_for((size_t)count), 256, 0, h->st>>>(count, d_idx, h->C, d_out);
    CTM_CUDA(cudaMemcpyAsync(out, d_out, sizeof(double) * count, cudaMemcpyDeviceToHost, h->st));
    CTM_CUDA(cudaFreeAsync(d_idx, h->st));
    CTM_CUDA(cudaFreeAsync(d_out, h->st));
    CTM_CUDA(cudaStreamSynchronize(h->st));
    return CTM_OK;
}

ctm_status ctm_eigen(ctm_handle* h, double* evals, double* vecs, int* b_out) {
    if (!h) return fail(CTM_EINVAL, "handle is NULL");
    const Layout& L = h->lay;
    bool conv = false;
    int iters = 0;
    ctm_status s = stage_eigen(h, h->cfg.max_subspace_iters, &conv, &iters);
    if (s != CTM_OK) return s;
    if (b_out) *b_out = L.b;
    if (evals) CTM_CUDA(cudaMemcpyAsync(evals, h->theta, sizeof(double) * L.b, cudaMemcpyDeviceToHost, h->st));
    if (vecs) {
        std::vector<double> tmp((size_t)L.N * L.b);
        CTM_CUDA(cudaMemcpyAsync(tmp.data(), h->Z, sizeof(double) * tmp.size(), cudaMemcpyDeviceToHost, h->st));
        CTM_CUDA(cudaStreamSynchronize(h->st));
        for (int i = 0; i < L.b; ++i)
            for (int g = 0; g < L.m; ++g)
                for (int sp = 0; sp < L.q; ++sp)
                    vecs[(g + (size_t)L.m * sp) + (size_t)L.N * i] = tmp[(sp + (size_t)L.q * g) + (size_t)L.N * i];
    }
    CTM_CUDA(cudaStreamSynchronize(h->st));
    return conv ? CTM_OK : fail(CTM_ENOTCONVERGED, "subspace iteration reached its cap");
}

// ------------------------------------------------------------- autotuner
}  // extern "C"
namespace {
// The FP64-emulating form: K slices of the two long-K products of the step,
// C~ V (N x b x N) and U^t X (m x N x N), whose output tiles (200 and 160 at
// m = 256) fill the 152 SMs in one and a bit waves.
ctm_status tune_oz(ctm_handle* h, int reps, ctm_tune_entry* out, int max_out, int* n_out) {
    const Layout& L = h->lay;
    const int S = L.slices, N = L.N, b = L.b, m = L.m;
    auto opA = [&](int R, int K) { return ctm::oz_operand_bytes(R, K, S, true); };
    auto opB = [&](int R, int K) { return ctm::oz_operand_bytes(R, K, S, false); };
    // digit-plane slots and exponents are scratch between steps: time on zeros
    CTM_CUDA(cudaMemsetAsync(h->ozBig, 0, std::max(opA(N, N), opB(N, N)), h->st));
    CTM_CUDA(cudaMemsetAsync(h->ozSA, 0, std::max({opA(N, b), opA(b, N), opA(m, N)}), h->st));
    CTM_CUDA(cudaMemsetAsync(h->ozSB, 0, std::max({opB(N, m), opB(b, N), opB(b, b)}), h->st));
    CTM_CUDA(cudaMemsetAsync(h->ozeBig, 0, N * sizeof(int), h->st));
    CTM_CUDA(cudaMemsetAsync(h->ozeSA, 0, N * sizeof(int), h->st));
    CTM_CUDA(cudaMemsetAsync(h->ozeSB, 0, N * sizeof(int), h->st));
    struct Shape {
        int M, Nn, K;
        OzSlot sa, sb;
        double* D;
        int ldd;
    };
    const Shape sh[2] = {{N, b, N, OZ_BIG, OZ_SB, h->Y, N}, {m, N, N, OZ_SA, OZ_BIG, h->Pn, m}};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CTM_CUDA(cudaEventCreate(&e0));
    CTM_CUDA(cudaEventCreate(&e1));
    auto done = [&](ctm_status st) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return st;
    };
    int n = 0;
    for (const Shape& X : sh) {
        void *pa, *pb;
        int *ea, *eb;
        oz_slot(h, X.sa, &pa, &ea);
        oz_slot(h, X.sb, &pb, &eb);
        double best_ms = 1e30, def_ms = 0.0;
        int best = 0, best_sl = 1, timed = 0;
        std::vector<int> seen;
        for (int req = 0; req <= 6; ++req) {
            const int sl = req == 0 ? -1 : ctm::oz_plan_slices(X.K, req);
            if (req > 0 && sl > 1 && (size_t)sl * X.M * X.Nn > L.part_cap) continue;
            if (req > 0 && std::find(seen.begin(), seen.end(), sl) != seen.end()) continue;
            if (req > 0) seen.push_back(sl);
            auto launch = [&]() {
                return ctm::oz_gemm(h->st, S, X.M, X.Nn, X.K, pa, ea, pb, eb, X.D, X.ldd, h->tcerr, h->part,
                                    L.part_cap, req);
            };
            cudaError_t ce = launch();
            if (ce != cudaSuccess) return done(fail(CTM_ECUDA, std::string("tune: ") + cudaGetErrorString(ce)));
            cudaEventRecord(e0, h->st);
            for (int r = 0; r < reps; ++r) launch();
            cudaEventRecord(e1, h->st);
            ce = cudaEventSynchronize(e1);
            if (ce != cudaSuccess) return done(fail(CTM_ECUDA, std::string("tune: ") + cudaGetErrorString(ce)));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double per = (double)ms / reps;
            if (req == 0) def_ms = per;
            if (per < best_ms) {
                best_ms = per;
                best = req;
                best_sl = req == 0 ? 1 : sl;
            }
            ++timed;
        }
        {
            std::lock_guard<std::mutex> g(g_tc_mu);
            g_oz_plans[TcKey{S, X.M, X.Nn, X.K}] = best;
        }
        if (out && n < max_out) out[n] = ctm_tune_entry{X.M, X.Nn, X.K, 64, best_sl, def_ms, best_ms, timed};
        ++n;
    }
    int err = 0;
    CTM_CUDA(cudaMemcpyAsync(&err, h->tcerr, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CTM_CUDA(cudaStreamSynchronize(h->st));
    if (n_out) *n_out = std::min(n, max_out);
    if (err) return done(fail(CTM_ETIMEOUT, "a bounded wait of the Ozaki GEMM gave up while tuning"));
    return done(CTM_OK);
}
}  // namespace
extern "C" {

ctm_status ctm_tune(ctm_handle* h, int reps, ctm_tune_entry* out, int max_out, int* n_out) {
    if (!h) return fail(CTM_EINVAL, "handle is NULL");
    if (n_out) *n_out = 0;
    const Layout& L = h->lay;
    if (reps <= 0) reps = 5;
    if (is_oz(h)) return tune_oz(h, reps, out, max_out, n_out);
    if (!L.esz) return CTM_OK;  // the FP64 form has no tensor-core launch shapes
    const bool bf16 = L.esz == 2;
    struct Shape {
        int M, N, K;
        const void *A, *B;
        int lda, ldb;
        double* D;
        int ldd;
    };
    // the three products of a step: X1 = P^t Omega P (and X1' = P^t U'),
    // C~ V, and P_new = U^t X
    const Shape sh[3] = {{L.N, L.N, L.m, h->opP, h->opPw, L.ldm, L.ldm, h->C, L.N},
                         {L.N, L.b, L.N, h->opC, h->opV, L.ldN, L.ldN, h->Y, L.N},
                         {L.m, L.N, L.N, h->opU, h->opC, L.ldN, L.ldN, h->Pn, L.m}};
    // operand copies, C, Y and Pn are scratch between steps; time on zeros
    const size_t e = L.esz;
    CTM_CUDA(cudaMemsetAsync(h->opP, 0, (size_t)L.N * L.ldm * e, h->st));
    CTM_CUDA(cudaMemsetAsync(h->opPw, 0, (size_t)L.N * L.ldm * e, h->st));
    CTM_CUDA(cudaMemsetAsync(h->opC, 0, (size_t)L.N * L.ldN * e, h->st));
    CTM_CUDA(cudaMemsetAsync(h->opV, 0, (size_t)L.b * L.ldN * e, h->st));
    CTM_CUDA(cudaMemsetAsync(h->opU, 0, (size_t)L.m * L.ldN * e, h->st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CTM_CUDA(cudaEventCreate(&e0));
    CTM_CUDA(cudaEventCreate(&e1));
    auto done = [&](ctm_status st) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return st;
    };
    int n = 0;
    for (const Shape& S : sh) {
        std::vector<ctm::TcPlan> cand{ctm::tc_default_plan(S.M, S.N, S.K, bf16)};
        for (int bn : {64, 128, 256})
            for (int sp : {1, 2, 3, 4, 6, 8}) cand.push_back({bn, sp});
        std::vector<std::pair<int, int>> seen;
        double best_ms = 1e30, def_ms = 0.0;
        ctm::TcPlan best = cand[0];
        int timed = 0;
        for (size_t ci = 0; ci < cand.size(); ++ci) {
            ctm::TcPlan p = cand[ci];
            const int sl = ctm::tc_plan_slices(p, S.K, bf16, nullptr);
            if (sl > 1 && (size_t)sl * S.M * S.N > L.tcpart_cap) continue;
            if (std::find(seen.begin(), seen.end(), std::make_pair(p.bn, sl)) != seen.end()) continue;
            seen.push_back({p.bn, sl});
            p.splits = sl;
            auto launch = [&]() {
                return ctm::tc_gemm(h->st, bf16, S.M, S.N, S.K, 1.0, S.A, S.lda, S.B, S.ldb, 0.0, S.D, S.ldd,
                                    h->tcerr, &p, h->tcpart, L.tcpart_cap);
            };
            cudaError_t ce = launch();  // warm-up
            if (ce != cudaSuccess) return done(fail(CTM_ECUDA, std::string("tune: ") + cudaGetErrorString(ce)));
            cudaEventRecord(e0, h->st);
            for (int r = 0; r < reps; ++r) launch();
            cudaEventRecord(e1, h->st);
            ce = cudaEventSynchronize(e1);
            if (ce != cudaSuccess) return done(fail(CTM_ECUDA, std::string("tune: ") + cudaGetErrorString(ce)));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double per = (double)ms / reps;
            if (ci == 0) def_ms = per;
            if (per < best_ms) {
                best_ms = per;
                best = p;
            }
            ++timed;
        }
        {
            std::lock_guard<std::mutex> g(g_tc_mu);
            g_tc_plans[TcKey{L.esz, S.M, S.N, S.K}] = best;
        }
        if (out && n < max_out) out[n] = ctm_tune_entry{S.M, S.N, S.K, best.bn, best.splits, def_ms, best_ms, timed};
        ++n;
    }
    int err = 0;
    CTM_CUDA(cudaMemcpyAsync(&err, h->tcerr, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CTM_CUDA(cudaStreamSynchronize(h->st));
    if (n_out) *n_out = std::min(n, max_out);
    if (err) return done(fail(CTM_ETIMEOUT, "a bounded wait of the tensor-core GEMM gave up while tuning"));
    return done(CTM_OK);
}

}  // extern "C"

// ------------------------------------------------------- temperature scan
// One handle per beta (own workspace); a pool of host threads, each with its
// own non-blocking stream, takes the betas in order and steps each one until
// it converges or reaches the step cap.  The handles share nothing on the
// device, so the betas' kernels overlap on the GPU wherever one beta's
// launches leave SMs idle (the latency-bound eigensolver and the host
// round trips of the subspace iteration).
struct ctm_scan {
    int dev = 0;
    int workers = 1;
    cudaStream_t caller = nullptr;
    std::vector<double> betas;
    std::vector<ctm_handle*> hs;
    std::vector<cudaStream_t> streams;
    char* ws = nullptr;  // owned block of all workspaces (NULL if the caller gave one)
};

extern "C" {

ctm_status ctm_scan_workspace_size(const ctm_config* base, int nbeta, size_t* bytes) {
    if (!bytes) return fail(CTM_EINVAL, "bytes is NULL");
    if (nbeta < 1) return fail(CTM_EINVAL, "nbeta must be >= 1");
    size_t one = 0;
    ctm_status s = ctm_workspace_size(base, &one);
    if (s != CTM_OK) return s;
    *bytes = align256(one) * (size_t)nbeta;
    return CTM_OK;
}

void ctm_scan_destroy(ctm_scan* sc) {
    if (!sc) return;
    for (ctm_handle* h : sc->hs) ctm_destroy(h);
    for (cudaStream_t st : sc->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    if (sc->ws) cudaFree(sc->ws);
    delete sc;
}

ctm_status ctm_scan_init(ctm_scan** out, const ctm_config* base, int nbeta, const double* betas, int workers,
                         void* cuda_stream) {
    if (!out) return fail(CTM_EINVAL, "scan pointer is NULL");
    *out = nullptr;
    if (!base || !betas) return fail(CTM_EINVAL, "NULL argument");
    if (nbeta < 1 || nbeta > 4096) return fail(CTM_EINVAL, "nbeta must be in [1, 4096]");
    if (workers < 1 || workers > 64) return fail(CTM_EINVAL, "workers must be in [1, 64]");
    for (int i = 0; i < nbeta; ++i) {
        ctm_config c = *base;
        c.beta = betas[i];
        c.workspace = nullptr;
        ctm_status s = validate(&c);
        if (s != CTM_OK) return s;
    }
    size_t one = 0;
    {
        ctm_config c = *base;
        c.workspace = nullptr;
        ctm_status s = ctm_workspace_size(&c, &one);
        if (s != CTM_OK) return s;
    }
    const size_t per = align256(one);
    if (base->workspace && base->workspace_bytes < per * (size_t)nbeta)
        return fail(CTM_ENOMEM, "workspace smaller than ctm_scan_workspace_size");
    ctm_scan* sc = new (std::nothrow) ctm_scan();
    if (!sc) return fail(CTM_ENOMEM, "host allocation of the scan failed");
    sc->caller = (cudaStream_t)cuda_stream;
    sc->workers = std::min(workers, nbeta);
    sc->betas.assign(betas, betas + nbeta);
    auto bail = [&](ctm_status st, const std::string& msg) {
        ctm_scan_destroy(sc);
        return fail(st, msg);
    };
    if (cudaGetDevice(&sc->dev) != cudaSuccess) return bail(CTM_ECUDA, "cudaGetDevice failed");
    // work already queued on the caller's stream (e.g. on the workspace) first
    if (cudaStreamSynchronize(sc->caller) != cudaSuccess) return bail(CTM_ECUDA, "caller stream sync failed");
    char* ws = (char*)base->workspace;
    if (!ws) {
        if (cudaMalloc(&sc->ws, per * (size_t)nbeta) != cudaSuccess)
            return bail(CTM_ENOMEM, "cudaMalloc of the scan workspaces failed");
        ws = sc->ws;
    }
    for (int w = 0; w < sc->workers; ++w) {
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
            return bail(CTM_ECUDA, "cudaStreamCreate failed");
        sc->streams.push_back(st);
    }
    for (int i = 0; i < nbeta; ++i) {
        ctm_config c = *base;
        c.beta = betas[i];
        c.workspace = ws + per * (size_t)i;
        c.workspace_bytes = per;
        ctm_handle* h = nullptr;
        ctm_status s = ctm_init(&h, &c, sc->streams[i % sc->workers]);
        if (s != CTM_OK) {
            std::string msg = g_err;
            ctm_scan_destroy(sc);
            return fail(s, "beta[" + std::to_string(i) + "]: " + msg);
        }
        sc->hs.push_back(h);
    }
    *out = sc;
    return CTM_OK;
}

ctm_status ctm_scan_tune(ctm_scan* sc, int reps, ctm_tune_entry* out, int max_out, int* n_out) {
    if (!sc) return fail(CTM_EINVAL, "scan is NULL");
    // every handle has the same layout: one tuning serves them all
    return ctm_tune(sc->hs[0], reps, out, max_out, n_out);
}

ctm_status ctm_scan_run(ctm_scan* sc, int max_steps, int* steps_done, int* converged) {
    if (!sc) return fail(CTM_EINVAL, "scan is NULL");
    if (max_steps < 0) return fail(CTM_EINVAL, "max_steps < 0");
    const int nb = (int)sc->hs.size();
    std::vector<int> done(nb, 0);
    std::vector<ctm_status> stat(nb, CTM_OK);
    std::vector<std::string> msg(nb);
    std::atomic<int> next{0};
    std::atomic<int> dev_fail{0};
    int caller_dev = 0;
    cudaGetDevice(&caller_dev);
    auto worker = [&](int w) {
        if (cudaSetDevice(sc->dev) != cudaSuccess) {
            // no beta is taken by this worker; the others finish the queue
            dev_fail.store(1);
            return;
        }
        for (;;) {
            const int i = next.fetch_add(1);
            if (i >= nb) break;
            ctm_handle* h = sc->hs[i];
            if (h->last.converged || max_steps == 0) continue;
            h->st = sc->streams[w];  // the previous owner synchronised its stream
            int d = 0;
            stat[i] = ctm_step(h, max_steps, &d, nullptr);
            done[i] = d;
            if (stat[i] != CTM_OK) msg[i] = g_err;
        }
    };
    // a thread that cannot be created leaves its share to the others
    std::vector<std::thread> pool;
    for (int w = 1; w < sc->workers; ++w) {
        try {
            pool.emplace_back(worker, w);
        } catch (...) {
            break;
        }
    }
    worker(0);
    for (auto& t : pool) t.join();
    cudaSetDevice(caller_dev);
    if (dev_fail.load() && next.load() < nb) return fail(CTM_ECUDA, "no worker could select the scan's device");
    ctm_status worst = CTM_OK;
    int worst_i = -1;
    for (int i = 0; i < nb; ++i) {
        if (steps_done) steps_done[i] = done[i];
        if (converged) converged[i] = sc->hs[i]->last.converged;
        if (stat[i] == CTM_OK) continue;
        const bool hard = stat[i] != CTM_ENOTCONVERGED;
        if (worst_i < 0 || (hard && worst == CTM_ENOTCONVERGED)) {
            worst = stat[i];
            worst_i = i;
        }
    }
    if (worst_i >= 0) return fail(worst, "beta[" + std::to_string(worst_i) + "]: " + msg[worst_i]);
    return CTM_OK;
}

ctm_status ctm_scan_observables(ctm_scan* sc, ctm_obs* out) {
    if (!sc || !out) return fail(CTM_EINVAL, "NULL argument");
    const int nb = (int)sc->hs.size();
    std::vector<ctm_status> stat(nb, CTM_OK);
    std::vector<std::string> msg(nb);
    std::atomic<int> next{0};
    int caller_dev = 0;
    cudaGetDevice(&caller_dev);
    auto worker = [&](int w) {
        if (cudaSetDevice(sc->dev) != cudaSuccess) return;
        for (;;) {
            const int i = next.fetch_add(1);
            if (i >= nb) break;
            sc->hs[i]->st = sc->streams[w];
            stat[i] = ctm_observables(sc->hs[i], &out[i]);
            if (stat[i] != CTM_OK) msg[i] = g_err;
        }
    };
    // a thread that cannot be created leaves its share to the others
    std::vector<std::thread> pool;
    for (int w = 1; w < sc->workers; ++w) {
        try {
            pool.emplace_back(worker, w);
        } catch (...) {
            break;
        }
    }
    worker(0);
    for (auto& t : pool) t.join();
    cudaSetDevice(caller_dev);
    if (next.load() < nb) return fail(CTM_ECUDA, "no worker could select the scan's device");
    for (int i = 0; i < nb; ++i)
        if (stat[i] != CTM_OK && stat[i] != CTM_ENOTCONVERGED)
            return fail(stat[i], "beta[" + std::to_string(i) + "]: " + msg[i]);
    for (int i = 0; i < nb; ++i)
        if (stat[i] != CTM_OK) return fail(stat[i], "beta[" + std::to_string(i) + "]: " + msg[i]);
    return CTM_OK;
}

ctm_status ctm_scan_handle(ctm_scan* sc, int ibeta, ctm_handle** h) {
    if (!sc || !h) return fail(CTM_EINVAL, "NULL argument");
    if (ibeta < 0 || ibeta >= (int)sc->hs.size()) return fail(CTM_EINVAL, "ibeta out of range");
    *h = sc->hs[ibeta];
    return CTM_OK;
}

ctm_status ctm_scan_get_spectrum(ctm_scan* sc, int ibeta, double* omega) {
    ctm_handle* h = nullptr;
    ctm_status s = ctm_scan_handle(sc, ibeta, &h);
    if (s != CTM_OK) return s;
    return ctm_get_spectrum(h, omega);
}

}  // extern "C"

// ================================================================ no-allocation variant
// ctm_symeig_noalloc: the same Jacobi solver as ctm_symeig for callers that
// cannot allocate device memory themselves -- for example code running inside
// a memory pool that must not grow, or a host process that only receives
// device pointers from another framework and has no allocator of its own.
// Its scratch is a file-scope device array (every GPU that loads this library
// reserves it until the process exits), so nothing is allocated per call.
namespace {
constexpr int kNoAllocMaxN = CTM_SYMEIG_NOALLOC_MAX_N;
constexpr size_t kNoAllocPad = (size_t)kNoAllocMaxN + (kNoAllocMaxN & 1);
// Upper bound of symeig_layout(kNoAllocMaxN).total (every piece rounded up to
// 256 bytes); checked against the layout at every call.
constexpr size_t kNoAllocBytes = 3 * ((kNoAllocPad * kNoAllocPad * sizeof(double) + 255) / 256 * 256) +
                                 (kNoAllocPad * sizeof(double) + 255) / 256 * 256 +
                                 (kNoAllocPad * sizeof(int) + 255) / 256 * 256 +
                                 (sizeof(ctm::DevCtl) + 255) / 256 * 256;
__device__ __align__(256) unsigned char g_symeig_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};
}  // namespace

extern "C" ctm_status ctm_symeig_noalloc(int n, const double* A, int lda, double* evals, double* vecs, int ldv,
                                         int max_sweeps, void* cuda_stream) {
    if (n < 1 || n > kNoAllocMaxN)
        return fail(CTM_EINVAL, "ctm_symeig_noalloc: n must be in [1, CTM_SYMEIG_NOALLOC_MAX_N = " +
                                    std::to_string(kNoAllocMaxN) + "]");
    if (!A || !evals || !vecs) return fail(CTM_EINVAL, "NULL argument");
    if (lda < n || ldv < n) return fail(CTM_EINVAL, "leading dimension smaller than n");
    if (max_sweeps <= 0) max_sweeps = 40;
    int dev = 0;
    CTM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(CTM_EINVAL, "device index out of range");
    void* base = nullptr;
    {
        // One-time set-up per device (with that device current): the host-side
        // name of the array is not a device address, so ask the runtime for it.
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_symeig_scratch);
            if (e != cudaSuccess)
                return fail(CTM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_scratch_ptr[dev] = p;
        }
        base = g_scratch_ptr[dev];
    }
    // The scratch is carved exactly as the workspace of ctm_symeig is.
    const SymeigLayout L = symeig_layout(n);
    if (L.total > kNoAllocBytes || symeig_layout(kNoAllocMaxN).total > kNoAllocBytes)
        return fail(CTM_EINVAL, "ctm_symeig_noalloc: scratch layout exceeds its array");
    char* ws = (char*)base;
    ctm::EigWork w{};
    w.A0 = (double*)(ws + L.A0);
    w.A1 = (double*)(ws + L.A1);
    w.S = (double*)(ws + L.S);
    w.diag = (double*)(ws + L.diag);
    w.rank = (int*)(ws + L.rank);
    ctm::DevCtl* ctl = (ctm::DevCtl*)(ws + L.ctl);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // The array keeps the previous call's contents: the control block (barrier
    // words, counters, status) must start at zero.
    CTM_CUDA(cudaMemsetAsync(ctl, 0, sizeof(ctm::DevCtl), st));
    CTM_CUDA(ctm::jacobi_f64(st, n, A, lda, w, evals, vecs, ldv, max_sweeps, ctl));
    int jst = 0;
    CTM_CUDA(cudaMemcpyAsync(&jst, &ctl->jac_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CTM_CUDA(cudaStreamSynchronize(st));
    if (jst == 2) return fail(CTM_ETIMEOUT, "a device-side barrier of the Jacobi solver gave up");
    if (jst == 1) return fail(CTM_ENOTCONVERGED, "Jacobi reached its sweep cap");
    return CTM_OK;
}
