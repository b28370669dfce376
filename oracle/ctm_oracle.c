/*
 * ctm_oracle.c -- plain FP64 CPU oracle for the CTMRG of arXiv:2004.08669.
 *
 * TEST INFRASTRUCTURE ONLY (see ctm_oracle.h).  Plain loops, OpenMP over
 * host cores, no blocking or fusion beyond what Algorithm 3 states.  The
 * readings R1-R6 taken where the paper is silent or inconsistent are listed
 * in ctm_oracle.h.
 */
#include "ctm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static double dot3(const double* a, const double* b, int dim) {
    double s = 0.0;
    for (int k = 0; k < dim; ++k) s += a[k] * b[k];
    return s;
}

/* Eq. (1): E = h(s,sig) + h(sig,s') + h(s',sig') + h(sig',s), h = -v.v'.
 * Eq. (2): W = exp(-E/T) = exp(beta * sum of the four dot products).
 * Reading R1: the matrix element w[(a + q b), (c + q d)] carries the
 * plaquette whose corners in cyclic order are a, b, d, c. */
static double plaquette_weight(int q, int dim, const double* v, double beta,
                               int a, int b, int c, int d) {
    (void)q;
    double e = dot3(v + a * dim, v + b * dim, dim) + dot3(v + b * dim, v + d * dim, dim) +
               dot3(v + d * dim, v + c * dim, dim) + dot3(v + c * dim, v + a * dim, dim);
    return exp(beta * e);
}

void or_weight_matrix(int q, int dim, const double* spins, double beta, double* w) {
    int q2 = q * q;
    for (int d = 0; d < q; ++d)
        for (int c = 0; c < q; ++c)
            for (int b = 0; b < q; ++b)
                for (int a = 0; a < q; ++a)
                    w[(a + q * b) + (size_t)q2 * (c + q * d)] =
                        plaquette_weight(q, dim, spins, beta, a, b, c, d);
}

void or_weight_matrix_bond(int q, int dim, const double* spins, double beta, double* w) {
    int q2 = q * q;
    for (int d = 0; d < q; ++d)
        for (int c = 0; c < q; ++c)
            for (int b = 0; b < q; ++b)
                for (int a = 0; a < q; ++a) {
                    double h = -dot3(spins + a * dim, spins + b * dim, dim);
                    w[(a + q * b) + (size_t)q2 * (c + q * d)] =
                        h * plaquette_weight(q, dim, spins, beta, a, b, c, d);
                }
}

/* Algorithm 1 (P-Index). */
void or_pindex(const double* A, int a, int b, int c, int d, double* B) {
    size_t ldA = (size_t)a * b, ldB = (size_t)a * c;
    for (int s = 0; s < d; ++s)
        for (int r = 0; r < c; ++r)
            for (int qq = 0; qq < b; ++qq)
                for (int p = 0; p < a; ++p)
                    B[(p + (size_t)a * r) + ldB * (qq + (size_t)b * s)] =
                        A[(p + (size_t)a * qq) + ldA * (r + (size_t)c * s)];
}

/* Algorithm 2 (P-Index2). */
void or_pindex2(const double* A, int a, int b, int c, double* B) {
    size_t ldA = (size_t)a * b;
    for (int qq = 0; qq < b; ++qq)
        for (int r = 0; r < c; ++r)
            for (int p = 0; p < a; ++p)
                B[p + (size_t)a * (r + (size_t)c * qq)] = A[(p + (size_t)a * qq) + ldA * r];
}

/* C = A^t B with A (k x n1), B (k x n2), C (n1 x n2), all column-major. */
static void gemm_tn(int n1, int n2, int k, const double* A, const double* B, double* C) {
#pragma omp parallel for schedule(static)
    for (int j = 0; j < n2; ++j) {
        const double* bj = B + (size_t)k * j;
        for (int i = 0; i < n1; ++i) {
            const double* ai = A + (size_t)k * i;
            double s = 0.0;
            for (int l = 0; l < k; ++l) s += ai[l] * bj[l];
            C[i + (size_t)n1 * j] = s;
        }
    }
}

/* C = A B with A (n1 x k), B (k x n2), C (n1 x n2), all column-major. */
static void gemm_nn(int n1, int n2, int k, const double* A, const double* B, double* C) {
#pragma omp parallel for schedule(static)
    for (int j = 0; j < n2; ++j) {
        double* cj = C + (size_t)n1 * j;
        for (int i = 0; i < n1; ++i) cj[i] = 0.0;
        for (int l = 0; l < k; ++l) {
            double blj = B[l + (size_t)k * j];
            if (blj == 0.0) continue;
            const double* al = A + (size_t)n1 * l;
            for (int i = 0; i < n1; ++i) cj[i] += al[i] * blj;
        }
    }
}

/* Sub-CTMRG(P, P', W) of Algorithm 3, step by step. */
void or_sub_ctmrg(int m, int q, const double* P, const double* Pp, const double* w,
                  double* out) {
    int N = m * q;
    size_t NN = (size_t)N * N;
    double* X1 = (double*)malloc(NN * sizeof(double));
    double* X2 = (double*)malloc(NN * sizeof(double));
    gemm_tn(N, N, m, P, Pp, X1);              /* X1 := P^t P'            */
    or_pindex(X1, m, q, m, q, X2);            /* X2 := P-Index(X1,m,q,m,q) */
    gemm_nn(m * m, q * q, q * q, X2, w, X1);  /* X3 := X2 W  (kept in X1) */
    or_pindex(X1, m, m, q, q, out);           /* P-Index(X3,m,m,q,q)      */
    free(X1);
    free(X2);
}

/* One entry of C~ = Sub-CTMRG(P, Omega P, W) at a time, straight from the
 * composition of Algorithm 3: row gamma + m s', column gamma' + m sigma',
 *   C~ = sum_{s,sigma} X1[(gamma,s),(gamma',sigma)] w[(s + q sigma), (s' + q sigma')],
 *   X1[(gamma,s),(gamma',sigma)] = sum_alpha P[alpha,(gamma,s)] omega_alpha P[alpha,(gamma',sigma)]. */
void or_ctilde_entries(int m, int q, const double* P, const double* omega, const double* w,
                       int count, const int* rows, const int* cols, double* out) {
    size_t q2 = (size_t)q * q;
#pragma omp parallel for schedule(static)
    for (int e = 0; e < count; ++e) {
        int g = rows[e] % m, sp = rows[e] / m;
        int gp = cols[e] % m, sgp = cols[e] / m;
        double acc = 0.0;
        for (int sg = 0; sg < q; ++sg)
            for (int s = 0; s < q; ++s) {
                double x1 = 0.0;
                for (int a = 0; a < m; ++a)
                    x1 += P[a + (size_t)m * (g + (size_t)m * s)] * omega[a] *
                          P[a + (size_t)m * (gp + (size_t)m * sg)];
                acc += x1 * w[(s + (size_t)q * sg) + q2 * (sp + (size_t)q * sgp)];
            }
        out[e] = acc;
    }
}

/* ---------------------------------------------------------------------
 * Dense symmetric eigensolver.
 * Householder reduction to tridiagonal form and the implicit symmetric QR
 * step with Wilkinson shift, as in Golub & Van Loan, "Matrix Computations",
 * sections 8.3.1 (tridiagonalisation) and 8.3.3 (implicit QR), written out
 * here from those descriptions.
 * ------------------------------------------------------------------- */

/* Givens pair with c*a - s*b = r and s*a + c*b = 0. */
static void givens(double a, double b, double* c, double* s) {
    if (b == 0.0) {
        *c = 1.0;
        *s = 0.0;
    } else if (fabs(b) > fabs(a)) {
        double t = -a / b;
        *s = 1.0 / sqrt(1.0 + t * t);
        *c = (*s) * t;
    } else {
        double t = -b / a;
        *c = 1.0 / sqrt(1.0 + t * t);
        *s = (*c) * t;
    }
}

int or_eigh(int n, double* A, double* evals, double* Z) {
    if (n <= 0) return 0;
    double* d = (double*)calloc((size_t)n, sizeof(double));
    double* e = (double*)calloc((size_t)n, sizeof(double));
    double* tau = (double*)calloc((size_t)n, sizeof(double));
    double* p = (double*)calloc((size_t)n, sizeof(double));
    double* wv = (double*)calloc((size_t)n, sizeof(double));
    const size_t ld = (size_t)n;

    /* --- tridiagonalisation: A <- H_k A H_k, H_k = I - tau_k v v^t,
     *     v stored in A[k+1:, k] with v[0] = 1 implicit scaling kept explicit. */
    for (int k = 0; k + 2 < n; ++k) {
        double* x = A + (k + 1) + ld * k; /* column k below the diagonal */
        int len = n - k - 1;
        double sig = 0.0;
        for (int i = 1; i < len; ++i) sig += x[i] * x[i];
        if (sig == 0.0) {
            tau[k] = 0.0;
            e[k] = x[0];
            continue;
        }
        double nx = sqrt(x[0] * x[0] + sig);
        double alpha = (x[0] >= 0.0) ? -nx : nx;
        x[0] -= alpha; /* v = x - alpha e1 */
        double vtv = x[0] * x[0] + sig;
        double t = 2.0 / vtv;
        tau[k] = t;
        e[k] = alpha;
        /* p = t * A22 v  (A22 symmetric, full storage) */
        double* A22 = A + (k + 1) + ld * (k + 1);
#pragma omp parallel for schedule(static)
        for (int i = 0; i < len; ++i) {
            double s = 0.0;
            const double* col = A22 + ld * i; /* row i of A22 = column i */
            for (int j = 0; j < len; ++j) s += col[j] * x[j];
            p[i] = t * s;
        }
        double K = 0.0;
        for (int i = 0; i < len; ++i) K += p[i] * x[i];
        K *= 0.5 * t;
        for (int i = 0; i < len; ++i) wv[i] = p[i] - K * x[i];
        /* A22 <- A22 - v w^t - w v^t */
#pragma omp parallel for schedule(static)
        for (int j = 0; j < len; ++j) {
            double vj = x[j], wj = wv[j];
            double* col = A22 + ld * j;
            for (int i = 0; i < len; ++i) col[i] -= x[i] * wj + wv[i] * vj;
        }
    }
    for (int k = 0; k < n; ++k) d[k] = A[k + ld * k];
    if (n >= 2) e[n - 2] = A[(n - 1) + ld * (n - 2)];

    /* --- accumulate Q = H_0 H_1 ... H_{n-3} into Z, innermost first. */
    for (size_t i = 0; i < ld * ld; ++i) Z[i] = 0.0;
    for (int i = 0; i < n; ++i) Z[i + ld * i] = 1.0;
    for (int k = n - 3; k >= 0; --k) {
        if (tau[k] == 0.0) continue;
        const double* v = A + (k + 1) + ld * k;
        int len = n - k - 1;
        double t = tau[k];
#pragma omp parallel for schedule(static)
        for (int j = k + 1; j < n; ++j) {
            double* col = Z + (k + 1) + ld * j;
            double s = 0.0;
            for (int i = 0; i < len; ++i) s += v[i] * col[i];
            s *= t;
            for (int i = 0; i < len; ++i) col[i] -= s * v[i];
        }
    }

    /* --- implicit symmetric QR with Wilkinson shift on (d, e).  The
     *     rotations act on columns k, k+1 of Z; Z is held transposed (row i
     *     of Z contiguous) while they are applied, so that each row is
     *     streamed once per sweep. */
    double* Zt = (double*)malloc(ld * ld * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) Zt[k + ld * i] = Z[i + ld * k];
    double* cs = (double*)malloc(2 * (size_t)n * sizeof(double));
    int hi = n - 1;
    long iter = 0, maxiter = 60L * n + 60;
    int status = 0;
    const double eps = 2.220446049250313e-16;
    while (hi > 0) {
        /* deflate from the bottom */
        if (fabs(e[hi - 1]) <= eps * (fabs(d[hi - 1]) + fabs(d[hi]))) {
            e[hi - 1] = 0.0;
            --hi;
            continue;
        }
        /* find start of the unreduced block ending at hi */
        int lo = hi - 1;
        while (lo > 0 && fabs(e[lo - 1]) > eps * (fabs(d[lo - 1]) + fabs(d[lo]))) --lo;
        if (lo > 0) e[lo - 1] = 0.0;
        if (++iter > maxiter) {
            status = -1;
            break;
        }
        /* Wilkinson shift from the trailing 2x2 block */
        double dl = 0.5 * (d[hi - 1] - d[hi]);
        double b2 = e[hi - 1] * e[hi - 1];
        double sg = (dl >= 0.0) ? 1.0 : -1.0;
        double mu = d[hi] - b2 / (dl + sg * sqrt(dl * dl + b2));
        double x = d[lo] - mu, z = e[lo];
        int nrot = 0;
        for (int k = lo; k < hi; ++k) {
            double c, s;
            givens(x, z, &c, &s);
            if (k > lo) e[k - 1] = c * x - s * z;
            double a = d[k], b = e[k], cc = d[k + 1];
            d[k] = c * c * a - 2.0 * c * s * b + s * s * cc;
            e[k] = c * s * (a - cc) + (c * c - s * s) * b;
            d[k + 1] = s * s * a + 2.0 * c * s * b + c * c * cc;
            if (k + 1 < hi) {
                x = e[k];
                z = -s * e[k + 1];
                e[k + 1] = c * e[k + 1];
            }
            cs[2 * nrot] = c;
            cs[2 * nrot + 1] = s;
            ++nrot;
        }
        /* Z <- Z G_lo ... G_{hi-1}; rows are independent. */
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; ++i) {
            double* zr = Zt + ld * i;
            for (int r = 0; r < nrot; ++r) {
                int k = lo + r;
                double c = cs[2 * r], s = cs[2 * r + 1];
                double zk = zr[k], zk1 = zr[k + 1];
                zr[k] = c * zk - s * zk1;
                zr[k + 1] = s * zk + c * zk1;
            }
        }
    }
    free(cs);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < n; ++k)
        for (int i = 0; i < n; ++i) Z[i + ld * k] = Zt[k + ld * i];
    free(Zt);

    /* --- sort by |eigenvalue| descending (stable in the original order). */
    int* ord = (int*)malloc((size_t)n * sizeof(int));
    for (int i = 0; i < n; ++i) ord[i] = i;
    for (int i = 1; i < n; ++i) { /* insertion sort: plain and stable */
        int oi = ord[i];
        int j = i - 1;
        while (j >= 0 && fabs(d[ord[j]]) < fabs(d[oi])) {
            ord[j + 1] = ord[j];
            --j;
        }
        ord[j + 1] = oi;
    }
    double* Zs = (double*)malloc(ld * ld * sizeof(double));
    for (int i = 0; i < n; ++i) {
        evals[i] = d[ord[i]];
        memcpy(Zs + ld * i, Z + ld * ord[i], ld * sizeof(double));
    }
    memcpy(Z, Zs, ld * ld * sizeof(double));
    free(Zs);
    free(ord);
    free(d);
    free(e);
    free(tau);
    free(p);
    free(wv);
    return status;
}

/* ---------------------------------------------------------------------
 * Symmetric-CTMRG (Algorithm 3).
 * ------------------------------------------------------------------- */
struct or_state {
    int q, dim, m, N, bspin;
    double beta, tol_cluster, tol_zero;
    double* spins;
    double* w;     /* q^2 x q^2 */
    double* wh;    /* bond-impurity weight */
    double* P;     /* m x N */
    double* omega; /* N: kept normalised eigenvalues, zero beyond m_eff */
    int live;      /* D: rows of P that may be non-zero */
    double* prev_ratio;
    int have_prev;
    double S_prev;
    double last_kappa;
    double last_kappa_prev;
    int steps;
};

or_state* or_create(int q, int dim, const double* spins, int m, double beta,
                    int boundary_spin, double tol_cluster, double tol_zero) {
    if (q < 2 || m < 1 || dim < 1 || boundary_spin < 0 || boundary_spin >= q) return NULL;
    or_state* s = (or_state*)calloc(1, sizeof(or_state));
    s->q = q;
    s->dim = dim;
    s->m = m;
    s->N = m * q;
    s->bspin = boundary_spin;
    s->beta = beta;
    s->tol_cluster = tol_cluster;
    s->tol_zero = tol_zero;
    s->spins = (double*)malloc((size_t)q * dim * sizeof(double));
    memcpy(s->spins, spins, (size_t)q * dim * sizeof(double));
    size_t q4 = (size_t)q * q * q * q;
    s->w = (double*)malloc(q4 * sizeof(double));
    s->wh = (double*)malloc(q4 * sizeof(double));
    or_weight_matrix(q, dim, spins, beta, s->w);
    or_weight_matrix_bond(q, dim, spins, beta, s->wh);
    s->P = (double*)calloc((size_t)m * s->N, sizeof(double));
    s->omega = (double*)calloc((size_t)s->N, sizeof(double));
    s->prev_ratio = (double*)calloc((size_t)m, sizeof(double));
    /* initialisation of Algorithm 3: p = 1 at alpha = 1, (gamma=1, s=boundary);
     * omega = 1 at the first entry; fixed boundary spin (Sec. II). */
    s->P[0 + (size_t)m * (0 + (size_t)m * boundary_spin)] = 1.0;
    s->omega[0] = 1.0;
    s->live = 1;
    s->S_prev = 0.0;
    s->last_kappa = 0.0;
    return s;
}

void or_destroy(or_state* s) {
    if (!s) return;
    free(s->spins);
    free(s->w);
    free(s->wh);
    free(s->P);
    free(s->omega);
    free(s->prev_ratio);
    free(s);
}

int or_steps_done(const or_state* s) { return s->steps; }

void or_get_state(const or_state* s, double* P, double* omega, int* live) {
    if (P) memcpy(P, s->P, (size_t)s->m * s->N * sizeof(double));
    if (omega) memcpy(omega, s->omega, (size_t)s->N * sizeof(double));
    if (live) *live = s->live;
}

void or_set_weights(or_state* s, const double* w, const double* wh) {
    size_t q4 = (size_t)s->q * s->q * s->q * s->q;
    if (w) memcpy(s->w, w, q4 * sizeof(double));
    if (wh) memcpy(s->wh, wh, q4 * sizeof(double));
}

void or_set_state(or_state* s, const double* P, const double* omega, int live) {
    memcpy(s->P, P, (size_t)s->m * s->N * sizeof(double));
    memcpy(s->omega, omega, (size_t)s->N * sizeof(double));
    s->live = live;
    s->have_prev = 0;
}

/* P' := {omega_alpha p_alpha beta} (Algorithm 3). */
static void scaled_P(const or_state* s, double* Pp) {
    int m = s->m, N = s->N;
    for (int j = 0; j < N; ++j)
        for (int a = 0; a < m; ++a) Pp[a + (size_t)m * j] = s->omega[a] * s->P[a + (size_t)m * j];
}

void or_extend(or_state* s, double* out) {
    double* Pp = (double*)malloc((size_t)s->m * s->N * sizeof(double));
    scaled_P(s, Pp);
    or_sub_ctmrg(s->m, s->q, s->P, Pp, s->w, out);
    free(Pp);
}

/* Live row indices (gamma < live, any s) of C~ in the paper's combined
 * index gamma + m s. */
static int live_indices(const or_state* s, int* idx) {
    int L = 0;
    for (int sp = 0; sp < s->q; ++sp)
        for (int g = 0; g < s->live; ++g) idx[L++] = g + s->m * sp;
    return L;
}

/* Reading R4: number of kept states. */
static int kept_count(const double* ev, int L, int m, double tol_c, double tol_z) {
    if (L == 0) return 0;
    double a1 = fabs(ev[0]);
    int meff = (m < L) ? m : L;
    while (meff > 0 && meff < L && fabs(fabs(ev[meff - 1]) - fabs(ev[meff])) <= tol_c * a1) --meff;
    while (meff > 0 && fabs(ev[meff - 1]) <= tol_z * a1) --meff;
    return meff;
}

/* Entanglement entropy of Eq. (6): S = -sum_i p_i ln p_i with the weights
 * p_i = |ev_i|^power / sum_j |ev_j|^power of the density matrix.  The method
 * takes power = 4 (rho~ = C~^4 / Tr C~^4, Eq. 4); the power is a parameter only
 * so that a test can show that another power fails the exact pin. */
double or_entropy(const double* ev, int n, int power) {
    double z = 0.0;
    for (int i = 0; i < n; ++i) z += pow(fabs(ev[i]), power);
    double S = 0.0;
    for (int i = 0; i < n; ++i) {
        double p = pow(fabs(ev[i]), power) / z;
        if (p > 0.0) S -= p * log(p);
    }
    return S;
}

static double entropy4(const double* ev, int n) { return or_entropy(ev, n, 4); }

/* Diagonalise the live block of C (N x N).  Returns L; fills ev (L) and
 * Z (L x L) and idx (L). */
static int live_eig(or_state* s, const double* C, int* idx, double* ev, double* Z, int* status) {
    int N = s->N;
    int L = live_indices(s, idx);
    double* A = (double*)malloc((size_t)L * L * sizeof(double));
    for (int j = 0; j < L; ++j)
        for (int i = 0; i < L; ++i) A[i + (size_t)L * j] = C[idx[i] + (size_t)N * idx[j]];
    *status = or_eigh(L, A, ev, Z);
    free(A);
    return L;
}

int or_step(or_state* s, double* info) {
    int m = s->m, q = s->q, N = s->N;
    size_t NN = (size_t)N * N;
    double* C = (double*)malloc(NN * sizeof(double));
    or_extend(s, C); /* C := Sub-CTMRG(P, P', W) */

    int* idx = (int*)malloc((size_t)N * sizeof(int));
    double* ev = (double*)malloc((size_t)N * sizeof(double));
    double* Z = (double*)malloc(NN * sizeof(double));
    int st = 0;
    int L = live_eig(s, C, idx, ev, Z, &st); /* diagonalisation */
    free(C);
    if (st != 0) {
        free(idx);
        free(ev);
        free(Z);
        return -1;
    }
    int meff = kept_count(ev, L, m, s->tol_cluster, s->tol_zero);

    /* U: N x m, kept eigenvectors scattered back to the combined index. */
    double* U = (double*)calloc((size_t)N * m, sizeof(double));
    for (int a = 0; a < meff; ++a)
        for (int t = 0; t < L; ++t) U[idx[t] + (size_t)N * a] = Z[t + (size_t)L * a];

    double* Up = (double*)malloc((size_t)m * N * sizeof(double));
    or_pindex2(U, m, q, m, Up);                  /* U' := P-Index2(U, m, q, m) */
    double* X = (double*)malloc(NN * sizeof(double));
    or_sub_ctmrg(m, q, s->P, Up, s->w, X);       /* X := Sub-CTMRG(P, U', W)   */
    gemm_tn(m, N, N, U, X, s->P);                /* P := U^t X                 */
    double nrm = 0.0;
    for (size_t i = 0; i < (size_t)m * N; ++i) nrm += s->P[i] * s->P[i];
    nrm = sqrt(nrm);
    for (size_t i = 0; i < (size_t)m * N; ++i) s->P[i] /= nrm; /* reading R5 */
    s->last_kappa = nrm;

    /* Omega normalisation and S_E (Algorithm 3), paper's full live spectrum
     * and the kept-state version. */
    double S_paper = entropy4(ev, L);
    double S_kept = entropy4(ev, meff);
    double z4 = 0.0;
    for (int i = 0; i < meff; ++i) z4 += pow(ev[i], 4);
    double sc = pow(z4, -0.25);
    for (int i = 0; i < N; ++i) s->omega[i] = (i < meff) ? ev[i] * sc : 0.0;

    /* Reading R6: spectrum change. */
    double delta = 0.0;
    double a1 = fabs(s->omega[0]);
    for (int i = 0; i < m; ++i) {
        double r = fabs(s->omega[i]) / a1;
        if (s->have_prev) {
            double dd = fabs(r - s->prev_ratio[i]);
            if (dd > delta) delta = dd;
        }
        s->prev_ratio[i] = r;
    }
    if (s->have_prev) {
        double dk = fabs(nrm / s->last_kappa_prev - 1.0);
        if (dk > delta) delta = dk;
    } else {
        delta = INFINITY;
    }
    s->have_prev = 1;
    s->last_kappa_prev = nrm;
    double cpaper = fabs(1.0 - S_paper / s->S_prev);
    s->S_prev = S_paper;
    s->live = meff;
    s->steps += 1;
    if (info) {
        info[0] = nrm;
        info[1] = delta;
        info[2] = S_paper;
        info[3] = S_kept;
        info[4] = meff;
        info[5] = cpaper;
        info[6] = L;
    }
    free(idx);
    free(ev);
    free(Z);
    free(U);
    free(Up);
    free(X);
    return 0;
}

int or_observables(or_state* s, double* out) {
    int m = s->m, q = s->q, N = s->N, dim = s->dim;
    size_t NN = (size_t)N * N;
    double* Pp = (double*)malloc((size_t)m * N * sizeof(double));
    scaled_P(s, Pp);
    double* C = (double*)malloc(NN * sizeof(double));
    double* Ch = (double*)malloc(NN * sizeof(double));
    or_sub_ctmrg(m, q, s->P, Pp, s->w, C);
    or_sub_ctmrg(m, q, s->P, Pp, s->wh, Ch);
    free(Pp);
    int* idx = (int*)malloc((size_t)N * sizeof(int));
    double* ev = (double*)malloc((size_t)N * sizeof(double));
    double* Z = (double*)malloc(NN * sizeof(double));
    int st = 0;
    int L = live_eig(s, C, idx, ev, Z, &st);
    if (st != 0) {
        free(C); free(Ch); free(idx); free(ev); free(Z);
        return -1;
    }
    int meff = kept_count(ev, L, m, s->tol_cluster, s->tol_zero);

    /* Eq. (5): M = Tr[(v_b . v_s) rho~], rho~ = C~^4 / Tr C~^4, s the spin
     * leg of the row index.  In the eigenbasis: sum_i p_i sum_t z_ti^2 h_t. */
    const double* vb = s->spins + (size_t)s->bspin * dim;
    double* mag = (double*)malloc((size_t)L * sizeof(double));
    for (int t = 0; t < L; ++t) {
        int sp = idx[t] / m;
        mag[t] = dot3(vb, s->spins + (size_t)sp * dim, dim);
    }
    /* Bond energy: <h> = Tr(C~_h C~^3) / Tr(C~^4) = sum_i w_i^3 z_i^t C~_h z_i / sum w^4. */
    double Mk = 0, Mf = 0, Hk = 0, Hf = 0, Zk = 0, Zf = 0;
    for (int i = 0; i < L; ++i) {
        const double* zi = Z + (size_t)L * i;
        double mi = 0.0;
        for (int t = 0; t < L; ++t) mi += zi[t] * zi[t] * mag[t];
        double hi = 0.0;
#pragma omp parallel for reduction(+ : hi) schedule(static)
        for (int u = 0; u < L; ++u) {
            double acc = 0.0;
            const double* col = Ch + (size_t)N * idx[u];
            for (int t = 0; t < L; ++t) acc += zi[t] * col[idx[t]];
            hi += acc * zi[u];
        }
        double w4 = pow(ev[i], 4), w3 = pow(ev[i], 3);
        Mf += w4 * mi;
        Hf += w3 * hi;
        Zf += w4;
        if (i < meff) {
            Mk += w4 * mi;
            Hk += w3 * hi;
            Zk += w4;
        }
    }
    out[0] = -0.5 / s->beta * log(s->last_kappa);
    out[1] = Mk / Zk;
    out[2] = Mf / Zf;
    out[3] = 2.0 * Hk / Zk;
    out[4] = 2.0 * Hf / Zf;
    out[5] = entropy4(ev, meff);
    out[6] = entropy4(ev, L);
    out[7] = s->last_kappa;
    free(mag);
    free(C);
    free(Ch);
    free(idx);
    free(ev);
    free(Z);
    return 0;
}

/* ---------------------------------------------------------------------
 * Effective correlation length (Sec. II): the renormalised row-to-row
 * transfer matrix reconstructed from P~.  A row through the centre is the
 * left half-row P, the centre vertex W and the right half-row P; its legs
 * are the upper block legs of the two halves with the centre's upper spin,
 * and the lower ones (reading R10):
 *   T[(a, t, a'), (g, u, g')] = sum_{s, s'} P[a, g + m s] W(s, t, s', u) P[a', g' + m s'],
 * with W's arguments in the cyclic corner order of Eq. (1); by reading R1,
 * W(s, t, s', u) = w[s + q t, u + q s'].  Row index a + m t + m q a'.
 * ------------------------------------------------------------------- */
void or_row_transfer(int m, int q, const double* P, const double* w, double* T) {
    const size_t n = (size_t)m * q * m;
#pragma omp parallel for schedule(static)
    for (long col = 0; col < (long)n; ++col) {
        const int g = (int)(col % m), u = (int)((col / m) % q), g2 = (int)(col / ((size_t)m * q));
        for (size_t row = 0; row < n; ++row) {
            const int a = (int)(row % m), t = (int)((row / m) % q), a2 = (int)(row / ((size_t)m * q));
            double acc = 0.0;
            for (int s = 0; s < q; ++s) {
                const double pl = P[a + (size_t)m * (g + (size_t)m * s)];
                if (pl == 0.0) continue;
                for (int s2 = 0; s2 < q; ++s2) {
                    const double W = w[(s + (size_t)q * t) + (size_t)q * q * (u + (size_t)q * s2)];
                    acc += pl * W * P[a2 + (size_t)m * (g2 + (size_t)m * s2)];
                }
            }
            T[row + n * col] = acc;
        }
    }
}

/* The k eigenvalues of T of largest modulus (sorted by |lambda| descending)
 * from a full dense diagonalisation; returns -1 if the eigensolver failed. */
int or_row_transfer_spectrum(const or_state* s, int k, double* lam) {
    const int m = s->m, q = s->q;
    const size_t n = (size_t)m * q * m;
    double* T = (double*)malloc(n * n * sizeof(double));
    double* Z = (double*)malloc(n * n * sizeof(double));
    double* ev = (double*)malloc(n * sizeof(double));
    or_row_transfer(m, q, s->P, s->w, T);
    /* symmetric by the reflection of the row (P[a, g, s] = P[g, a, s]) */
    for (size_t i = 0; i < n; ++i)
        for (size_t j = i + 1; j < n; ++j) {
            double v = 0.5 * (T[i + n * j] + T[j + n * i]);
            T[i + n * j] = T[j + n * i] = v;
        }
    int st = or_eigh((int)n, T, ev, Z);
    for (int i = 0; i < k; ++i) lam[i] = i < (int)n ? ev[i] : 0.0;
    free(T);
    free(Z);
    free(ev);
    return st;
}
