/*
 * ctm_oracle.h -- plain FP64 CPU oracle for the CTMRG of arXiv:2004.08669.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library. The GPU
 * product path never links, imports or calls it, and shares no code with it.
 *
 * Everything here follows the paper's Algorithm 3 (Symmetric-CTMRG and
 * Sub-CTMRG), Algorithm 1 (P-Index) and Algorithm 2 (P-Index2) in the
 * paper's own storage convention: matrices are column-major, combined
 * indices put the first leg fastest, so P is m x (m q) with column index
 * gamma + m*s, and the extended corner C~ is (m q) x (m q) with row index
 * gamma + m*s.  All indices here are 0-based.
 *
 * Readings of the paper that this oracle takes (each is also listed in the
 * design notes of the repository):
 *  R1  Matrix form of W (Alg. 3, initialisation of W).  The open corner leg
 *      that joins the row index of C~ must be the plaquette neighbour of the
 *      corner leg contracted with the row-side P.  With Eq. (1)'s cyclic
 *      corner order (s, sigma, s', sigma') this is
 *          w[(s + q sigma), (s' + q sigma')] = W(s, sigma, sigma', s').
 *      The literal assignment W(s, sigma, s', sigma') builds a different
 *      (twisted) network whose Ising free energy misses Onsager's by 4e-3.
 *  R2  Temperature convention (Eq. 2 and Sec. II): every bond belongs to
 *      exactly one vertex tensor, so each bond carries the full beta.
 *  R3  Diagonalisation acts on the live block of C~ (rows/columns whose
 *      gamma < D, D = live rows of P); the other rows and columns are zero.
 *  R4  Truncation keeps the m largest |w|; a multiplet (|w_i|-|w_j| within
 *      tol_cluster*|w_1|) that straddles the cut is dropped whole, and
 *      eigenvalues with |w| <= tol_zero*|w_1| are dropped. Dropped states
 *      get omega = 0 and zero rows of P.
 *  R5  P is normalised by its Frobenius norm (the paper uses max|p|); the
 *      factor kappa_k = ||P_{k+1}|| is recorded; the free energy per spin is
 *      f = -(T/2) ln kappa at the fixed point (two spins per vertex).
 *  R6  Convergence: delta_k is the larger of max_i | |w_i|/|w_1| (step k)
 *      - same (step k-1) | over i < m and |kappa_k/kappa_{k-1} - 1|; the
 *      normalised spectrum settles many steps before kappa (and so f) does.
 *      The paper's c = |1 - S_E/S| is reported too.
 *  R10 Effective correlation length (Sec. II, "row-to-row transfer matrices
 *      reconstructed from P~"): the row through the centre is the left
 *      half-row P, the centre vertex W and the right half-row P, joined at
 *      the opposite (side) corners of W; xi_e = 1 / ln|l0 / l1| of that
 *      matrix, in units of the vertex-row spacing.
 */
#ifndef CTM_ORACLE_H
#define CTM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Eq. (1)-(2) with reading R1/R2: w is q^2 x q^2, column-major.
 * spins: q x dim row-major unit vectors. */
void or_weight_matrix(int q, int dim, const double* spins, double beta, double* w);

/* Same weight with one bond energy h(s,sigma) = -v_s.v_sigma inserted as a
 * factor (impurity used for the internal energy). */
void or_weight_matrix_bond(int q, int dim, const double* spins, double beta, double* w);

/* Algorithm 1: B[p + a r, q + b s] = A[p + a q, r + c s]; A is (ab)x(cd). */
void or_pindex(const double* A, int a, int b, int c, int d, double* B);

/* Algorithm 2: B[p, r + c q] = A[p + a q, r]; A is (ab) x c. */
void or_pindex2(const double* A, int a, int b, int c, double* B);

/* Sub-CTMRG(P, P', W) of Algorithm 3: returns P-Index(P-Index(P^t P') W).
 * P, Pp: m x (m q); w: q^2 x q^2; out: (m q) x (m q). */
void or_sub_ctmrg(int m, int q, const double* P, const double* Pp,
                  const double* w, double* out);

/* Sampled entries of C~ = Sub-CTMRG(P, Omega P, W), computed one by one
 * (rows/cols in the paper's combined index gamma + m s). */
void or_ctilde_entries(int m, int q, const double* P, const double* omega, const double* w,
                       int count, const int* rows, const int* cols, double* out);

/* Dense symmetric eigensolver (Householder tridiagonalisation followed by the
 * implicit symmetric QR iteration with Wilkinson shift).  A (n x n,
 * column-major, symmetric) is destroyed.  On return evals[i] and column i of
 * Z are the i-th eigenpair, sorted by |eval| descending.  Returns 0 on
 * success, -1 if the QR iteration did not converge. */
int or_eigh(int n, double* A, double* evals, double* Z);

/* Number of OpenMP threads the oracle uses. */
int or_num_threads(void);

/* Entropy -sum p ln p of the weights p_i = |ev_i|^power / sum |ev|^power
 * (Eq. 6 with power = 4, the density matrix rho~ = C~^4 / Tr C~^4 of Eq. 4). */
double or_entropy(const double* ev, int n, int power);

typedef struct or_state or_state;

or_state* or_create(int q, int dim, const double* spins, int m, double beta,
                    int boundary_spin, double tol_cluster, double tol_zero);
void or_destroy(or_state* s);

/* One CTMRG iteration of Algorithm 3. info (may be NULL) receives
 * [kappa, delta, S_E_paper, S_E_kept, m_eff, c_paper, live_dim].
 * Returns 0, or -1 on eigensolver failure. */
int or_step(or_state* s, double* info);

/* Observables from the current state (one more extension, full eig):
 * out = [f, M_kept, M_full, u_kept, u_full, S_E_kept, S_E_full, kappa].
 * ln kappa uses the factor of the last step. */
int or_observables(or_state* s, double* out);

/* Extension only: C~ = Sub-CTMRG(P, Omega P, W) of the current state,
 * written to out ((m q) x (m q), column-major). */
void or_extend(or_state* s, double* out);

/* Accessors: P is m x (m q) column-major, omega has m q entries. */
void or_get_state(const or_state* s, double* P, double* omega, int* live);
void or_set_state(or_state* s, const double* P, const double* omega, int live);
int  or_steps_done(const or_state* s);

/* Effective correlation length (Sec. II, reading R10): the renormalised
 * row-to-row transfer matrix T built from P and the vertex weight,
 *   T[(a, t, a'), (g, u, g')] = sum_{s,s'} P[a, g + m s] W(s, t, s', u) P[a', g' + m s'],
 * (m^2 q) x (m^2 q), row index a + m t + m q a', W in the cyclic order of
 * Eq. (1) (w[s + q t, u + q s'] by reading R1).  T is symmetric. */
void or_row_transfer(int m, int q, const double* P, const double* w, double* T);

/* The k largest-modulus eigenvalues of T for the current P (full dense
 * diagonalisation, sorted by |lambda| descending; xi_e = 1 / ln|l0/l1|).
 * Returns 0, or -1 on eigensolver failure. */
int or_row_transfer_spectrum(const or_state* s, int k, double* lam);

/* Replace the weight matrices (q^2 x q^2 each, either may be NULL).  Used by
 * the tests that plant a mistake in the oracle and check that a pin fails. */
void or_set_weights(or_state* s, const double* w, const double* wh);

#ifdef __cplusplus
}
#endif
#endif
