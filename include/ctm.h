/*
 * ctm.h -- C-ABI of the GB300 CTMRG library (libctm_gb300.so).
 *
 * One handle runs the corner transfer matrix renormalisation group of
 * arXiv:2004.08669 (Algorithm 3, "Symmetric-CTMRG") for one polyhedron
 * vector-spin model at one temperature on one GPU.  Every step of the method
 * runs in the library's own CUDA kernels; the library never calls cuBLAS,
 * cuSOLVER or any CPU fallback.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Indices are 0-based.  Matrices exchanged with the caller are
 *    column-major, combined indices put the first leg fastest, exactly as in
 *    the paper's Algorithms 1-3: the half-row transfer tensor P is m x (m q)
 *    with column index gamma + m*s, and the extended corner C~ is (m q) x (m q)
 *    with row index gamma + m*s (gamma: renormalised leg, s: spin).  The
 *    device keeps its own layout internally and converts on the way in/out.
 *  - "host" pointers are ordinary CPU memory owned by the caller; the library
 *    copies from them before returning and never keeps them.  The library
 *    owns every device buffer it allocates; a caller-provided workspace
 *    (ctm_config.workspace) stays owned by the caller and must outlive the
 *    handle.
 *  - All work is issued on the caller's CUDA stream (borrowed, never
 *    destroyed).  Calls that return host data synchronise that stream.
 *  - Errors: every call returns a ctm_status; nothing throws across the ABI.
 *    ctm_last_error() returns a thread-local message for the last failure.
 *    A handle stays usable after CTM_ENOTCONVERGED (the caller may keep
 *    stepping); after CTM_ECUDA or CTM_ETIMEOUT it should be destroyed.
 *  - A handle is not thread-safe: one host thread at a time per handle.
 */
#ifndef CTM_H
#define CTM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CTM_OK = 0,
    CTM_EINVAL = 1,          /* invalid argument or configuration            */
    CTM_ENOMEM = 2,          /* device allocation or workspace too small     */
    CTM_ENOTCONVERGED = 3,   /* an iteration cap was reached (result usable) */
    CTM_ENUMERIC = 4,        /* NaN/Inf or a non-positive pivot was produced */
    CTM_ETIMEOUT = 5,        /* a bounded device-side wait gave up           */
    CTM_ECUDA = 6,           /* a CUDA runtime call failed                   */
    CTM_EUNSUPPORTED = 7     /* precision mode or feature not built          */
} ctm_status;

/* Arithmetic of the contractions (extension, C~ V products, P update).
 * The Rayleigh-Ritz eigensolve and the Cholesky factor of the CholQR2
 * re-orthonormalisation are FP64 in CTM_FP64 and double-float (an unevaluated
 * sum of two FP32 words, unit roundoff 2^-46, on the FP32 pipe) in the other
 * modes; the normalisations are FP64 in every mode. */
typedef enum {
    CTM_FP64 = 0,     /* plain FP64 on the CUDA cores                         */
    CTM_TF32 = 1,     /* tcgen05 kind::tf32, FP32 accumulate                  */
    CTM_BF16 = 2,     /* tcgen05 kind::f16 with bf16 operands, FP32 accumulate */
    CTM_OZAKI64 = 3   /* FP64 emulated by bf16 slice products on tcgen05      */
} ctm_precision;

typedef struct {
    int q;                    /* number of spin states (q >= 2)                    */
    int dim;                  /* spin-vector dimension (1..4)                       */
    const double* spins;      /* host, q x dim row-major unit vectors (Sec. I)      */
    int m;                    /* cutoff dimension (Sec. II), 1 <= m                 */
    double beta;              /* inverse temperature 1/T, finite, >= 0              */
    int boundary_spin;        /* fixed boundary spin "s = 1" of Sec. II (0-based)   */
    ctm_precision prec;
    int ozaki_slices;         /* digit planes per operand for CTM_OZAKI64 (0: 7)    */
    double tol_spectrum;      /* convergence of the step loop (default 1e-12)      */
    int max_steps;            /* cap used by ctm_run (default 5000)                 */
    int block_extra;          /* subspace width b = m + block_extra (0: default)    */
    int max_subspace_iters;   /* per step (0: default 50)                           */
    double subspace_tol;      /* Ritz residual / |w_1| (0: default 1e-13)           */
    double tol_cluster;       /* multiplet tolerance, relative to |w_1| (0: 1e-10)  */
    void* workspace;          /* optional device workspace (NULL: library allocates) */
    size_t workspace_bytes;   /* its size; see ctm_workspace_size                   */
} ctm_config;

/* Per-step diagnostics (the paper's S_E and c of Algorithm 3 plus the
 * quantities the build needs). */
typedef struct {
    double kappa;          /* Frobenius growth factor of P this step           */
    double delta;          /* convergence measure (spectrum and kappa change)  */
    double S_E;            /* entanglement entropy of the kept spectrum (Eq. 6) */
    double residual;       /* max Ritz residual / |w_1| of the kept states     */
    int m_eff;             /* states kept after the multiplet rule             */
    int live_dim;          /* live dimension of C~ this step                   */
    int subspace_iters;    /* subspace iterations used                          */
    int jacobi_sweeps;     /* sweeps of the last cooperative Jacobi solve      */
    int steps;             /* CTMRG steps done by this handle                   */
    int converged;         /* delta < tol_spectrum                              */
    long long rr_refined;  /* Rayleigh-Ritz solves by simultaneous rotations   */
    long long rr_jacobi;   /* Rayleigh-Ritz solves by the cooperative Jacobi   */
    int rr_fail_reason;    /* last refinement.  Mixed-precision forms (the
                              cluster-aware refinement): 0 ok, 1 more than 8b
                              strongly coupled pairs, 2 a cluster above 32
                              states, 3 iteration cap, 4 a non-finite value.
                              FP64 form: 0 ok, 1 coupled non-doublet pair,
                              2 large rotation, 3 iteration cap, 4 triplet  */
    int rr_last_iter;      /* its iterations                                   */
    double rr_last_max;    /* its last largest coupling (mixed forms) or
                              rotation / orthonormality defect (FP64 form)  */
    int jacobi_rotations[8]; /* rotations per sweep of the last Jacobi solve
                                (first 8 sweeps)                           */
    long long rr_fail_counts[5]; /* refinements that fell back to Jacobi, by
                                    rr_fail_reason (index 0 unused)         */
} ctm_step_info;

/* Observables of the current state (Eq. 4-6 and the free energy). */
typedef struct {
    double f;       /* free energy per spin, -(T/2) ln kappa                       */
    double M;       /* spontaneous magnetisation, Eq. (5), kept states             */
    double u;       /* internal energy per spin, 2 <h> from Tr(C~_h C~^3)/Tr C~^4 */
    double S_E;     /* entanglement entropy, Eq. (6), kept states                  */
    double delta;   /* last convergence measure                                    */
    int steps;      /* CTMRG steps done                                            */
    int converged;
} ctm_obs;

typedef struct ctm_handle ctm_handle;

/* Device bytes a handle needs for this configuration. */
ctm_status ctm_workspace_size(const ctm_config* cfg, size_t* bytes);

/* Create a handle: validates cfg, copies the spin table, builds the vertex
 * weight of Eq. (1)-(2) on the device and sets the fixed-boundary initial
 * P and Omega of Algorithm 3.  cuda_stream: a cudaStream_t (NULL = legacy
 * default stream).  Validation: q >= 2, 1 <= dim <= 4, m >= 1, beta >= 0
 * finite, spins of unit norm within 1e-12, 0 <= boundary_spin < q. */
ctm_status ctm_init(ctm_handle** h, const ctm_config* cfg, void* cuda_stream);

/* Run up to nsteps iterations of the while-loop of Algorithm 3 (extension,
 * leading eigenpairs of C~, renormalisation, normalisation, S_E and the
 * convergence test).  Stops early once converged.  *steps_done (may be
 * NULL) receives the number of steps taken; info (may be NULL) the
 * diagnostics of the last one.  Returns CTM_ENOTCONVERGED if a subspace
 * iteration hit its cap (the step is still applied). */
ctm_status ctm_step(ctm_handle* h, int nsteps, int* steps_done, ctm_step_info* info);

/* Observables of the current state: one more extension and its leading
 * eigenpairs, then Eq. (5)-(6) and the free energy. out: host. */
ctm_status ctm_observables(ctm_handle* h, ctm_obs* out);

/* One step of the forward-mode beta tangent (FP64 form; the derivative of
 * the step of Algorithm 3).  At the handle's current state (P, omega), set
 * for instance by ctm_set_state, it takes one step and its tangent along the
 * input tangent (P_dot, omega_dot) and, with source != 0, along W's own beta
 * dependence (dW/dbeta = W times the plaquette's sum of dot products):
 *   C~ = Sub-CTMRG(P, Omega P, W) and dC~ by the product rule;
 *   the kept eigenpairs' first-order perturbation: the coupling among the
 *   leading Ritz pairs that are eigenpairs to 1e-11 |theta_0| (zero inside a
 *   cluster, |theta_i - theta_j| <= tol_cluster |theta_0|), and the part
 *   outside them by the deflated iteration
 *   Y <- (R + (I - Z Z^t) C~ Y) diag(theta)^-1 to a change of 1e-14;
 *   U, U' = P-Index2(U), X = Sub-CTMRG(P, U', W), P_raw = U^t X and their
 *   tangents; kappa = ||P_raw||, P_new = P_raw / kappa; omega_new = theta
 *   (sum theta^4)^(-1/4) on the kept states; and the tangents of all three.
 * P_dot, P_new, P_dot_new: m x (m q) in the paper's layout (as
 * ctm_get_state); omega_dot, omega_new, omega_dot_new: m entries (zero past
 * m_eff); all host memory owned by the caller.  The handle's P and omega are
 * not changed; its C~ buffer, Ritz block and warm start are (the next
 * ctm_step starts its subspace iteration cold).  Allocates about 6 (m q)^2
 * doubles of device scratch for the call.  CTM_EUNSUPPORTED for the other
 * precision forms; CTM_ENOTCONVERGED if the subspace or the deflated
 * iteration does not converge. */
typedef struct {
    double* P_new;          /* out, m x m q                                  */
    double* omega_new;      /* out, m                                        */
    double* P_dot_new;      /* out, m x m q                                  */
    double* omega_dot_new;  /* out, m                                        */
    double kappa;           /* growth factor ||P_raw||                       */
    double kappa_dot;       /* its tangent                                   */
    int m_eff;              /* kept states                                   */
    int ritz_pairs;         /* Ritz pairs coupled inside the block           */
    int deflate_iterations; /* iterations of the deflated solve              */
    int subspace_iterations;
} ctm_tangent_out;
ctm_status ctm_tangent_step(ctm_handle* h, const double* P_dot, const double* omega_dot, int source,
                            ctm_tangent_out* out);

/* Derivative of the converged fixed point with respect to beta, contracted
 * with the gradient of the observables:
 *   *grad_beta = grad_obs->f df/dbeta + grad_obs->M dM/dbeta
 *              + grad_obs->u du/dbeta + grad_obs->S_E dS_E/dbeta
 * (the other fields of grad_obs are ignored), by implicit differentiation
 * of the gauge-fixed step at the current state: one more step whose Ritz
 * block is rotated onto the last step's must repeat P (entries weighted by
 * |omega| of both block legs, to 1e-8), else CTM_ENOTCONVERGED; then the
 * linear fixed-point equation (I - J) x = d(step)/dbeta, J = d(step)/d(state),
 * is solved by GMRES on the host (to 1e-12, at most 300 iterations) with J
 * applied as the tangent step of ctm_tangent_step; df/dbeta follows from
 * the growth factor's tangent (f = -ln kappa / (2 beta)), and, when their
 * gradients are nonzero, dM, du and dS_E from the kept eigenpairs' tangent
 * along the solution and the tangent of C~_h (the extension with the bond
 * energy inserted, with its own beta-derivative).  FP64 form only (else
 * CTM_EUNSUPPORTED); the state must come from ctm_step (else CTM_EINVAL).
 * The handle's P and omega are unchanged. */
ctm_status ctm_step_backward(ctm_handle* h, const ctm_obs* grad_obs, double* grad_beta);

/* Effective correlation length (Sec. II): the leading eigenvalues of the
 * renormalised row-to-row transfer matrix reconstructed from the current P
 * (the row through the centre: half-row P, centre vertex W, half-row P),
 *   T[(a, t, a'), (g, u, g')] = sum_{s,s'} P(a, g, s) W(s, t, s', u) P(a', g', s'),
 * W in the cyclic corner order of Eq. (1), of order m^2 q and symmetric.
 * T is applied implicitly (two GEMMs and a centre-vertex contraction per
 * application, all FP64) inside a Lanczos iteration with full
 * reorthogonalisation from a seeded Gaussian vector; the Ritz values of
 * its tridiagonal matrix come from the library's Jacobi solver.  It stops
 * when the residual bounds of the two leading Ritz pairs fall below
 * tol * |lambda_0| (tol <= 0: 1e-12), checked every 4 iterations, or at
 * max_iters (<= 0: 64; at most 120; at most m^2 q).  xi = 1 / ln|lambda_0 /
 * lambda_1| in units of the spacing of vertex rows (one diagonal of the
 * spin lattice).  Call it at a converged state (after ctm_step); it
 * allocates about (max_iters + 3) m^2 q doubles of scratch for the call and
 * overwrites the handle's C~ buffer (scratch between steps).  Returns
 * CTM_ENOTCONVERGED at max_iters (the result is still written). */
typedef struct {
    double lambda[4];    /* leading Ritz values, sorted by |lambda| descending */
    double residual[4];  /* their residual bounds / |lambda_0|                 */
    double xi;           /* 1 / ln|lambda_0 / lambda_1|                        */
    int iterations;      /* Lanczos iterations                                 */
    int converged;
} ctm_xi_result;
ctm_status ctm_xi(ctm_handle* h, int max_iters, double tol, ctm_xi_result* out);

/* Normalised kept spectrum Omega (host, m entries; zeros past m_eff). */
ctm_status ctm_get_spectrum(ctm_handle* h, double* omega);

/* State exchange (host buffers, paper layout).  P: m x (m q); omega: m;
 * live: rows of P that may be non-zero.  ctm_set_state also discards the
 * warm start of the subspace iteration. */
ctm_status ctm_get_state(ctm_handle* h, double* P, double* omega, int* live);
ctm_status ctm_set_state(ctm_handle* h, const double* P, const double* omega, int live);

/* Checkpoint: serialise the whole iteration state (P, Omega, warm start,
 * counters) into a host buffer.  Call with buf == NULL to get *len. */
ctm_status ctm_save(ctm_handle* h, void* buf, size_t* len);
ctm_status ctm_load(ctm_handle* h, const void* buf, size_t len);

/* Inspection for tests: compute only the extension C~ = Sub-CTMRG(P, Omega P,
 * W) of the current state, then read `count` sampled entries
 * (row[i], col[i]) in the paper's index into out (host). */
ctm_status ctm_extend(ctm_handle* h);
ctm_status ctm_get_ctilde(ctm_handle* h, const int* rows, const int* cols, int count, double* out);

/* Inspection for tests: leading eigenpairs of the C~ last built by
 * ctm_extend (subspace iteration to subspace_tol, cold or warm start).
 * evals: host, b entries; vecs: host, (m q) x b in the paper's row index,
 * or NULL.  *b_out receives b. */
ctm_status ctm_eigen(ctm_handle* h, double* evals, double* vecs, int* b_out);

/* Dense symmetric FP64 eigensolver on device memory: the cyclic Jacobi
 * solver (round-robin parallel order) that the step uses for its
 * Rayleigh-Ritz problem, exposed on its own.  A: n x n symmetric, device,
 * column-major with leading dimension lda (only read; (A + A^t)/2 is
 * diagonalised).  evals: device, n entries; vecs: device, n x n with
 * leading dimension ldv; on return column i of vecs and evals[i] are the
 * i-th eigenpair, sorted by |eigenvalue| descending (ties by index).
 * workspace: device scratch of at least ctm_symeig_workspace_size(n) bytes,
 * owned by the caller.  max_sweeps <= 0 selects 40 (cap 64).  Synchronises
 * the stream.  Returns CTM_ENOTCONVERGED if the sweep cap was reached
 * (the result is still written), CTM_ETIMEOUT if a device-side barrier
 * gave up, CTM_EINVAL for n < 1, n > 4096 or a short workspace. */
ctm_status ctm_symeig_workspace_size(int n, size_t* bytes);
ctm_status ctm_symeig(int n, const double* A, int lda, double* evals, double* vecs, int ldv, int max_sweeps,
                      void* workspace, size_t workspace_bytes, void* cuda_stream);

/* No-allocation variant of ctm_symeig.  The paper has no counterpart; this
 * exists for callers that cannot allocate device memory themselves -- code
 * running inside a fixed memory pool that must not grow, or a host program
 * that only holds device pointers handed to it by another framework.  The
 * caller still passes A, evals and vecs (device, same layout and results as
 * ctm_symeig); the solver's scratch is a file-scope device array of
 * CTM_SYMEIG_NOALLOC_MAX_N-sized buffers (about 6.3 MB), which every GPU that
 * loads this library keeps reserved until the process exits.  No call
 * allocates or frees anything.
 *  - n > CTM_SYMEIG_NOALLOC_MAX_N (or n < 1) returns CTM_EINVAL with a message.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.  The scratch is picked by the device that is
 *    current at the call: pass a stream and pointers of that device.  The
 *    address is kept for the life of the process and does not survive a
 *    cudaDeviceReset of that device (calls after a reset would use a stale
 *    address): do not reset a device between calls.
 *  - All calls share the one array and each call clears the parts that must
 *    start at zero.  Calls whose work overlaps on the GPU (concurrent streams
 *    or host threads) race on the array and give wrong results: serialise
 *    them.
 *  - Synchronises the stream; statuses as for ctm_symeig. */
#define CTM_SYMEIG_NOALLOC_MAX_N 512
ctm_status ctm_symeig_noalloc(int n, const double* A, int lda, double* evals, double* vecs, int ldv, int max_sweeps,
                              void* cuda_stream);

/* One contraction of the step's shape on device memory:
 *   D (M x N) = A^t B,  A: K x M (lda), B: K x N (ldb), D: M x N (ldd),
 * all column-major FP64 (both operands contiguous along K, as every GEMM of
 * Algorithm 3 is here).  prec selects the arithmetic:
 *   CTM_FP64     the FP64 CUDA-core kernel;
 *   CTM_TF32 /   A and B rounded to that type (nearest, ties away for TF32,
 *   CTM_BF16     ties to even for BF16), tcgen05 tensor cores, FP32 accumulation;
 *   CTM_OZAKI64  FP64 emulated on the bf16 tensor cores: every row of A and
 *                of B is split into ozaki_slices (3..7; 0 selects 6) exact
 *                7-bit digit planes; the digit products with i + j <= s + 1
 *                are accumulated exactly over K-chunks of 512 and combined in
 *                double-float; the error is below about 2^(-7s) K max|A_row|
 *                max|B_row| per element.
 * D is written in FP64.  workspace: device scratch of at least
 * ctm_contract_workspace_size(...) bytes, owned by the caller.  Synchronises
 * the stream; CTM_ETIMEOUT if a bounded device-side wait gave up. */
ctm_status ctm_contract_workspace_size(ctm_precision prec, int ozaki_slices, int M, int N, int K, size_t* bytes);
ctm_status ctm_contract(ctm_precision prec, int ozaki_slices, int M, int N, int K, const double* A, int lda,
                        const double* B, int ldb, double* D, int ldd, void* workspace, size_t workspace_bytes,
                        void* cuda_stream);

/* Profiling.  While enabled, every kernel class of the step is bracketed by
 * CUDA events on the handle's stream; ctm_profile_read synchronises the
 * stream and returns, per class, the launches, the summed device time and
 * the algorithmic FLOPs and bytes of those launches (the minimum traffic of
 * each kernel's inputs and outputs).  The last entry, "all", counts every
 * kernel the handle launched while enabled.  Reading clears the records. */
typedef struct {
    const char* name;     /* static string owned by the library */
    long long launches;
    double ms;
    double flops;
    double bytes;
} ctm_prof_entry;
ctm_status ctm_profile(ctm_handle* h, int enable);
ctm_status ctm_profile_read(ctm_handle* h, ctm_prof_entry* out, int max_entries, int* n_entries);

/* Kernels launched by this handle since ctm_init. */
ctm_status ctm_launch_count(ctm_handle* h, long long* launches);

/* Autotuner of the tensor-core GEMMs (a no-op with *n_out = 0 for CTM_FP64).
 * CTM_TF32 / CTM_BF16: for each of the three products of the step --
 * X1 = P^t Omega P (N x N x m), C~ V (N x b x N) and U^t X (m x N x N),
 * N = m q -- it times every launch shape (tile width 64, 128 or 256
 * columns; 1 to 8 K slices, whose partial tiles fit the handle's split-K
 * buffer of 4 N b doubles).  CTM_OZAKI64: the K slices (1 to 6 whole
 * 512-wide exact chunks, or the kernel's own rule) of the two long-K
 * products C~ V and U^t X (entries report bn = 64, the kernel's fixed tile
 * width).  Timing uses CUDA events on the handle's stream, reps launches
 * each (<= 0: 5), on zeroed operands; the fastest shape is kept for every
 * later GEMM of that shape and precision in this process (all handles).  Uses only scratch buffers: call it between steps.  out (host,
 * may be NULL) receives up to max_out entries, *n_out their count.  Split
 * shapes sum their K slices in a fixed order, so results stay deterministic
 * but change in the last bits of the FP32 accumulation when the shape
 * changes. */
typedef struct {
    int M, N, K;         /* GEMM D (M x N) = A (M x K) . B^t                  */
    int bn, splits;      /* chosen tile width and K slices                     */
    double ms_default;   /* time per launch of the untuned shape               */
    double ms_best;      /* time per launch of the chosen shape                */
    int candidates;      /* shapes timed                                       */
} ctm_tune_entry;
ctm_status ctm_tune(ctm_handle* h, int reps, ctm_tune_entry* out, int max_out, int* n_out);

/* The process-wide table of launch shapes that ctm_tune fills, also read by
 * ctm_contract: pin (bn in {64, 128, 256}, splits 1..16) or clear
 * (splits = 0) the shape of the TF32 / BF16 GEMM D (M x N) = A (M x K) B^t,
 * or read the shape in force (*splits: the K slices it launches).
 * ctm_contract_workspace_size includes the partial tiles of the shape in
 * force when it is called. */
ctm_status ctm_tc_plan_set(ctm_precision prec, int M, int N, int K, int bn, int splits);
ctm_status ctm_tc_plan_get(ctm_precision prec, int M, int N, int K, int* bn, int* splits);

/* Temperature scan: nbeta independent runs of Algorithm 3 that differ only
 * in beta (the paper's temperature sweeps, Figs. 3-5).  Each beta gets its
 * own handle and workspace; a pool of `workers` host threads (1..64), each
 * with its own non-blocking CUDA stream, takes the betas in order and steps
 * each one until it converges (delta < tol_spectrum) or has taken max_steps
 * steps in this call, so betas converge independently with uneven step
 * counts and the kernels of different betas overlap on the GPU.
 *  - ctm_scan_init: base is the configuration of every beta except beta
 *    itself (betas: host, nbeta entries, each validated as in ctm_init).
 *    base->workspace NULL: the scan allocates all workspaces; otherwise it
 *    must hold ctm_scan_workspace_size bytes (caller-owned).  cuda_stream is
 *    synchronised once so that work queued on the workspace comes first;
 *    the scan then uses its own streams.  Uses the device current at init.
 *  - ctm_scan_run: steps every not-yet-converged beta; steps_done and
 *    converged (host, nbeta entries each, may be NULL) receive the steps
 *    taken in this call and the convergence flags.  Returns the first hard
 *    error of any beta (with "beta[i]:" in the message), else
 *    CTM_ENOTCONVERGED if a subspace iteration hit its cap, else CTM_OK.
 *    Returns after every beta's work has finished.
 *  - ctm_scan_observables: ctm_observables of every beta (out: nbeta).
 *  - ctm_scan_handle: the handle of one beta (owned by the scan) for the
 *    per-handle calls; ctm_scan_get_spectrum: its Omega (m entries).
 *  - ctm_scan_tune: ctm_tune on the first beta's handle (the shapes are
 *    the same for all).
 * A scan is not thread-safe: one host thread at a time per scan. */
typedef struct ctm_scan ctm_scan;
ctm_status ctm_scan_workspace_size(const ctm_config* base, int nbeta, size_t* bytes);
ctm_status ctm_scan_init(ctm_scan** s, const ctm_config* base, int nbeta, const double* betas, int workers,
                         void* cuda_stream);
ctm_status ctm_scan_tune(ctm_scan* s, int reps, ctm_tune_entry* out, int max_out, int* n_out);
ctm_status ctm_scan_run(ctm_scan* s, int max_steps, int* steps_done, int* converged);
ctm_status ctm_scan_observables(ctm_scan* s, ctm_obs* out);
ctm_status ctm_scan_handle(ctm_scan* s, int ibeta, ctm_handle** h);
ctm_status ctm_scan_get_spectrum(ctm_scan* s, int ibeta, double* omega);
void ctm_scan_destroy(ctm_scan* s);

const char* ctm_last_error(void);
void ctm_destroy(ctm_handle* h);

#ifdef __cplusplus
}
#endif
#endif
