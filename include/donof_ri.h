/*
 * donof_ri.h -- C ABI of the GB300 resolution-of-the-identity Coulomb/exchange
 * engine for PNOF7 (arXiv 2012.15662, "Resolution of the identity
 * approximation applied to PNOF correlation calculations").
 *
 * The engine evaluates, on one GPU, the RI algebra of Sec. 2:
 *   Eq. (AOERI)       (mu nu|s l) = sum_kl (mu nu|k) G^-1_kl (l|s l), G_kl = (k|l)
 *   fitted tensor     B^P_{mu nu} = sum_Q (L^-1)_PQ (Q|mu nu), G = L L^T
 *   half transform    b^P_{p nu} = sum_mu C_{mu p} B^P_{mu nu}      (Tables 2/3, step 2)
 *   diagonal          b^P_{pp}   = sum_nu C_{nu p} b^P_{p nu}       (Table 3, step 3)
 *   full transform    b^P_{pq}   = sum_nu C_{nu q} b^P_{p nu}       (Table 2, step 3)
 *   MO J / K          J_pq = sum_P b^P_pp b^P_qq, K_pq = sum_P (b^P_pq)^2 (Table 2, step 4)
 *   per-orbital AO    J^(q) = sum_P b^P_qq B^P,
 *                     K^(q)_{mu nu} = sum_P b^P_{q mu} b^P_{q nu}   (Table 3, steps 3-4)
 *   PNOF7 energy      Eq. (PNOF) with the PNOF7 Delta / Pi, and the
 *                     orthonormality Lagrangian lambda of Sec. 2
 *                     ("Orbital Optimization with RI").
 *
 * Basis: s-type Gaussians (orbital basis L2-normalised, auxiliary basis
 * Coulomb-normalised so that (k|k) = 1); all integrals are evaluated on the
 * device at init.
 *
 * Conventions (every entry point):
 *  - Returns DONOF_RI_OK (0) or a negative status; no exception crosses the ABI.
 *  - Matrices of orbital coefficients and lambda are column-major
 *    [nbf x nbf] FP64: element (mu, p) at index p*nbf + mu (column p is
 *    orbital p), matching the paper's C_{mu p}.
 *  - J, K are row-major [N_Omega x N_Omega] FP64 (symmetric).
 *  - Pointers documented "host or device" may be either; the engine asks the
 *    CUDA runtime which one it is.  Outputs to host memory are complete when
 *    the call returns (the call synchronises the context's stream); outputs
 *    to device memory are written asynchronously on the context's stream.
 *  - Inputs are copied; the caller keeps ownership of every pointer it passes.
 *  - A context is bound to the stream given at init, is not thread-safe, and
 *    owns all of its device buffers until donof_ri_destroy.
 *  - Device-side faults detected asynchronously (a non-finite orbital
 *    coefficient, a non-positive metric pivot) are reported by the next call
 *    that synchronises (any call with a host output, or donof_ri_sync).
 */
#ifndef DONOF_RI_H
#define DONOF_RI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define DONOF_RI_OK 0
#define DONOF_RI_E_ARG (-1)            /* bad size, null pointer, bad mode          */
#define DONOF_RI_E_OOM (-2)            /* device allocation failed                  */
#define DONOF_RI_E_CUDA (-3)           /* CUDA runtime / launch error               */
#define DONOF_RI_E_METRIC_NOT_PD (-4)  /* Cholesky pivot of G (or, for DONOF_RI_SLICE4,
                                          of the overlap S) below 1e-14 of the largest
                                          diagonal element                          */
#define DONOF_RI_E_NONFINITE (-5)      /* NaN / Inf in an input                     */
#define DONOF_RI_E_TIMEOUT (-6)        /* a bounded device-side wait gave up        */
#define DONOF_RI_E_STATE (-7)          /* call order (e.g. jk_mo before a FULL transform) */
#define DONOF_RI_E_UNSUPPORTED (-8)    /* device is not sm_103 / precision not built */

/* Arithmetic of the hot path. */
#define DONOF_RI_FP64 0    /* every product and sum in FP64 (CUDA cores)              */
#define DONOF_RI_TF32X3 1  /* split-precision tensor-core products (3 TF32 MMAs per
                              product, FP32 accumulation); FP64 metric, fitting and
                              energy/lambda sums                                     */
#define DONOF_RI_SLICE4 2  /* fixed-point BF16 digit planes: every GEMM operand row as a
                              power-of-two exponent and four balanced 8-bit digits;
                              13 BF16 tensor-core MMAs per product (digit pairs of
                              weight >= 2^-32 of the leading pair), summed exactly in
                              FP32 within 512-wide K chunks and across chunks in
                              int64 or double-float: FP64-class results (about 2^-31
                              of the row scale) from BF16 tensor cores.  Computes in
                              the orbital basis orthonormalised by the Cholesky
                              factor of the overlap (S = L L^T: orbitals L^T C,
                              fitted tensor L^-1 B L^-T, set up at init), where the
                              orbital coefficients of orthonormal orbitals are at
                              most 1 and the fixed-point products lose no bits to
                              cancellation; AO outputs (b_half, J^(q), K^(q)) are
                              transformed back when they are copied out             */

/* Transform modes. */
#define DONOF_RI_HALF 0  /* half transform + diagonal (orbital step, Table 3)          */
#define DONOF_RI_FULL 1  /* half transform + diagonal + full transform (Table 2)       */

typedef struct donof_ri_ctx donof_ri_ctx;

/*
 * Problem statement (Sec. 2): the molecule, its s-type orbital and auxiliary
 * bases and the electron-pairing scheme.  All arrays are host memory owned by
 * the caller; init copies them.
 *   nbf, naux          N_b and N_aux (>= 1)
 *   n_atoms            number of nuclei; atom_xyz [n_atoms*3] (bohr), atom_charge [n_atoms]
 *   bf_atom, bf_alpha  [nbf]  centre index and exponent of each orbital basis function
 *   aux_atom, aux_alpha [naux] centre index and exponent of each auxiliary function
 *   n_strong           N_I: strong orbitals, one per pairing subspace
 *   n_weak_per         N_g: weak orbitals per subspace (>= 1)
 *   subspace           [N_Omega] subspace g (0..N_I-1) of each pairing-space column,
 *                      N_Omega = N_I (1 + N_g) <= nbf; columns N_Omega..nbf-1 are empty
 *   weak_rank          [N_Omega] -1 for the strong orbital of its subspace, i for its
 *                      i-th weak orbital (each subspace: one strong, ranks 0..N_g-1)
 */
typedef struct donof_ri_system {
  int nbf;
  int naux;
  int n_atoms;
  int n_strong;
  int n_weak_per;
  const double* atom_xyz;
  const double* atom_charge;
  const int* bf_atom;
  const double* bf_alpha;
  const int* aux_atom;
  const double* aux_alpha;
  const int* subspace;
  const int* weak_rank;
} donof_ri_system;

/*
 * Build a context: evaluates S, T, V, E_nuc, the metric G_kl = (k|l) and the
 * three-centre integrals (k|mu nu) on the device, factorises G = L L^T in FP64
 * (plain Cholesky in place of the paper's modified LDL^T, Sec. 2), solves for
 * the fitted tensor B (Table 2/3 step 1) and lays B out for the chosen
 * precision.  Synchronous.
 *   precision  DONOF_RI_FP64, DONOF_RI_TF32X3 or DONOF_RI_SLICE4
 *   stream     cudaStream_t to run on (NULL = legacy default stream)
 *   out        receives the context
 * Errors: E_ARG (sizes, pairing map), E_OOM, E_CUDA, E_METRIC_NOT_PD,
 *         E_UNSUPPORTED (no sm_103 device).
 */
int donof_ri_init(const donof_ri_system* sys, int precision, void* stream, donof_ri_ctx** out);

/* Factorisations of the Coulomb metric G (Sec. 2, "Occupancy Optimization with RI"). */
#define DONOF_RI_METRIC_CHOLESKY 0  /* G = L L^T, B = L^-1 (k|mu nu); E_METRIC_NOT_PD
                                       below a pivot of 1e-14 max_k G_kk (the default) */
#define DONOF_RI_METRIC_MODIFIED 1  /* the paper's modified Cholesky: G = P L D L^T P^T
                                       (Bunch-Kaufman partial pivoting, alpha =
                                       (1 + sqrt 17)/8, 1x1 and 2x2 blocks in D), every
                                       eigenvalue of a D block below delta =
                                       metric_tol * max_k G_kk raised to delta
                                       (Cheng-Higham) giving D~, and b from
                                       P L D~^(1/2) b^T = (mu nu|k) with D~^(1/2) the
                                       symmetric square root of each block.  With a
                                       positive-definite G and no raised eigenvalue, b
                                       is the Cholesky fit up to an orthogonal rotation
                                       of the auxiliary index (every J/K result equal). */

/* Options of donof_ri_init_ex (host memory, read during the call). */
typedef struct donof_ri_options {
  int metric;         /* DONOF_RI_METRIC_CHOLESKY or DONOF_RI_METRIC_MODIFIED     */
  double metric_tol;  /* MODIFIED: relative eigenvalue floor, 0 < metric_tol < 1  */
} donof_ri_options;

/*
 * donof_ri_init with options; opt == NULL is donof_ri_init.  The modified
 * factorisation runs one pivot step per pair of launches (O(naux^3) FP64 work,
 * once per context) and uses a temporary copy of the three-centre tensor.
 * After init, donof_ri_fetch(METRIC) returns L (unit lower triangular, in the
 * pivoted order) in place of the Cholesky factor.
 * Errors: as donof_ri_init; E_ARG for an unknown metric or a tolerance outside
 * (0, 1).
 */
int donof_ri_init_ex(const donof_ri_system* sys, int precision, void* stream, const donof_ri_options* opt,
                     donof_ri_ctx** out);

/*
 * Counts of the metric factorisation of a context (host outputs, any may be
 * NULL): 2x2 pivot blocks, eigenvalues raised by the correction, symmetric
 * interchanges.  All zero for the Cholesky factorisation.  Errors: E_ARG.
 */
int donof_ri_metric_info(const donof_ri_ctx* ctx, int* n_pivots_2x2, int* n_raised, int* n_interchanges);

/*
 * Transform the fitted tensor to the orbitals C (host or device, [nbf*nbf]
 * column-major FP64).  HALF: b^P_{p nu} and b^P_pp for p < N_Omega (Tables
 * 2/3 step 2, Table 3 step 3).  FULL: additionally b^P_pq and the MO J, K
 * (Table 2 steps 3-4), kept for donof_ri_jk_mo.  Asynchronous.
 * Errors: E_ARG, E_CUDA; E_NONFINITE is reported at the next synchronising call.
 */
int donof_ri_transform(donof_ri_ctx* ctx, const double* C, int mode);

/*
 * MO Coulomb and exchange matrices of the last FULL transform (Table 2 step 4):
 * J, K [N_Omega*N_Omega] row-major FP64, host or device, either may be NULL.
 * Errors: E_STATE if no FULL transform preceded it.
 */
int donof_ri_jk_mo(donof_ri_ctx* ctx, double* J, double* K);

/*
 * Per-orbital AO Coulomb and exchange matrices of the last transform (Table 3
 * steps 3-4), J^(q) and K^(q) for every pairing-space orbital q, kept in the
 * context for donof_ri_energy_lagrangian.  Jao / Kao, if not NULL, receive a
 * copy as [N_Omega][nbf][nbf] FP64 (host or device).
 * Errors: E_STATE if no transform preceded it.
 */
int donof_ri_jk_ao_batch(donof_ri_ctx* ctx, double* Jao, double* Kao);

/*
 * PNOF7 energy and Lagrangian (Eq. (PNOF); Sec. 2, orbital optimisation) from
 * the occupation angles gamma (host or device, [N_I*N_g] FP64: N_I strong
 * angles, then N_g-1 weak angles per subspace) and the J^(q), K^(q) of the last
 * donof_ri_jk_ao_batch:
 *   n_g = (1+cos^2 gamma_g)/2, n_{g,i} = (1-n_g) alpha_i (alpha from the weak angles),
 *   F^(p) = n_p H + sum_q (A_pq J^(q) - B_pq K^(q)),
 *   lambda_qp = C_q^T F^(p) C_p (q < nbf, p < N_Omega; 0 for p >= N_Omega),
 *   E = E_nuc + sum_p (n_p H_pp + lambda_pp).
 * E (host or device, one FP64) and lambda ([nbf*nbf] column-major, host or
 * device) may each be NULL.
 * Errors: E_STATE if donof_ri_jk_ao_batch has not run since the last transform.
 */
int donof_ri_energy_lagrangian(donof_ri_ctx* ctx, const double* gamma, double* E, double* lambda);

/*
 * One whole PNOF7 iteration of the engine in one call: donof_ri_transform(C,
 * mode); for FULL, donof_ri_jk_mo(J, K); donof_ri_jk_ao_batch(NULL, NULL);
 * donof_ri_energy_lagrangian(gamma, E, lambda).  Arguments as in those calls
 * (J, K, E, lambda may be NULL).
 * use_graph != 0: when every non-NULL pointer is device memory or page-locked
 * host memory (cudaHostAlloc, cudaHostRegister) and the context's stream is not
 * the legacy default stream, the launch sequence, including the copies from and
 * to host memory, is captured once into a CUDA graph, keyed by (C, gamma, mode,
 * J, K, E, lambda), and replayed on later calls with the same key (one graph
 * launch per iteration; a replay reads the inputs' current contents).  With a
 * host output the call returns after the stream has written it.  Otherwise
 * (pageable host memory, or use_graph == 0) the calls run eagerly.  Profiling events are not
 * recorded inside graphs.  Unless per-row profiling is on, the part of the
 * energy row that needs only C, H and gamma (occupations, couplings, Fock
 * weights, H C) runs on an internal side stream concurrently with the
 * transforms and is joined back before F^(p) C_p; the call is still ordered on
 * the context's stream as a whole.  Errors: as the four calls; E_CUDA if
 * capture fails.
 */
int donof_ri_iteration(donof_ri_ctx* ctx, const double* C, const double* gamma, int mode, double* J, double* K,
                       double* E, double* lambda, int use_graph);

/*
 * The paper's orbital step (Sec. 2, "Orbital Optimization with RI"): diagonalise
 * the symmetric matrix F^lambda built from the Lagrangian of the last
 * donof_ri_energy_lagrangian and rotate the orbitals onto its eigenvectors, in
 * increasing order of eigenvalue (aufbau):
 *   F_qp = lambda_qp - lambda_pq for q > p (mirrored); an element larger than
 *   `bound` in magnitude is scaled by the smallest power of 1/10 that brings it to
 *   `bound` or below; F_pp = diag[p] (the previous step's eigenvalues), or
 *   lambda_pp when `first` is nonzero.
 * At a stationary point (lambda symmetric) the step changes nothing.  The
 * eigenproblem is solved in FP32 with the rotation kept as V - I: cyclic Jacobi
 * in one CTA for nbf <= 160, two-sided block Jacobi (32-wide blocks, one launch per
 * round for the 64 x 64 sub-problems and one for the update) above; the
 * eigenvectors are then refined in FP64 against F^lambda, C V is formed in FP64
 * and re-orthonormalised by one Newton-Schulz step.  nbf <= 2048.
 *   diag    [nbf] in (unless first) / out: the eigenvalues, host or device
 *   bound   > 0
 *   C       out or NULL: the rotated orbitals (column-major, host or device); the
 *           context keeps them, and the next transform must be called with them
 *   gmax    out (host) or NULL: max |lambda_qp - lambda_pq| before the step
 *   sweeps  out (host) or NULL: Jacobi sweeps used (at most 30)
 * Synchronous.  Errors: E_ARG, E_OOM, E_STATE (no Lagrangian since the orbitals
 * last changed), E_NONFINITE (diag), E_UNSUPPORTED (nbf > 2048).
 */
int donof_ri_flambda_step(donof_ri_ctx* ctx, double* diag, int first, double bound, double* C, double* gmax,
                          int* sweeps);

/*
 * Energy and Lagrangian in the contracted form: F^(p) C_p straight from the RI
 * transforms, without the per-orbital AO matrices J^(q), K^(q):
 *   J^(q) C_p = sum_P b^P_qq b^P_{p .},   K^(q) C_p = sum_P b^P_{q .} b^P_qp,
 * so F^(p) C_p = n_p H C_p + sum_P w_pP b^P_{p .} - sum_P sum_q B_pq b^P_qp b^P_{q .}
 * with w_pP = sum_q A_pq b^P_qq (one batched DGEMM over P of N_b x N_Omega x
 * N_Omega, N_b N_aux N_Omega^2 multiply-adds in place of 2 N_b^2 N_aux N_Omega for
 * J^(q), K^(q) and the Fock sum).  lambda and E as in donof_ri_energy_lagrangian,
 * which gives the same values (no donof_ri_jk_ao_batch needed).
 * FP64 contexts: needs the full transform b^P_qp (call after a FULL
 * donof_ri_transform); scratch of N_aux N_Omega (1 + N_Omega + N_b) doubles,
 * allocated on first use.
 * DONOF_RI_SLICE4 contexts: needs a HALF or FULL transform; the call runs the full
 * transform's digit-plane GEMM once more with b^P_qp stored (FP64), forms
 * X^P_qp = [q = p] w_pP - B_pq b^P_qp as digit rows (q, p) over P, and contracts
 * sum_q sum_P X^P_qp b^P_{q .} in one digit-plane GEMM over K = (q, P) (exact
 * sums per K chunk, double-float across chunks and orbitals); scratch of
 * N_aux N_Omega (N_Omega + 1) doubles, 8 N_Omega^2 N_aux bytes of digits and
 * N_Omega^2 exponents, allocated on first use.  lambda and E within the digit
 * path's tolerances of the per-orbital form.
 * Errors: E_ARG, E_OOM, E_STATE (no FULL transform (FP64) or no transform
 * (SLICE4) since the orbitals changed), E_UNSUPPORTED (DONOF_RI_TF32X3),
 * E_TIMEOUT (SLICE4: a bounded device wait ran out).
 */
int donof_ri_energy_lagrangian_contracted(donof_ri_ctx* ctx, const double* gamma, double* E, double* lambda);

/*
 * Exact four-centre J and K for orbitals C (the conventional algorithm of Table 1,
 * Eqs. (Jpq), (Pmat), (Kpq), with exact s-type integrals (mu nu|l s) in place of
 * Eq. (AOERI)): the paper's RI -> exact restart finishes an RI-converged
 * calculation with a few exact iterations (Sec. 1, Sec. 4).  Computes
 * J^(q)_{mu nu} = sum_{l s} (mu nu|l s) C_{l q} C_{s q},
 * K^(q)_{mu nu} = sum_{l s} (mu l|nu s) C_{l q} C_{s q} and
 * J_pq = C_p^T J^(q) C_p, K_pq = C_p^T K^(q) C_p in FP64 and leaves them in the
 * context in place of the RI ones, so that donof_ri_energy_lagrangian and
 * donof_ri_optimize_occupations that follow use exact integrals (until the next
 * transform).  The integrals are stored (nbf^4 doubles) together with one
 * half-contracted copy (nbf^3 N_Omega doubles), allocated for the call.
 *   C      [nbf][nbf] column-major orbitals, host or device
 *   J, K   [N_Omega][N_Omega] outputs, host or device, or NULL
 * Synchronous.  Errors: E_ARG, E_OOM, E_CUDA, E_NONFINITE, E_UNSUPPORTED (a
 * precision other than DONOF_RI_FP64, or nbf > 256).
 */
int donof_ri_exact_jk(donof_ri_ctx* ctx, const double* C, double* J, double* K);

/* Internal arrays readable through donof_ri_fetch (converted to FP64). */
#define DONOF_RI_FETCH_B 0        /* [naux][nbf][nbf]   fitted tensor B^P_{mu nu}      */
#define DONOF_RI_FETCH_BHALF 1    /* [naux][N_Omega][nbf] b^P_{p nu}                   */
#define DONOF_RI_FETCH_DIAG 2     /* [naux][N_Omega]    b^P_pp                         */
#define DONOF_RI_FETCH_HCORE 3    /* [nbf][nbf]         H = T + V                      */
#define DONOF_RI_FETCH_OVERLAP 4  /* [nbf][nbf]         S                              */
#define DONOF_RI_FETCH_METRIC 5   /* [naux][naux]       G (lower triangle holds L after init) */
#define DONOF_RI_FETCH_ENUC 6     /* [1]                E_nuc                          */
#define DONOF_RI_FETCH_OCC 7      /* [N_Omega]          occupations of the last energy call */

/*
 * Copy an internal array to host memory dst (count FP64 elements, which must
 * equal the array's size).  Synchronous.  Errors: E_ARG, E_STATE.
 */
int donof_ri_fetch(donof_ri_ctx* ctx, int what, double* dst, size_t count);

/* Wait for the context's stream and report any deferred device-side error. */
int donof_ri_sync(donof_ri_ctx* ctx);

/* Free every device buffer of the context.  Accepts NULL. */
int donof_ri_destroy(donof_ri_ctx* ctx);

/* Static, human-readable text for a status code. */
const char* donof_ri_strerror(int status);

/* Number of kernels the context has launched since init (for launch accounting). */
long long donof_ri_launch_count(const donof_ri_ctx* ctx);

/*
 * Check of the fault path of the bounded device-side waits (the paper has no
 * counterpart: this is the engine's own failure detection).  Every mbarrier wait
 * in the engine's tensor-core kernels gives up after about two seconds, records
 * a timeout in the context's status word and lets its CTA exit with no copy or
 * MMA in flight; the next synchronising call returns DONOF_RI_E_TIMEOUT and the
 * context stays usable.  This call launches one CTA on the context's stream whose
 * wait, on an mbarrier that nothing completes, runs out after limit_ns
 * nanoseconds (1e3 <= limit_ns <= 5e9), so that the same path can be tested
 * without faulting or hanging the GPU.  Asynchronous; the timeout is reported by
 * the next synchronising call (e.g. donof_ri_sync).  Errors: E_ARG, E_CUDA.
 */
int donof_ri_check_wait_timeout(donof_ri_ctx* ctx, long long limit_ns);

/* Hot-path rows timed by the profiler (CUDA events on the context's stream). */
#define DONOF_RI_ROW_HALF 0      /* a1: half transform b^P_{p nu}                     */
#define DONOF_RI_ROW_DIAG 1      /* a2: diagonal b^P_pp                               */
#define DONOF_RI_ROW_FULL_K 2    /* a3: full transform b^P_pq and K_pq                */
#define DONOF_RI_ROW_J 3         /* a4: J_pq                                          */
#define DONOF_RI_ROW_JAO 4       /* a5: per-orbital J^(q)                             */
#define DONOF_RI_ROW_KAO 5       /* a6: per-orbital K^(q)                             */
#define DONOF_RI_ROW_ENERGY 6    /* a7: occupations, F^(p) C_p, lambda and E          */
#define DONOF_RI_ROW_OTHER 7     /* input copies, finiteness checks, conversions      */
/* The tensor-core GEMM kernel of a row alone (SLICE4 and TF32X3; the FP64 form
 * records none): one event pair around that one launch, nested inside the row's. */
#define DONOF_RI_GEMM_HALF 8     /* a1 GEMM                                           */
#define DONOF_RI_GEMM_FULL_K 9   /* a3 GEMM (full transform with the squares summed)  */
#define DONOF_RI_GEMM_J 10       /* a4 GEMM                                           */
#define DONOF_RI_GEMM_JAO 11     /* a5 GEMM                                           */
#define DONOF_RI_GEMM_KAO 12     /* a6 GEMM                                           */
#define DONOF_RI_GEMM_FOCK 13    /* a7 GEMM: sum_q (A_pq J^(q) - B_pq K^(q)) C_p      */
/* The memory-bound passes of SLICE4 alone (one event pair around the launch, nested
 * inside its row's; the other forms record none). */
#define DONOF_RI_MEM_DIGITS 14   /* a1/a2: b_half's two digit layouts + diagonal partials */
#define DONOF_RI_MEM_SPLIT 15    /* a5/a6: J^(q), K^(q) as digit planes for a7's GEMM    */
#define DONOF_RI_NUM_ROWS 16

/*
 * Enable (1) or disable (0) per-row timing.  While enabled, every launch group
 * of a hot-path row is bracketed by a pair of CUDA events recorded on the
 * context's stream (this also works inside a captured CUDA graph).
 * Disabling discards pending records.  Errors: E_ARG.
 */
int donof_ri_profile(donof_ri_ctx* ctx, int enable);

/*
 * Synchronise, then return for row `row` the summed event time (ms) and the
 * number of timed launch groups since the last read, and reset that row.
 * Errors: E_ARG, E_CUDA.
 */
int donof_ri_profile_read(donof_ri_ctx* ctx, int row, double* total_ms, long long* count);

/*
 * Occupation optimisation for fixed orbitals (Sec. 2, "Occupancy Optimization
 * with RI"): with J, K of the last FULL transform fixed, the PNOF7 energy of
 * Eq. (PNOF) is minimised over the unconstrained angles gamma (occupation map as
 * in donof_ri_energy_lagrangian).  The paper names no optimiser: L-BFGS (8
 * pairs, backtracking Armijo line search) on the analytic gradient
 * dE/dgamma = sum_p dE/dn_p dn_p/dgamma, FP64, in one single-CTA kernel.
 *   gamma     in: start, out: result folded into [0, pi/2] (E depends on cos^2 and
 *             sin^2 of the angles only); [N_I*N_g] FP64, host or device
 *   max_iter  iteration cap, 0..1000000 (0: only evaluates E and the gradient)
 *   gtol      stop when max_k |dE/dgamma_k| <= gtol (>= 0)
 *   etol      stop when an iteration lowers E by at most etol * max(1, |E|) (>= 0); a
 *             minimum where an occupation reaches 0 or 1 lies on a kink of E(gamma)
 *             (the sqrt(n) terms), where the gradient need not vanish
 *   E         out: energy at the result (host or device, one FP64) or NULL
 *   grad      out: dE/dgamma at the result ([N_I*N_g] FP64, host or device) or NULL
 *   info      out (host) or NULL: info[0] iterations, info[1] stop reason
 *             (0 gradient below gtol, 1 iteration cap, 2 line search found no
 *             decrease, 3 energy decrease below etol)
 * Synchronous when any output is in host memory.
 * Errors: E_ARG, E_STATE (no FULL transform since the orbitals last changed),
 *         E_UNSUPPORTED (N_g > 16 or N_Omega too large for one CTA's shared memory).
 */
int donof_ri_optimize_occupations(donof_ri_ctx* ctx, double* gamma, int max_iter, double gtol, double etol, double* E,
                                  double* grad, int* info);

/*
 * Tile-schedule autotuner of the SLICE4 engine (the paper has no counterpart):
 * times every digit-plane GEMM kind on the context's own problem (reps launches
 * each) for every pipeline depth that fits its shared memory, the split kinds
 * (full transform, J, F^(p)C_p) also for one and two waves of CTAs, J^(q)
 * with and without its symmetric skip-and-mirror and the half transform as the
 * two-CTA-per-SM kernel or the one-CTA kernel with two accumulator sets (each
 * launch timed from a flushed L2, as inside an iteration), and keeps for every
 * later call the fastest setting of each kind when it beats the default by at
 * least 3 %; finally J^(q) and K^(q) in one persistent launch (the default)
 * against two launches.  Needs a FULL transform and
 * donof_ri_jk_ao_batch first (their data are the timing inputs); afterwards
 * every result must be recomputed (the state returns to "no transform").
 *   reps    launches timed per setting, 1..1000
 *   report  out (host) or NULL: 6 x 4 ints, per kind (half, full, J, J^(q), K^(q),
 *           F^(p)C_p): pipeline stages, split count (J^(q): 1 if symmetric; half
 *           transform: 1 for the one-CTA kernel; K^(q): 1 if in one launch with
 *           J^(q)), CTAs, best time in microseconds
 *   tried   out (host) or NULL: settings timed
 * Synchronous.  Errors: E_ARG, E_STATE, E_UNSUPPORTED (precision other than SLICE4).
 */
int donof_ri_autotune(donof_ri_ctx* ctx, int reps, int* report, int* tried);

/*
 * Set one GEMM kind's schedule directly (a choice the autotuner can make):
 *   kind     0 half transform, 1 full transform, 2 J, 3 J^(q), 4 K^(q), 5 F^(p)C_p
 *   stages   pipeline depth, 2 .. what fits the kind's shared memory
 *   option   half transform: 0 two CTAs per SM, 1 one CTA with two accumulator
 *            sets; J^(q): 1 symmetric skip-and-mirror, 0 full; full transform,
 *            J and F^(p)C_p: 1 or 2 waves of CTAs; K^(q): 1 in one persistent
 *            launch together with J^(q) (the default), 0 in a launch of its own
 * Takes effect at the next launch (a captured iteration graph is dropped).
 * Errors: E_ARG, E_UNSUPPORTED (precision other than SLICE4).
 */
int donof_ri_set_schedule(donof_ri_ctx* ctx, int kind, int stages, int option);

/*
 * One orbital rotation step for fixed occupations (Sec. 2, "Orbital Optimization
 * with RI"; the plain rotation driver's step, which the paper's iterative
 * diagonalisation of F^lambda replaces): with G = lambda - lambda^T from the last
 * donof_ri_energy_lagrangian (the rotation gradient dE/dkappa = 4 G),
 *   C <- C expm(kappa),  kappa = -radius G / max|G|,
 * then one Newton-Schulz re-orthonormalisation C <- C (3 I - C^T C) / 2 (FP64).
 *   radius  largest rotation angle of the step, 0..3.2 (0: only reports max|G|)
 *   C       out (host or device, [nbf*nbf] column-major) or NULL: the rotated orbitals,
 *           also kept as the context's orbitals; the transforms must be redone
 *   gmax    out (host) or NULL: max|lambda_qp - lambda_pq| before the step
 * Synchronous.  Errors: E_ARG, E_STATE (no donof_ri_energy_lagrangian since the
 * last transform), E_OOM (scratch of 4 nbf^2 doubles, allocated on first use).
 */
int donof_ri_rotate_orbitals(donof_ri_ctx* ctx, double radius, double* C, double* gmax);

/*
 * Rotate the context's orbitals by a given generator: C <- C expm(kappa), then one
 * Newton-Schulz step in the overlap metric (C^T S C = I, the orbitals' constraint;
 * Sec. 2, "Orbital Optimization with RI").  kappa [nbf][nbf] FP64 row-major
 * antisymmetric (kappa_qp = -kappa_pq mixes orbital q into orbital p), host or
 * device; the exponential by scaling and squaring with a degree-12 Taylor
 * polynomial.  With the gradient dE/dkappa_qp = 4 (lambda_qp - lambda_pq) (q > p)
 * of the last donof_ri_energy_lagrangian, this is the step of a quasi-Newton
 * orbital optimisation.  C (optional) receives the rotated orbitals, column-major,
 * host or device.  Invalidates the transforms.  Errors: E_ARG, E_NONFINITE, E_CUDA.
 */
int donof_ri_apply_rotation(donof_ri_ctx* ctx, const double* kappa, double* C);

/* ------------------------------------------------------------------------
 * Learned warm start for the occupation optimisation.  The paper has no
 * learned part: this is the project's own addition.  A 3-layer MLP
 * (F -> H tanh -> H tanh -> O) with BF16 weights and FP32 arithmetic maps the
 * features of one pairing subspace to its converged angles (strong angle,
 * then the N_g - 1 weak angles, folded into [0, pi/2]).
 * ------------------------------------------------------------------------ */
typedef struct donof_mlp donof_mlp;

/* Create a network with zero parameters and identity input scaling.
 * max_batch: largest batch any later call may pass (1..2^24).  stream: the
 * cudaStream_t its kernels run on (NULL = legacy default stream).
 * Errors: E_ARG (sizes), E_OOM, E_CUDA. */
int donof_mlp_create(int n_in, int n_hidden, int n_out, int max_batch, void* stream, donof_mlp** out);
/* Number of parameters: H*F + H + H*H + H + O*H + O (W1, b1, W2, b2, W3, b3; W row-major [out][in]). */
long long donof_mlp_param_count(const donof_mlp* net);
/* Copy parameters in (host or device FP32, param_count values); resets the Adam state.  Synchronous. */
int donof_mlp_set_params(donof_mlp* net, const float* params);
/* Copy the FP32 master parameters out (host or device).  Synchronous. */
int donof_mlp_get_params(donof_mlp* net, float* params);
/* Input scaling z = (x - mean) * inv_std, F values each (host or device).  Synchronous. */
int donof_mlp_set_normalization(donof_mlp* net, const float* mean, const float* inv_std);
/* Y [batch][O] = network(X [batch][F]); FP32, host or device.  Synchronous for host Y. */
int donof_mlp_forward(donof_mlp* net, const float* X, int batch, float* Y);
/* Mean squared error against T [batch][O] and its gradient with respect to every
 * parameter (through the BF16 weight values); loss (one float) and grads
 * (param_count floats), host or device, either may be NULL.  Synchronous. */
int donof_mlp_loss_grad(donof_mlp* net, const float* X, const float* T, int batch, float* loss, float* grads);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, decoupled weight decay on the
 * matrices) on the batch (X, T); loss (host or device) may be NULL (then asynchronous). */
int donof_mlp_train_step(donof_mlp* net, const float* X, const float* T, int batch, float lr, float weight_decay,
                         float* loss);
int donof_mlp_destroy(donof_mlp* net);

/* Features of every pairing subspace g from J, K of the last FULL transform and
 * H_pp = C_p^T H C_p: X [N_I][3 + 4 N_g] FP32 (host or device), row g =
 * [H_ss, J_ss, mf_s, then per weak orbital w (rank order): H_ww, J_ww, K_sw, mf_w],
 * mf_p = sum_{q outside g} n0_q (2 J_pq - K_pq), n0 = standard-guess occupations
 * (strong 0.98, weak 0.02/N_g).  Errors: E_ARG, E_STATE. */
int donof_ri_on_features(donof_ri_ctx* ctx, float* X);
/* gamma [N_I*N_g] FP64 (host or device) predicted by net from the features of the
 * current orbitals, each angle clipped to [clip, pi/2 - clip] (0 <= clip < pi/4):
 * the warm start for donof_ri_optimize_occupations.  net must have F = 3 + 4 N_g
 * inputs and O = N_g outputs.  Errors: E_ARG, E_STATE. */
int donof_ri_gamma_guess(donof_ri_ctx* ctx, donof_mlp* net, double clip, double* gamma);

/*
 * Closed-shell RI Hartree-Fock orbitals, the starting natural orbitals of the
 * paper's calculations (Sec. 4, Computational Details: the guess NOs come from a
 * Hartree-Fock calculation).  Roothaan-Hall iterations F C = S C eps in the
 * overlap metric, F = H + J[D] - K[D]/2, D = 2 C_occ C_occ^T over the N_I lowest
 * orbitals, J[D] and K[D] from the context's fitted tensor B (FP64, every
 * precision), from the core-Hamiltonian guess with Pulay's DIIS over the last 8
 * Fock matrices (error F D S - S D F).  The eigenproblem is solved on the device
 * in the basis orthonormalised by the Cholesky factor of S.  Synchronous; device
 * work buffers are allocated for the call and freed before it returns.
 *   max_iter    iterations at most (>= 1)
 *   tol         stop when max |F D S - S D F| <= tol (> 0)
 *   C           [nbf][nbf] FP64 column-major (column p = orbital p), host or
 *               device: the orbitals in increasing order of eps, C^T S C = I
 *   eps         [nbf] orbital energies (host or device) or NULL
 *   E           SCF energy (host) or NULL; iterations, commutator (host) or NULL
 * Not converged after max_iter: the last iteration's orbitals and energy are
 * returned, with commutator above tol.
 * Errors: E_ARG, E_OOM, E_CUDA, E_UNSUPPORTED (nbf > 2048), E_NONFINITE,
 *         E_METRIC_NOT_PD (the overlap is not positive definite).
 */
int donof_ri_rhf(donof_ri_ctx* ctx, int max_iter, double tol, double* C, double* eps, double* E, int* iterations,
                 double* commutator);

/*
 * J_pq = sum_P b^P_pp b^P_qq with no device allocation.
 * The paper has no counterpart: this entry point exists for callers that may
 * not allocate device memory (code running under an allocator or memory pool
 * that forbids cudaMalloc, or a service that must keep its device footprint
 * fixed after start-up), so it takes no context.
 *   d        [naux][n_omega] FP64, device: b^P_pp, e.g. from donof_ri_fetch
 *            (DONOF_RI_FETCH_DIAG) copied to the device
 *   J        [n_omega][n_omega] FP64 row-major, device, written asynchronously
 *   stream   cudaStream_t to run on (NULL = legacy default stream)
 * Arithmetic: split TF32 tensor-core products with FP32 accumulation over
 * chunks of naux and an FP64 sum of the chunks (as DONOF_RI_TF32X3).
 * Scratch: a file-scope device array of 24 MiB that every GPU loading the
 * library holds until the process exits; it holds the split d (2 x n_omega x
 * naux floats, naux rounded up to 4) and up to 16 chunk partials (n_omega^2
 * floats each).  Sizes that do not fit return DONOF_RI_E_ARG before any work.
 * The first call on a device (the current one) looks up the array's device
 * address and the tensor-map encoder; make that first call before any stream
 * capture.  First calls from several host threads are serialised inside the
 * library.  Every call uses the same array, which keeps the last call's
 * contents (the status word is cleared by each call); calls whose work
 * overlaps on the GPU (other streams, other host threads) race on it and must
 * be serialised by the caller.  A device-side wait that times out (a bounded
 * spin of about two seconds) is not returned as a status, since the call does
 * not synchronise: every element of J is then set to NaN instead.
 * Errors: E_ARG (null pointer, sizes), E_CUDA, E_UNSUPPORTED.
 */
int donof_ri_jmo_noalloc(const double* d, int naux, int n_omega, double* J, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DONOF_RI_H */
