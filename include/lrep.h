/*
 * lrep.h - C ABI of the GB300 BOSP solver for the linear response
 * eigenvalue problem (LREP).
 *
 * Problem (eq. bse / eq. xy_algebra): with A, B symmetric, K = A - B
 * symmetric positive semi-definite and M = A + B symmetric positive
 * definite, find the nev smallest positive eigenvalues lambda of
 *     H [y; x] = lambda [y; x],   H = [[0, K], [M, 0]],
 * i.e. K x = lambda y, M y = lambda x, normalised X^T Y = I (Alg. 2,
 * output).  Zero eigenvalues (a nullspace of K, Lemma "generalized
 * nullspace") are deflated through a caller-supplied basis X0 of N(K).
 *
 * Method: the Bi-Orthogonal Structure-Preserving subspace iteration
 * (Alg. 2) with MGS biorthogonalisation (Alg. 1) and the batch-by-batch
 * moving window (Section 3.3).  Every step runs in this library's CUDA
 * kernels on one GPU; nothing runs on the host but control.
 *
 * Conventions for every entry point:
 *  - Status codes only; nothing is thrown across the ABI.  On error the
 *    problem keeps a message readable by lrep_last_error().
 *  - Memory kinds: LREP_MEM_HOST pointers are host memory and are copied;
 *    LREP_MEM_DEVICE_COPY pointers are device memory and are copied;
 *    LREP_MEM_DEVICE_BORROW pointers are device memory used in place and
 *    must stay valid and unchanged until lrep_destroy().
 *  - Blocks are column-major float64 with a leading dimension ld >= n.
 *  - Dense K, M (or A, B) are symmetric n x n; the full matrix is read and
 *    not symmetrised.
 *  - One problem is used from one host thread at a time.  All device work
 *    of a problem runs on the CUDA stream given at creation (NULL = the
 *    legacy default stream).
 */
#ifndef LREP_H
#define LREP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lrep_problem_s* lrep_problem;
typedef struct lrep_server_s* lrep_server;

typedef enum {
  LREP_OK = 0,
  LREP_NOT_CONVERGED = 1,   /* maxit reached; converged pairs are valid   */
  LREP_ERR_ARG = -1,        /* invalid argument                            */
  LREP_ERR_NOMEM = -2,      /* device or host allocation failed            */
  LREP_ERR_CUDA = -3,       /* a CUDA call failed                          */
  LREP_ERR_NOT_SPD = -4,    /* Cholesky of K^ or M^ failed (K singular
                               without a nullspace basis, or M not SPD)    */
  LREP_ERR_BREAKDOWN = -5,  /* NaN/Inf, or every search column discarded   */
  LREP_ERR_TIMEOUT = -6,    /* host-side deadline passed                   */
  LREP_ERR_STATE = -7,      /* call out of order (e.g. query before solve) */
  LREP_ERR_CALLBACK = -8    /* the operator callback returned non-zero     */
} lrep_status;

enum { LREP_MEM_HOST = 0, LREP_MEM_DEVICE_COPY = 1, LREP_MEM_DEVICE_BORROW = 2 };
/* LREP_FORM_AB: inputs are A and B (K = A - B, M = A + B, eq. xy_algebra);
 * LREP_FORM_KM: inputs are K and M directly. */
enum { LREP_FORM_AB = 0, LREP_FORM_KM = 1 };
/* LREP_OP_B: the SPD mass matrix B of the generalized LREP (set by
 * lrep_set_mass_*; a callback operator is asked for it when
 * lrep_set_mass_callback was called). */
enum { LREP_OP_K = 0, LREP_OP_M = 1, LREP_OP_B = 2 };
/* Arithmetic of the float64-accurate work and of the CG products (two
 * independent bits; bit 0 needs a dense, stencil or spectral operator).
 * FP64: every product in float64 (FP64 FMA units).
 * MIXED_BF16X3 (bit 0): the inexact CG products of eq. block_GS use K, M
 *   split as hi + lo bfloat16 pairs (three bf16 tensor-core products, fp32
 *   accumulation); every product that enters H^ (eq. hat_H) and every
 *   residual (eq. tol) keeps float64 accuracy.  Spectral operators: the CG
 *   products run their transforms in float32 instead; stencil operators
 *   their 7-point sums (float64 loads and stores).
 * FP64_SLICED (bit 1): the float64-accurate dense products (and, without
 *   bit 0, the CG products too) and, for every operator kind, the large
 *   tall-skinny Grams and block updates of the solve run on the bf16 tensor
 *   cores by error-free slicing: each factor held as seven base-2^8 digit
 *   planes under power-of-two row / column scales, the 28 leading
 *   digit-pair products summed exactly in integer arithmetic (levels 2..5)
 *   or in fp32 (levels 6..8, weight <= 2^-48).  Error <= ~2^-54.7 k
 *   2^(e_i + f_j) per entry (k the contracted length, 2^e_i and 2^f_j
 *   bounding row i of the left and column j of the right factor): the form
 *   of the float64 product's own bound.  Holds 14 bytes per dense K, M
 *   entry.
 * MIXED_SLICED = both bits. */
enum {
  LREP_PREC_FP64 = 0,
  LREP_PREC_MIXED_BF16X3 = 1,
  LREP_PREC_FP64_SLICED = 2,
  LREP_PREC_MIXED_SLICED = 3
};

typedef struct {
  int32_t struct_size;    /* sizeof(lrep_options), for versioning          */
  int32_t precision;      /* LREP_PREC_*; default FP64                     */
  int32_t s;              /* window multiplier, X holds s*nb columns (3)   */
  int32_t ngs;            /* block Gauss-Seidel sweeps of eq. block_GS (1) */
  int32_t cg_maxit;       /* CG iterations per solve (20)                  */
  double cg_tol;          /* CG relative residual tolerance (1e-2)         */
  int32_t maxit;          /* outer BOSP iterations (500)                   */
  double discard_tol;     /* Alg. 1 discard threshold tau (1e-10)          */
  uint64_t seed;          /* Philox key of the random start (Step 1)       */
  int32_t refresh_every;  /* recompute K U, M V every this many iterations
                             (they are otherwise updated by recurrence)     */
  double rebiorth_tol;    /* re-biorthogonalise U, V when max|U^T V - I|
                             exceeds this (1e-12)                          */
  int32_t verbose;        /* print one line per iteration to stderr        */
  int32_t profile;        /* time every operator product with CUDA events
                             (LREP_Q_PROFILE)                              */
} lrep_options;

/* y = f(x) for one operator: write op(X) into Y for ncols columns.
 * X, Y are device pointers (column-major, leading dimensions ldx, ldy),
 * stream is the cudaStream_t to run on.  Return 0 on success. */
typedef int (*lrep_apply_fn)(void* user, int32_t op, int64_t n, int32_t ncols,
                             const double* X, int64_t ldx, double* Y,
                             int64_t ldy, void* stream);

/* Fill *opts with the defaults listed above. */
void lrep_default_options(lrep_options* opts);

/* Dense symmetric operators (Section 1; Examples 1-2; BLAS3 products).
 * P1, P2: n x n, leading dimension ld; form LREP_FORM_KM: P1 = K, P2 = M;
 * LREP_FORM_AB: P1 = A, P2 = B.  mem: LREP_MEM_*.  BORROW requires
 * form KM.  stream: cudaStream_t for all work of the problem. */
lrep_status lrep_create_dense(lrep_problem* out, int64_t n, const double* P1,
                              const double* P2, int64_t ld, int32_t form,
                              int32_t mem, void* stream);

/* Sparse operators in CSR (the finite element example, Section 4.3):
 * rowptr int64[n+1], colind int32[nnz], values float64[nnz] for each of
 * the two matrices (K, M or A, B per form; with form AB both must have the
 * same pattern).  Column indices within a row may be in any order. */
lrep_status lrep_create_csr(lrep_problem* out, int64_t n, int32_t form,
                            const int64_t* rp1, const int32_t* ci1,
                            const double* v1, const int64_t* rp2,
                            const int32_t* ci2, const double* v2, int32_t mem,
                            void* stream);

/* Matrix-free 7-point stencil on an nx*ny*nz grid (index i + nx*(j + ny*k)),
 * the finite-difference analogue of the BdG example (Section 4.4):
 *   K x = lap_coef * Lap_h x + dK .* x,   M x = lap_coef * Lap_h x + dM .* x,
 *   Lap_h x = sum_d (x[+e_d] + x[-e_d] - 2 x) / h^2, zero values outside.
 * dK, dM: float64[n]. */
lrep_status lrep_create_stencil(lrep_problem* out, int32_t nx, int32_t ny,
                                int32_t nz, double h, double lap_coef,
                                const double* dK, const double* dM,
                                int32_t mem, void* stream);

/* Matrix-free Fourier spectral operator of the BdG example (Section 4,
 * Example "large-scale dense matrix", eq. bdg_KM): a periodic box of side
 * lengths L[0..2] sampled on an nx*ny*nz grid (index i + nx*(j + ny*k),
 * spacing L_d / n_d), and
 *   K x = lap_coef * Lap_F x + dK .* x,   M x = lap_coef * Lap_F x + dM .* x,
 * where Lap_F multiplies Fourier mode m of axis d by -(2 pi m / L_d)^2 for
 * the signed frequencies m in [-n_d/2, n_d/2) (the Nyquist mode included).
 * nx, ny, nz: powers of two from 1 to 256 (1 = a flat axis).  With
 * lap_coef = -1/2 and dK = V + beta phi^2 - mu, dM = dK + 2 beta phi^2 this
 * is the BdG pair L_GP, L_GP + 2 beta |phi_s|^2 of eq. bdg_KM.  Products are
 * one FFT pass per axis on the GPU (float64; float32 transforms for the CG
 * products under LREP_PREC_MIXED_BF16X3).  L: host float64[3].  dK, dM:
 * float64[n], mem as for lrep_create_stencil (copied unless borrowed; a
 * borrowed array must outlive the problem).  LREP_ERR_ARG when a grid size
 * is not a power of two in 1..256, a length is not positive and finite, or
 * a pointer is NULL. */
lrep_status lrep_create_spectral(lrep_problem* out, int32_t nx, int32_t ny,
                                 int32_t nz, const double* L, double lap_coef,
                                 const double* dK, const double* dM,
                                 int32_t mem, void* stream);

/* User operator (the matrix-free interface of Section 1): fn is called
 * with device blocks; it must not retain the pointers. */
lrep_status lrep_create_operator(lrep_problem* out, int64_t n,
                                 lrep_apply_fn fn, void* user, void* stream);

/* Basis X0 (n x r) of N(K) (Alg. 2 input).  Y0 (n x r) with M Y0 = X0 may
 * be given; when NULL it is computed by CG on M (Remark on the numerical
 * computation of the generalized nullspace).  X0, Y0 are then normalised
 * to X0^T Y0 = I (eq. V0_basis).  r = 0 clears it. */
lrep_status lrep_set_nullspace(lrep_problem p, int32_t r, const double* X0,
                               const double* Y0, int64_t ld, int32_t mem);

/* Pre-step for singular K (Remark on the numerical computation of the
 * generalized nullspace): computes an orthonormal basis X0 of N(K) on the
 * GPU by block LOBPCG on K (r_max + 4 columns, the problem's float64
 * operator products) and installs it as by lrep_set_nullspace(p, r, X0,
 * NULL, ...), so Y0 = M^-1 X0 follows by CG in the solve.  A Ritz pair
 * counts as a null vector when its Ritz value is <= sqrt(tol) ||K||_2 and
 * its residual <= tol ||K||_2 (||K||_2 by power steps); the search stops
 * once every such pair has converged and the next Ritz value is certainly
 * above sqrt(tol) ||K||_2.  0 <= r_max <= 60.  *r_host: dimension found
 * (0: K nonsingular), *iters_host: LOBPCG iterations (may be NULL).  When
 * X0_out is not NULL the basis is also copied there (n x r, leading
 * dimension ld_out >= n, host memory for mem_out = LREP_MEM_HOST, device
 * memory for LREP_MEM_DEVICE_COPY; room for r_max columns).
 * LREP_NOT_CONVERGED after maxit iterations (no basis installed);
 * LREP_ERR_ARG when the nullity exceeds r_max or K = 0. */
lrep_status lrep_find_nullspace(lrep_problem p, int32_t r_max, double tol,
                                int32_t maxit, double* X0_out, int64_t ld_out,
                                int32_t mem_out, int32_t* r_host,
                                int32_t* iters_host);

/* Generalized LREP (Remark on the generalized LREP):
 *   [[0, K], [M, 0]] [y; x] = lam [[B, 0], [0, B]] [y; x],
 * i.e. K x = lam B y, M y = lam B x, with B symmetric positive definite.
 * The solve then runs Alg. 2 in the B-inner product <u, v>_B = u^T B v:
 * X^T B Y = I, residuals of eq. tol with B Y, B X in the lam terms, the
 * block Gauss-Seidel right-hand sides B X~ Lam - M Y~ and B Y~ Lam - K X~,
 * the projections of eq. update_W/Z and Alg. 1 in the B-inner product, and
 * M Y0 = B X0 with X0^T B Y0 = I for the nullspace.
 * Dense problems: B n x n column-major (ld >= n; mem as for
 * lrep_create_dense).  CSR problems: B as CSR arrays (rowptr int64[n+1],
 * colind int32[nnz], values float64[nnz]).  Callback problems: the callback
 * is called with op = LREP_OP_B.  B = NULL (dense, CSR) clears it. */
lrep_status lrep_set_mass_dense(lrep_problem p, const double* B, int64_t ld, int32_t mem);
lrep_status lrep_set_mass_csr(lrep_problem p, const int64_t* rowptr,
                              const int32_t* colind, const double* values, int32_t mem);
lrep_status lrep_set_mass_callback(lrep_problem p, int32_t enable);

lrep_status lrep_set_options(lrep_problem p, const lrep_options* opts);

/* Optional start blocks U0, V0 (n x ncols, ncols >= s*nb + 2*nb for the
 * solve that follows) replacing the Philox draw of Step 1. */
lrep_status lrep_set_start(lrep_problem p, int32_t ncols, const double* U0,
                           const double* V0, int64_t ld, int32_t mem);

/* Alg. 2: the nev smallest positive eigenpairs, batch size nb = block
 * (nb >= nev runs Alg. 2 as printed, nb < nev the moving window),
 * convergence when eq. tol's normalised residual < tol.
 * Returns LREP_OK, LREP_NOT_CONVERGED (partial results queryable) or an
 * error. */
lrep_status lrep_solve(lrep_problem p, int32_t nev, int32_t block, double tol);

/* The same solve in steps, batch by batch (Section 3.3: with the moving
 * window the eigenpairs are computed batch by batch, 2*nb of them locked
 * at a time).  lrep_solve_begin runs Steps 1-2 (random start, projection
 * off V0, Alg. 1) and returns; lrep_solve_advance then runs outer
 * iterations of Alg. 2 until `locks` (>= 1) more lock events have happened
 * (each locks the converged 2*nb-pair prefix of the window, or the
 * remaining nev - locked pairs) or the solve ends, always stopping between
 * iterations.  *locked (may be NULL) receives the number of pairs locked so
 * far in this solve.  *done (may be NULL) is set to 1 when the solve has ended:
 * the return value is then the solve's status (LREP_OK, LREP_NOT_CONVERGED
 * or an error) and the results are queryable exactly as after lrep_solve;
 * before that it returns LREP_OK and lrep_query reports LREP_ERR_STATE
 * (except for the LREP_Q_PROFILE* queries, which report the work so far).
 * lrep_solve_begin(p, ...) followed by lrep_solve_advance until done gives
 * the same iterations and results as lrep_solve(p, ...).  Any other call
 * that changes the problem (options, nullspace, start, mass matrix,
 * lrep_solve, lrep_destroy) ends a solve in progress; LREP_ERR_STATE when
 * advancing without one. */
lrep_status lrep_solve_begin(lrep_problem p, int32_t nev, int32_t block, double tol);
lrep_status lrep_solve_advance(lrep_problem p, int32_t locks, int32_t* locked,
                               int32_t* done);

/* What lrep_query returns.  dst receives dst_bytes at most; mem is
 * LREP_MEM_HOST or LREP_MEM_DEVICE_COPY (device destination). */
enum {
  LREP_Q_NCONV = 0,      /* int32: converged pairs                          */
  LREP_Q_EIGVALS = 1,    /* float64[nconv], ascending                       */
  LREP_Q_X = 2,          /* float64 n x nconv, column-major, X^T Y = I      */
  LREP_Q_Y = 3,          /* float64 n x nconv                               */
  LREP_Q_U = 4,          /* float64 n x nconv: u = y + x (eq. bse variables)*/
  LREP_Q_V = 5,          /* float64 n x nconv: v = y - x                    */
  LREP_Q_RESID = 6,      /* float64[nconv]: eq. tol residual at exit        */
  LREP_Q_ITERS = 7,      /* int32: outer iterations                         */
  LREP_Q_MATVECS = 8,    /* int64: operator columns applied                 */
  LREP_Q_TIMINGS = 9,    /* float64[5] seconds: init U,V / small problem /
                            convergence check / P,Q / W,Z (Table 6 buckets)*/
  LREP_Q_BIORTH_ERR = 10,/* float64: max |X^T Y - I| of the result          */
  LREP_Q_HISTORY = 11,   /* float64[iters]: max residual per iteration      */
  LREP_Q_REBIORTHS = 12, /* int32: safeguard re-biorthogonalisations        */
  LREP_Q_PROFILE = 13,   /* float64[4] with options.profile set: operator
                            product device time (s), product launches,
                            product flops (2 nnz per column), and product
                            algorithmic bytes (operator read once per
                            launch + input and output blocks)             */
  LREP_Q_PROFILE_CG = 14,/* float64[4]: the same for the products of the CG
                            operator alone (eq. block_GS)                 */
  LREP_Q_PROFILE_CLASSES = 15 /* float64[2 * LREP_PC_COUNT] with
                            options.profile set: (device seconds, timed
                            spans) of each LREP_PC_* class of solver work,
                            every span timed by CUDA events on the
                            problem's stream                              */
};
/* Classes of solver work in LREP_Q_PROFILE_CLASSES. */
enum {
  LREP_PC_PROD_CG = 0, /* CG operator products (eq. block_GS)              */
  LREP_PC_PROD = 1,    /* float64-accurate operator products               */
  LREP_PC_GRAM = 2,    /* tall-skinny Grams (eq. hat_H, projections, Alg. 1) */
  LREP_PC_UPDATE = 3,  /* block updates (pullback, P~, projections, Alg. 1)  */
  LREP_PC_SMALL = 4,   /* small LREP and eq. hat_pq                        */
  LREP_PC_CGVEC = 5,   /* CG vector updates (alpha, x/r update, directions) */
  LREP_PC_ALG1 = 6,    /* Alg. 1 coefficients on the Gram                  */
  LREP_PC_OTHER = 7,   /* residuals, right-hand sides, column norms        */
  LREP_PC_COUNT = 8
};
lrep_status lrep_query(lrep_problem p, int32_t what, void* dst,
                       int64_t dst_bytes, int32_t mem);

/* Message of the last error on p (never NULL; "" when none). */
const char* lrep_last_error(lrep_problem p);

lrep_status lrep_destroy(lrep_problem p);

/* ---- serving: continuous batching of concurrent solves ----------------
 * A server owns max_slots host threads, each running one admitted solve at
 * a time on its own CUDA stream, so the device work of concurrent requests
 * overlaps; the small projected problems of order < 40 of the running
 * solves are batched into shared launches.  When a slot is free, the
 * queued request with the smallest HBM footprint that fits
 * hbm_budget_bytes next to the running solves starts (a request passed
 * over 64 times goes first once it fits, and nothing overtakes it while it
 * waits).  The problems passed to submit must stay alive until wait
 * returns.
 */
/* Device bytes a solve of (nev, block) on p needs beyond the operator
 * itself (solver workspace, plus the bf16 operator split in mixed mode when
 * it is not built yet): the footprint the server admits requests by. */
lrep_status lrep_footprint(lrep_problem p, int32_t nev, int32_t block, int64_t* bytes);

lrep_status lrep_server_create(lrep_server* out, int64_t hbm_budget_bytes,
                               int32_t max_slots, void* stream);
lrep_status lrep_server_submit(lrep_server s, lrep_problem p, int32_t nev,
                               int32_t block, double tol, uint64_t* ticket);
/* Wait for a ticket with a host-side deadline (timeout_ms < 0: forever).
 * Returns the solve's status, or LREP_ERR_TIMEOUT. */
lrep_status lrep_server_wait(lrep_server s, uint64_t ticket, int32_t timeout_ms);
/* Stops accepting work after the queued requests finish, then frees. */
lrep_status lrep_server_destroy(lrep_server s);
/* Shared-launch statistics: out3[0] batched small-LREP launches,
 * out3[1] small problems solved by them, out3[2] largest batch. */
lrep_status lrep_server_stats(lrep_server s, int64_t* out3);

#ifdef __cplusplus
}
#endif
#endif /* LREP_H */
