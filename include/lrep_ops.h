/*
 * lrep_ops.h - the hot-path steps of one BOSP iteration as separate
 * C entry points, for callers that drive their own iteration and for
 * step-by-step verification.  All pointers are DEVICE pointers unless a
 * parameter name ends in _host; blocks are column-major float64; every
 * call is asynchronous on `stream` (a cudaStream_t, NULL = legacy default)
 * except those returning a count through a _host pointer, which
 * synchronise that stream.  Return values are lrep_status codes.
 * Scratch memory is drawn from a per-device pool owned by the library
 * (grown with cudaMalloc on first use, kept until process exit); calls
 * that share a device and overlap in time must use one stream.
 */
#ifndef LREP_OPS_H
#define LREP_OPS_H

#include <stdint.h>

#include "lrep.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Step 3 / Step 6 products: Y = K X (op = LREP_OP_K) or Y = M X
 * (LREP_OP_M) for ncols columns of a problem's operator (dense, CSR,
 * stencil or callback), in the problem's precision for float64 products
 * (Section 3.2, "(2d) mv" of the Step 3 cost).  Runs on the problem's
 * stream. */
lrep_status lrep_op_apply(lrep_problem p, int32_t op, int32_t ncols,
                          const double* X, int64_t ldx, double* Y, int64_t ldy);

/* Same as lrep_op_apply but with the problem's low-precision CG operator
 * (MIXED_BF16X3: hi/lo bfloat16 split of K or M, fp32 accumulation);
 * identical to lrep_op_apply for FP64 problems. */
lrep_status lrep_op_apply_cg(lrep_problem p, int32_t op, int32_t ncols,
                             const double* X, int64_t ldx, double* Y,
                             int64_t ldy);

/* Step 6 inner solve (eq. block_GS and the text after it): one CG per
 * column for op * X = B (op = LREP_OP_K or LREP_OP_M), zero start, the
 * problem's CG operator (as lrep_op_apply_cg), the solver's own kernels.
 * Column j stops once ||r_j||_2 <= tol ||b_j||_2; the block stops after
 * maxit iterations or when every column has stopped.  B: n x ncols device
 * block (ldb >= n), X: n x ncols device output (ldx >= n), 1 <= ncols <= 64,
 * maxit >= 0.  *iters (host, may be NULL): iterations in which at least
 * one column was still active.  Runs on the problem's stream and
 * synchronises it. */
lrep_status lrep_op_cg(lrep_problem p, int32_t op, int32_t ncols, const double* B,
                       int64_t ldb, double* X, int64_t ldx, double tol, int32_t maxit,
                       int32_t* iters);

/* Tall-skinny Gram G = A^T B (A n x a, B n x b), the inner products of
 * eq. hat_H (K^ = U^T K U, M^ = V^T M V) and eq. update_W/Z.  G is a x b
 * with leading dimension ldg.  Deterministic (fixed reduction order). */
lrep_status lrep_op_gram(int64_t n, int32_t a, int32_t b, const double* A,
                         int64_t lda, const double* B, int64_t ldb, double* G,
                         int64_t ldg, void* stream);

/* Block update C = alpha C + beta A B (A n x k, B k x c): the Ritz
 * pullback X~ = U X^ (eq. eigenVector-pullback) and the projection of
 * eq. update_W/Z.  C must not overlap A. */
lrep_status lrep_op_update(int64_t n, int32_t k, int32_t c, double alpha,
                           const double* A, int64_t lda, const double* B,
                           int64_t ldb, double beta, double* C, int64_t ldc,
                           void* stream);

/* lrep_op_gram and lrep_op_update with float64 accuracy on the bf16 tensor
 * cores (error-free slicing, the route of precision FP64_SLICED): every
 * column of A and B (Gram), every row of A and column of B (update) is
 * written as a power-of-two scale times seven base-2^8 digits, and the 28
 * leading digit-pair products are summed exactly (or, below 2^-48 of the
 * scale, in fp32).  Error <= ~2^-54.7 * k * 2^(e_i + f_j), k the contracted
 * length, 2^e_i and 2^f_j bounding row i of the left and column j of the
 * right factor: the form of the float64 product's bound.  For the update,
 * 1 <= k <= 768 and beta != 0.  Synchronises `stream` (reads the kernels'
 * timeout flag); LREP_ERR_CUDA if a tensor-core pipeline wait expired.
 * Not in the paper: a GB300 device for its Grams (eq. hat_H) and block
 * updates (eq. eigenVector-pullback, eq. update_W/Z), FP64 being its
 * scarcest unit. */
lrep_status lrep_op_gram_sliced(int64_t n, int32_t a, int32_t b,
                                const double* A, int64_t lda, const double* B,
                                int64_t ldb, double* G, int64_t ldg,
                                void* stream);
lrep_status lrep_op_update_sliced(int64_t n, int32_t k, int32_t c,
                                  double alpha, const double* A, int64_t lda,
                                  const double* B, int64_t ldb, double beta,
                                  double* C, int64_t ldc, void* stream);

/* Small projected LREP (eq. small_eigen) of order d <= 256: K^, M^ are
 * d x d (leading dimension ld; symmetrised as (G + G^T)/2).  Writes the d
 * eigenvalues ascending to lam[d] and X^, Y^ (d x d, leading dimension
 * ldo) with K^ X^ = Y^ diag(lam), M^ Y^ = X^ diag(lam), X^T Y^ = I, by two
 * Cholesky factorisations and a one-sided Jacobi SVD.  *info_host: 0 ok,
 * 1 K^ not SPD, 2 M^ not SPD, 3 SVD did not converge. */
lrep_status lrep_op_small_lrep(int32_t d, const double* Khat,
                               const double* Mhat, int32_t ld, double* lam,
                               double* Xh, double* Yh, int32_t ldo,
                               int32_t* info_host, void* stream);

/* Alg. 1 (MGS-Biorth) of the pair (W, Z), n x m, with the discard rule of
 * the Remark after it (|eta| <= tau ||w_l|| ||z_l||).  Writes the kept
 * pairs to P, Q (n x kept, leading dimension ldo; must not overlap W, Z)
 * and the count to *kept_host.  P^T Q = I. */
lrep_status lrep_op_biorth(int64_t n, int32_t m, const double* W,
                           const double* Z, int64_t ld, double tau, double* P,
                           double* Q, int64_t ldo, int32_t* kept_host,
                           void* stream);

/* eq. tol residuals: eps_i = ||[KX_i - lam_i Y_i; MY_i - lam_i X_i]|| /
 * ((1 + lam_i) ||[Y_i; X_i]||) for w columns (all blocks share ld). */
lrep_status lrep_op_residuals(int64_t n, int32_t w, const double* X,
                              const double* Y, const double* KX,
                              const double* MY, int64_t ld, const double* lam,
                              double* eps, void* stream);

/* Step 1 random start: n x ncols N(0,1) block from Philox4x32-10 with key
 * (seed_lo, seed_hi) and counter (t lo, t hi, stream_id, 0), t = e / 2 for
 * element e = row + n * col, two normals per counter by Box-Muller on the
 * first two output words (u = (w + 0.5) / 2^32). */
lrep_status lrep_op_philox_normal(int64_t n, int32_t ncols, uint64_t seed,
                                  int32_t stream_id, double* out, int64_t ld,
                                  void* stream);

/* Tall-skinny Gram G = A^T B exactly like lrep_op_gram, but without any
 * device allocation, for callers that cannot allocate device memory at the
 * time of the call: processes whose HBM was reserved up front by another
 * allocator (cudaMalloc could fail), or latency-critical loops that cannot
 * accept cudaMalloc/cudaFree stalls.  The paper has no counterpart; this is
 * a deployment variant of the Gram step.
 *  - Scratch: a fixed array of 2^19 doubles (4 MiB) in device memory that is
 *    part of the library image; every GPU that loads the library holds it
 *    until the process exits.  Limit: a * b <= LREP_GRAM_NOALLOC_MAX_AB
 *    (65536); larger requests return LREP_ERR_ARG with a message in
 *    lrep_last_error(NULL).
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  - Every call shares the array and leaves its partials there; nothing in
 *    it needs to start at zero (each call overwrites what it reads).  Calls
 *    that overlap on the GPU (different streams, or different host threads)
 *    race on the array: serialise them.
 *  - Asynchronous on `stream`; results may differ from lrep_op_gram in the
 *    last bits (the split of the reduction over rows may be coarser). */
#define LREP_GRAM_NOALLOC_MAX_AB 65536
lrep_status lrep_op_gram_noalloc(int64_t n, int32_t a, int32_t b,
                                 const double* A, int64_t lda, const double* B,
                                 int64_t ldb, double* G, int64_t ldg,
                                 void* stream);

/* Number of CUDA kernels this library has launched in this process (all
 * devices, all problems); a monotone counter for accounting. */
int64_t lrep_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* LREP_OPS_H */
