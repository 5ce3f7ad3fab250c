// Host-side launchers of the solver's CUDA kernels (internal interface).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace lrep {

// ---------------------------------------------------------------- products
// Y = A X for a symmetric dense n x n A (column-major, lda) and an n x c X.
// Uses split-K partials in ws when the row tiles alone cannot fill the GPU.
size_t dense_apply_ws_elems(int64_t n, int c);
cudaError_t dense_apply_f64(int64_t n, int c, const double* A, int64_t lda,
                            const double* X, int64_t ldx, double* Y, int64_t ldy,
                            double* ws, size_t ws_elems, const int* skip,
                            cudaStream_t st);

// 7-point stencil: Y = coef * Lap_h X + d .* X (coef already divided by h^2).
cudaError_t stencil_apply_f64(int nx, int ny, int nz, double coef_h2,
                              const double* d, int c, const double* X,
                              int64_t ldx, double* Y, int64_t ldy,
                              const int* skip, cudaStream_t st);
// the same product with float64 (f32 = false) or float32 arithmetic (f32 =
// true: the inexact CG products under the mixed precision)
cudaError_t stencil_apply(bool f32, int nx, int ny, int nz, double coef_h2, const double* d,
                          int c, const double* X, int64_t ldx, double* Y, int64_t ldy,
                          const int* skip, cudaStream_t st);

// Fourier spectral operator on a periodic grid (k_spectral.cu):
// Y = coef * Lap_F X + d .* X, with scale[ax] = -coef * (2 pi / L_ax)^2 / N_ax
// and dims[ax] = N_ax powers of two <= 2^kSpectralMaxLog (1 = flat axis).
// fp32: transforms in float (the inexact products of the block CG).
constexpr int kSpectralMaxLog = 8;
int spectral_log2(int N);
cudaError_t spectral_apply(bool fp32, const int dims[3], const double scale[3],
                           const double* d, int c, const double* X, int64_t ldx, double* Y,
                           int64_t ldy, const int* skip, cudaStream_t st);

// CSR SpMM: Y = A X.
cudaError_t csr_apply_f64(int64_t n, const int64_t* rp, const int32_t* ci,
                          const double* v, int c, const double* X, int64_t ldx,
                          double* Y, int64_t ldy, const int* skip,
                          cudaStream_t st);

// ------------------------------------------------------------ tall-skinny
// G (a x b, ldg) = A^T B with A, B segmented n-row blocks.
size_t gram_ws_elems(int64_t n, int a, int b);
cudaError_t gram_f64(int64_t n, const Segs& A, const Segs& B, double* G,
                     int64_t ldg, double* ws, size_t ws_elems, cudaStream_t st);

// Gram with the slab count capped to fit ws_elems (>= a*b) doubles.
cudaError_t gram_f64_capped(int64_t n, const Segs& A, const Segs& B, double* G,
                            int64_t ldg, double* ws, size_t ws_elems, cudaStream_t st);

// C (n x c) = alpha C + beta A B, A segmented (k columns), B k x c (ldb).
cudaError_t update_f64(int64_t n, int c, double alpha, const Segs& A,
                       const double* B, int64_t ldb, double beta, double* C,
                       int64_t ldc, cudaStream_t st);

// eq. tol residuals for w columns; part >= residual_ws_elems(n, w);
// counter: one zero-initialised word owned by the caller.
size_t residual_ws_elems(int64_t n, int w);
// BX, BY (optional): B X, B Y of the generalized LREP for the lam terms
// (K X - lam B Y, M Y - lam B X); the denominator keeps ||[Y; X]||.
cudaError_t residuals_f64(int64_t n, int w, const double* X, const double* Y,
                          const double* KX, const double* MY, int64_t ld,
                          const double* lam, double* eps, double* part,
                          unsigned int* counter, cudaStream_t st,
                          const double* BX = nullptr, const double* BY = nullptr);

// out[:, b] = s1[b] * P1[:, idx[b]] + s2 * P2[:, idx[b]] + (P3 ? s3[b] * P3[:, b] : 0)
cudaError_t gather_combine(int64_t n, int nb, const int* idx, const double* s1,
                           const double* P1, double s2, const double* P2,
                           const double* s3, const double* P3, int64_t ld_in,
                           double* out, int64_t ld_out, cudaStream_t st);

// squared 2-norms of c columns into out[c]; part >= colnorm_ws_elems(n, c)
size_t colnorm_ws_elems(int64_t n, int c);
cudaError_t colnorm2_f64(int64_t n, int c, const double* A, int64_t lda,
                         double* out, double* part, unsigned int* counter,
                         cudaStream_t st);

// V0 normalisation helper (one thread): Cholesky G = L L^T of an r x r SPD
// matrix and Cinv = L^-T (upper), so that X C^-1 = X Cinv (eq. V0_basis).
cudaError_t chol_upper_inverse(int r, const double* G, int ldg, double* Cinv,
                               int ldc, double* work, int* info, cudaStream_t st);

// copy c columns (n rows) between column-major blocks
cudaError_t copy_cols(int64_t n, int c, const double* src, int64_t lds,
                      double* dst, int64_t ldd, cudaStream_t st);

// x_i, y_i scaled by the sign of the largest-|.| entry of x_i (ties: first)
cudaError_t fix_sign(int64_t n, int c, double* X, double* Y, int64_t ld,
                     cudaStream_t st);

// u = y + x, v = y - x
cudaError_t uv_from_xy(int64_t n, int c, const double* X, const double* Y,
                       int64_t ld, double* U, double* V, int64_t ldo,
                       cudaStream_t st);

// K = A - B, M = A + B in place of (A, B) (n x n, ld)
cudaError_t km_from_ab(int64_t n, double* A, double* B, int64_t ld, cudaStream_t st);

// Philox4x32-10 normals (see lrep_ops.h)
cudaError_t philox_normal(int64_t n, int c, uint64_t seed, int stream_id,
                          double* out, int64_t ld, cudaStream_t st);

// ------------------------------------------------------------------ CG
struct CgState {  // device arrays of length nb (+ counters)
  double* rho;    // current r^T r
  double* stop;   // tol^2 * ||b||^2
  double* alpha;
  double* beta;
  int* active;
  int* done;      // all columns converged
  double* part;   // partials: nb * slabs
  unsigned int* counter;  // 128 counters, zero-initialised
  int* iters;     // iterations with an active column (device counter)
  int slabs;
};
size_t cg_part_elems(int64_t n, int nb);
cudaError_t cg_init(int64_t n, int nb, const double* B, int64_t ldb, double* X,
                    double* R, double* P, int64_t ld, double tol, CgState& s,
                    cudaStream_t st);
cudaError_t cg_alpha(int64_t n, int nb, const double* P, const double* Q,
                     int64_t ld, CgState& s, cudaStream_t st);
cudaError_t cg_update(int64_t n, int nb, double* X, double* R, const double* P,
                      const double* Q, int64_t ld, CgState& s, cudaStream_t st);
cudaError_t cg_pdir(int64_t n, int nb, const double* R, double* P, int64_t ld,
                    CgState& s, cudaStream_t st);
// Fused steps of the CG on the bf16 hi/lo tensor-core operator:
// cg_sum_alpha forms Q from the product's split-K partials (fp32,
// part[(z * nb + j) * n + i], summed over z in order in fp32) and then
// computes alpha as cg_alpha; cg_pdir_split is cg_pdir that also writes
// the new directions' bf16 hi/lo split (taken from their fp32 rounding;
// the next product's operand, leading dimension ldb).
cudaError_t cg_sum_alpha(int64_t n, int nb, const float* part, int splits, const double* P,
                         double* Q, int64_t ld, CgState& s, cudaStream_t st);
cudaError_t cg_pdir_split(int64_t n, int nb, const double* R, double* P, int64_t ld,
                          CgState& s, void* hi, void* lo, int64_t ldb, cudaStream_t st);
// The three fused steps above in one cooperative launch (per-column
// barriers for the two reductions of a CG step), when n, nb fit it
// (cg_step_coop_fits: slabs of at most 2048 rows, nb <= 120, every CTA
// co-resident).  CgState.counter[8 .. 8 + nb) are the column barrier
// counters: zero at the start of a CG solve, epoch = the solve's step
// index.  A barrier that does not complete within ~2 s sets *err to 6.
bool cg_step_coop_fits(int64_t n, int nb, const CgState& s);
cudaError_t cg_step_coop(int64_t n, int nb, const float* part, int splits, double* X,
                         double* R, double* P, int64_t ld, CgState& s, void* hi, void* lo,
                         int64_t ldb, int epoch, int* err, cudaStream_t st);

// ------------------------------------------------------------ small (1 CTA)
// Small LREP of order d (batched: one CTA per problem).  Per problem:
struct SmallJob {
  const double* Khat; const double* Mhat; int ld_in;
  const double* S;      // optional U^T V (d x d, ld_in) for the biorth check
  double* lam; double* Xh; double* Yh; int ldo;
  double* work;         // 4 * d * d doubles
  int* info;            // 0 ok, 1 K^ not SPD, 2 M^ not SPD, 3 no SVD conv.
  double* biorth_err;   // max |S - I| (when S given)
  int d;
  int w_prev;           // sign alignment of pairs j < w_prev (reading)
  int* sweeps = nullptr; // optional: Jacobi sweeps used
};
size_t small_work_elems(int d);
cudaError_t small_lrep_batched(const SmallJob* jobs_dev, int njobs, cudaStream_t st);
cudaError_t small_lrep_one(const SmallJob& job, cudaStream_t st);
// small_lrep_one spreads orders d >= this over the grid (FP64 refinement as
// multi-CTA products); below it, one CTA (as in small_lrep_batched)
int small_wide_min();

// eq. hat_pq + small Alg. 1 (one CTA).
struct PqJob {
  const double* Xh; const double* Yh; int ld;   // d x d Ritz coefficients
  int d, end, w_prev, na;
  const int* act;        // na Ritz indices (device)
  double* Ph; double* Qh; int ldo;  // d x na out, compacted to p columns
  double* work;          // 4 * d * na doubles
  int* count;            // p
  double tau;
};
size_t pq_work_elems(int d, int na);
cudaError_t small_pq(const PqJob& job, cudaStream_t st);

// Alg. 1 in coefficient space from the Gram G2 = [W Z]^T [W Z] (2m x 2m,
// ld2): writes A, B (m x m, ldc; first `count` columns valid) so that
// P = W A, Q = Z B are biorthogonal.  ref_w, ref_z: entering norms
// (nullptr: sqrt(diag)).  near_identity: W^T Z is known to be close to I
// (a pass over an already biorthogonal basis), which allows the parallel
// LU form.
size_t biorth_coef_work_elems(int m);
cudaError_t biorth_coef(int m, const double* G2, int ld2, const double* ref_w2,
                        const double* ref_z2, double tau, double* A, double* B,
                        int ldc, double* work, int* count, cudaStream_t st,
                        bool near_identity = false);

// max |S - I| of a d x d matrix into *out (one CTA)
cudaError_t biorth_error(int d, const double* S, int lds, double* out, cudaStream_t st);

}  // namespace lrep
