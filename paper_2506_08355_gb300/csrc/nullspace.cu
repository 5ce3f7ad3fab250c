// Pre-step of Alg. 2 for singular K: an orthonormal basis X0 of N(K)
// (Remark on the numerical computation of the generalized nullspace: the
// zero eigenvectors of the symmetric K by a symmetric eigensolver; Y0 then
// follows from M Y0 = X0 by CG inside the solve).
//
// Eigensolver: block LOBPCG on K for its m = r_max + 4 smallest eigenpairs,
// every step on the GPU with the solver's kernels:
//   R = K X - X diag(theta)          residuals, column norms
//   B = [R_act / |R_act|, P]         active residuals (unit) and directions,
//                                    projected off X twice, CholQR2
//   S = [X, B], T = S^T (K S)        Gram of the float64 operator products
//   T + tau I = Z diag(lam^2) Z^T    the small LREP kernel with M^ = I
//                                    (K^ x = lam y, y = lam x: K^ x = lam^2 x)
//   X = S Z, K X = (K S) Z, P = B Z_B
// ||K||_2 is estimated by 30 power steps.  With tol: a Ritz pair counts as a
// null vector when theta <= sqrt(tol) ||K|| and its residual <= tol ||K||;
// the search stops when all candidates are converged and the next Ritz value
// is certainly non-zero (residual <= theta / 100 and theta - residual >
// sqrt(tol) ||K||), so nonzero eigenvalues below ~sqrt(tol) ||K|| are not
// resolved.  Unpreconditioned: the iteration count grows like
// sqrt(||K|| / lambda_min+).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/lrep.h"
#include "kernels.h"
#include "problem.h"

namespace lrep {
namespace {

__global__ void ns_residual_kernel(int64_t n, int m, const double* __restrict__ X,
                                   const double* __restrict__ KX, const double* __restrict__ th,
                                   double* __restrict__ R, int64_t ld) {
  const int64_t tot = n * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / n, i = e % n;
    R[i + j * ld] = KX[i + j * ld] - th[j] * X[i + j * ld];
  }
}

// Kh = (T + T^T) / 2 + tau I, Mh = I (d x d, ld)
__global__ void ns_small_setup_kernel(int d, const double* __restrict__ T, int ld, double tau,
                                      double* __restrict__ Kh, double* __restrict__ Mh) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d * d; e += gridDim.x * blockDim.x) {
    const int i = e % d, j = e / d;
    Kh[i + j * ld] = 0.5 * (T[i + j * ld] + T[j + i * ld]) + (i == j ? tau : 0.0);
    Mh[i + j * ld] = (i == j) ? 1.0 : 0.0;
  }
}

// Z[:, j] = Xh[:, j] sqrt(lam_j) (unit eigenvectors of T), theta_j = lam_j^2 - tau
__global__ void ns_ritz_kernel(int d, int m, const double* __restrict__ Xh, int ld,
                               const double* __restrict__ lam, double tau,
                               double* __restrict__ Z, double* __restrict__ th) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d * m; e += gridDim.x * blockDim.x) {
    const int i = e % d, j = e / d;
    Z[i + j * ld] = Xh[i + j * ld] * sqrt(lam[j]);
    if (i == 0) th[j] = lam[j] * lam[j] - tau;
  }
}

// dst[:, q] = src[:, idx[q]]
__global__ void ns_gather_kernel(int64_t n, int c, const int* __restrict__ idx,
                                 const double* __restrict__ src, double* __restrict__ dst,
                                 int64_t ld) {
  const int64_t tot = n * c;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = e / n, i = e % n;
    dst[i + q * ld] = src[i + (int64_t)idx[q] * ld];
  }
}

// v = w / sqrt(nrm2[0])
__global__ void ns_scale_kernel(int64_t n, const double* __restrict__ w,
                                const double* __restrict__ nrm2, double* __restrict__ v) {
  const double s = nrm2[0] > 0.0 ? 1.0 / sqrt(nrm2[0]) : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = w[i] * s;
}

unsigned grid_for(int64_t tot) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((tot + 255) / 256, 8 * kNumSMs));
}

#define NCK(expr)                                                                        \
  do {                                                                                   \
    cudaError_t _e = (expr);                                                             \
    if (_e != cudaSuccess)                                                               \
      return p->fail(LREP_ERR_CUDA, std::string("nullspace: ") + #expr + ": " +          \
                                        cudaGetErrorString(_e));                         \
  } while (0)
#define NST(expr)                  \
  do {                             \
    lrep_status _s = (expr);       \
    if (_s != LREP_OK) return _s;  \
  } while (0)

struct NullFinder {
  lrep_problem p;
  cudaStream_t st;
  int64_t n, ld;
  int m, mm;
  Arena A;
  double *X, *KX, *R, *Ra, *P, *B, *S, *KS, *tmp, *v, *w;
  double *T, *Kh, *Mh, *Xh, *Yh, *lam, *swork, *Z, *G, *Rinv, *Rwork, *th, *nrm2, *scale;
  double *ws, *part, *berr;
  int *info, *idx;
  unsigned int* counters;
  size_t ws_elems = 0, part_elems = 0;

  void layout(Arena& a) {
    X = a.take<double>(ld * m); KX = a.take<double>(ld * m); R = a.take<double>(ld * m);
    Ra = a.take<double>(ld * m); P = a.take<double>(ld * m);
    B = a.take<double>(ld * 2 * m); tmp = a.take<double>(ld * 3 * m);
    S = a.take<double>(ld * 3 * m); KS = a.take<double>(ld * 3 * m);
    v = a.take<double>(ld); w = a.take<double>(ld);
    T = a.take<double>(mm * mm); Kh = a.take<double>(mm * mm); Mh = a.take<double>(mm * mm);
    Xh = a.take<double>(mm * mm); Yh = a.take<double>(mm * mm); Z = a.take<double>(mm * mm);
    lam = a.take<double>(mm); swork = a.take<double>(small_work_elems(mm));
    G = a.take<double>(4 * m * m); Rinv = a.take<double>(4 * m * m);
    Rwork = a.take<double>(4 * m * m); th = a.take<double>(mm); nrm2 = a.take<double>(mm);
    scale = a.take<double>(mm); berr = a.take<double>(8);
    ws = a.take<double>(std::max<size_t>(ws_elems, 1));
    part = a.take<double>(std::max<size_t>(part_elems, 1));
    info = a.take<int>(64); idx = a.take<int>(mm); counters = a.take<unsigned int>(64);
  }

  lrep_status alloc() {
    ld = ((n + 31) / 32) * 32;
    size_t wsz = gram_ws_elems(n, mm, mm);
    wsz = std::max(wsz, gram_ws_elems(n, m, 2 * m));
    wsz = std::max(wsz, apply_ws_elems(p, mm));
    ws_elems = wsz;
    part_elems = colnorm_ws_elems(n, mm);
    Arena dry;
    dry.cap = ~(size_t)0;
    layout(dry);
    NCK(A.reserve(dry.off + 4096, st));
    A.off = 0;
    layout(A);
    return LREP_OK;
  }

  lrep_status apply(int c, const double* in, double* out) {
    return apply_op(p, LREP_OP_K, c, in, ld, out, ld, nullptr, ws, ws_elems);
  }
  lrep_status gram(const double* a, int ca, const double* b, int cb, double* g) {
    NCK(gram_f64_capped(n, seg1(a, ld, ca), seg1(b, ld, cb), g, ca, ws, ws_elems, st));
    return LREP_OK;
  }
  // out = a (n x k) * coef (k x c, ldc) (+ beta out)
  lrep_status mul(const double* a, int k, const double* coef, int ldc, int c, double* out,
                  double alpha = 0.0, double beta = 1.0) {
    NCK(update_f64(n, c, alpha, seg1(a, ld, k), coef, ldc, beta, out, ld, st));
    return LREP_OK;
  }
  lrep_status norms(const double* a, int c, double* out) {
    NCK(cudaMemsetAsync(counters, 0, 64 * sizeof(unsigned int), st));
    NCK(colnorm2_f64(n, c, a, ld, out, part, counters, st));
    return LREP_OK;
  }
  // two passes of Cholesky QR on c columns of Q; info[slot] != 0 on failure
  lrep_status cholqr2(double* Q, int c, int slot) {
    for (int pass = 0; pass < 2; ++pass) {
      NST(gram(Q, c, Q, c, G));
      NCK(chol_upper_inverse(c, G, c, Rinv, c, Rwork, info + slot + pass, st));
      NST(mul(Q, c, Rinv, c, c, tmp));
      NCK(copy_cols(n, c, tmp, ld, Q, ld, st));
    }
    return LREP_OK;
  }
  // Ritz pairs of span(S) (d columns, K S given): Z (d x m), theta (m)
  lrep_status ritz(int d, double tau) {
    NST(gram(S, d, KS, d, T));  // T[i,j] = s_i^T (K s_j), ld = d
    ns_small_setup_kernel<<<grid_for((int64_t)d * d), 256, 0, st>>>(d, T, d, tau, Kh, Mh);
    LREP_COUNT_LAUNCH();
    NCK(cudaGetLastError());
    SmallJob job{};
    job.Khat = Kh; job.Mhat = Mh; job.ld_in = d; job.S = nullptr;
    job.lam = lam; job.Xh = Xh; job.Yh = Yh; job.ldo = d;
    job.work = swork; job.info = info + 8; job.biorth_err = berr;
    job.d = d; job.w_prev = 0;
    NCK(small_lrep_one(job, st));
    ns_ritz_kernel<<<grid_for((int64_t)d * m), 256, 0, st>>>(d, m, Xh, d, lam, tau, Z, th);
    LREP_COUNT_LAUNCH();
    NCK(cudaGetLastError());
    return LREP_OK;
  }

  lrep_status run(int maxit, double tol, int* r_out, int* iters_out) {
    // ||K||_2 by power steps
    NCK(philox_normal(n, 1, p->opts.seed, 3, v, ld, st));
    for (int it = 0; it < 30; ++it) {
      NST(apply(1, v, w));
      NST(norms(w, 1, nrm2));
      ns_scale_kernel<<<grid_for(n), 256, 0, st>>>(n, w, nrm2, v);
      LREP_COUNT_LAUNCH();
      NCK(cudaGetLastError());
    }
    double h2 = 0.0;
    NCK(cudaMemcpyAsync(&h2, nrm2, sizeof(double), cudaMemcpyDeviceToHost, st));
    NCK(cudaStreamSynchronize(st));
    const double nrm = std::sqrt(h2);
    if (!(nrm > 0.0)) {  // K = 0: everything is kernel
      return p->fail(LREP_ERR_ARG, "nullspace: K is zero (every vector is a null vector)");
    }
    const double tau = 1e-2 * nrm, zero = std::sqrt(tol) * nrm;
    // start: Philox block, orthonormalised, Rayleigh-Ritz on it
    NCK(philox_normal(n, m, p->opts.seed, 2, X, ld, st));
    NCK(cudaMemsetAsync(info, 0, 64 * sizeof(int), st));
    NST(cholqr2(X, m, 0));
    NCK(copy_cols(n, m, X, ld, S, ld, st));
    NST(apply(m, S, KS));
    NST(ritz(m, tau));
    NST(mul(S, m, Z, m, m, X));
    NST(mul(KS, m, Z, m, m, KX));
    std::vector<double> hth(m), hr2(m), hscale(2 * m);
    std::vector<int> hinfo(16), hact;
    int np = 0;  // columns of P
    for (int it = 0; it < maxit; ++it) {
      ns_residual_kernel<<<grid_for(n * m), 256, 0, st>>>(n, m, X, KX, th, R, ld);
      LREP_COUNT_LAUNCH();
      NCK(cudaGetLastError());
      NST(norms(R, m, nrm2));
      NCK(cudaMemcpyAsync(hth.data(), th, m * sizeof(double), cudaMemcpyDeviceToHost, st));
      NCK(cudaMemcpyAsync(hr2.data(), nrm2, m * sizeof(double), cudaMemcpyDeviceToHost, st));
      NCK(cudaMemcpyAsync(hinfo.data(), info, 16 * sizeof(int), cudaMemcpyDeviceToHost, st));
      NCK(cudaStreamSynchronize(st));
      if (it == 0 && (hinfo[0] || hinfo[1]))
        return p->fail(LREP_ERR_BREAKDOWN, "nullspace: start block lost rank");
      // info 3 (rotation refinement not converged) comes from the cluster of
      // Ritz values at zero, where any basis of the cluster will do; the
      // stop test below checks the vectors through their own residuals
      if (hinfo[8] == 1 || hinfo[8] == 2)
        return p->fail(LREP_ERR_BREAKDOWN, "nullspace: Ritz problem failed (info " +
                                               std::to_string(hinfo[8]) + ")");
      for (int j = 0; j < m; ++j)
        if (!std::isfinite(hth[j]) || !std::isfinite(hr2[j]))
          return p->fail(LREP_ERR_BREAKDOWN, "nullspace: non-finite Ritz value or residual");
      int cand = 0;
      while (cand < m && hth[cand] <= zero) ++cand;
      bool conv = cand < m;
      for (int j = 0; j < cand && conv; ++j) conv = std::sqrt(hr2[j]) <= tol * nrm;
      if (conv) {
        const double rg = std::sqrt(hr2[cand]);
        conv = rg <= 1e-2 * hth[cand] && hth[cand] - rg > zero;
      }
      if (conv) {
        *r_out = cand;
        *iters_out = it;
        return LREP_OK;
      }
      if (cand == m) {
        bool all = true;
        for (int j = 0; j < m && all; ++j) all = std::sqrt(hr2[j]) <= tol * nrm;
        if (all)
          return p->fail(LREP_ERR_ARG, "nullspace: dimension exceeds r_max (raise r_max)");
      }
      // active residual columns, unit length
      hact.clear();
      for (int j = 0; j < m; ++j)
        if (std::sqrt(hr2[j]) > 0.1 * tol * nrm) {
          hact.push_back(j);
          hscale[hact.size() - 1] = 1.0 / std::sqrt(hr2[j]);
        }
      const int na = (int)hact.size();
      if (na == 0) continue;
      NCK(cudaMemcpyAsync(idx, hact.data(), na * sizeof(int), cudaMemcpyHostToDevice, st));
      NCK(cudaMemcpyAsync(scale, hscale.data(), na * sizeof(double), cudaMemcpyHostToDevice, st));
      NCK(gather_combine(n, na, idx, scale, R, 0.0, R, nullptr, nullptr, ld, Ra, ld, st));
      NCK(copy_cols(n, na, Ra, ld, B, ld, st));  // B = [R_act | P]
      int nbk = na + np;
      if (np > 0) NCK(copy_cols(n, np, P, ld, B + ld * (int64_t)na, ld, st));
      for (int attempt = 0; attempt < 2; ++attempt) {
        for (int pass = 0; pass < 2; ++pass) {  // B -= X (X^T B)
          NST(gram(X, m, B, nbk, G));
          NST(mul(X, m, G, m, nbk, B, 1.0, -1.0));
        }
        NCK(cudaMemsetAsync(info, 0, 4 * sizeof(int), st));
        NST(cholqr2(B, nbk, 0));
        NCK(cudaMemcpyAsync(hinfo.data(), info, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
        NCK(cudaStreamSynchronize(st));
        if (!hinfo[0] && !hinfo[1]) break;
        if (attempt == 1 || np == 0)
          return p->fail(LREP_ERR_BREAKDOWN, "nullspace: search block lost rank");
        // drop the directions and retry with the residuals alone
        np = 0;
        nbk = na;
        NCK(copy_cols(n, na, Ra, ld, B, ld, st));
      }
      // S = [X | B], K S, Ritz pairs of span(S)
      const int d = m + nbk;
      NCK(copy_cols(n, m, X, ld, S, ld, st));
      NCK(copy_cols(n, nbk, B, ld, S + ld * (int64_t)m, ld, st));
      NST(apply(d, S, KS));
      NST(ritz(d, tau));
      NST(mul(S, d, Z, d, m, X));
      NST(mul(KS, d, Z, d, m, KX));
      // P = B Z_B (rows m..d-1 of Z) for the active columns
      NST(mul(B, nbk, Z + m, d, m, tmp));
      ns_gather_kernel<<<grid_for(n * na), 256, 0, st>>>(n, na, idx, tmp, P, ld);
      LREP_COUNT_LAUNCH();
      NCK(cudaGetLastError());
      np = na;
    }
    return p->fail(LREP_NOT_CONVERGED, "nullspace: LOBPCG did not converge within maxit");
  }
};

}  // namespace

lrep_status find_nullspace(lrep_problem p, int r_max, double tol, int maxit, int* r_out,
                           int* iters_out) {
  NullFinder f{};
  f.p = p;
  f.st = p->stream;
  f.n = p->op.n;
  f.m = r_max + 4;
  f.mm = 3 * f.m;
  if (f.m > f.n) return p->fail(LREP_ERR_ARG, "nullspace: r_max + 4 exceeds n");
  NST(f.alloc());
  int r = 0, its = 0;
  lrep_status s = f.run(maxit, tol, &r, &its);
  if (s == LREP_OK) {
    p->r = r;
    p->X0in = p->Y0in = nullptr;
    if (r > 0) {
      double* dst = nullptr;
      if (cudaMalloc(&dst, sizeof(double) * f.ld * r) != cudaSuccess) {
        f.A.release();
        return p->fail(LREP_ERR_NOMEM, "nullspace: out of device memory");
      }
      p->op.owned.push_back(dst);
      if (copy_cols(f.n, r, f.X, f.ld, dst, f.ld, f.st) != cudaSuccess ||
          cudaStreamSynchronize(f.st) != cudaSuccess) {
        f.A.release();
        return p->fail(LREP_ERR_CUDA, "nullspace: copy of the basis failed");
      }
      p->X0in = dst;
    }
    *r_out = r;
    *iters_out = its;
  }
  f.A.release();
  return s;
}

}  // namespace lrep
