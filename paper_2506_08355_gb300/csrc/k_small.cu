// Small dense steps of one BOSP iteration, one CTA per problem:
//  * the projected LREP of eq. small_eigen by two Cholesky factorisations
//    and one SVD (Section 3.3, cost item 2), the SVD by one-sided
//    (Hestenes) Jacobi with a round-robin pair order;
//  * P^, Q^ of eq. hat_pq followed by Alg. 1 in R^d;
//  * Alg. 1 for a large n x m pair (W, Z) carried out on the Gram
//    matrices of [W Z]: the coefficient vectors a_l, b_l with p_l = W a_l,
//    q_l = Z b_l follow Alg. 1's updates exactly, inner products
//    q_j^T p = (Z b_j)^T W a being read from the Grams.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace lrep {
namespace {

constexpr int SMALL_T = 512;
constexpr int SMALL_MAXD = 256;

__device__ __forceinline__ double block_max(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
    red[0] = t;
  }
  __syncthreads();
  t = red[0];
  __syncthreads();
  return t;
}

// In-place lower Cholesky of a d x d column-major matrix (ld = d); returns
// false (uniformly) when a pivot is not positive and finite.
__device__ bool chol_lower(double* L, int d, int* s_flag) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int j = 0; j < d; ++j) {
    if (tid == 0) {
      const double v = L[j + j * d];
      if (!(v > 0.0) || !isfinite(v)) *s_flag = 1;
      else L[j + j * d] = sqrt(v);
    }
    __syncthreads();
    if (*s_flag) return false;
    const double piv = L[j + j * d];
    for (int i = j + 1 + tid; i < d; i += nt) L[i + j * d] /= piv;
    __syncthreads();
    const int m = d - j - 1;
    for (int e = tid; e < m * m; e += nt) {
      const int ii = e % m, kk = e / m;
      if (ii < kk) continue;
      const int i = j + 1 + ii, k = j + 1 + kk;
      L[i + k * d] -= L[i + j * d] * L[k + j * d];
    }
    __syncthreads();
  }
  for (int e = tid; e < d * d; e += nt) {
    const int i = e % d, k = e / d;
    if (i < k) L[e] = 0.0;
  }
  __syncthreads();
  return true;
}

// ---------------------------------------------------------------- small LREP
// FP64 is scarce on GB300 (about 2 FMA per clock per SM), so the SVD of
// G = L1^T L2 runs in two phases inside the CTA:
//  1. one-sided (Hestenes) Jacobi in FP32 on a copy of G, round-robin pair
//     order, until every column pair's cosine is below 2 sqrt(d) eps_32;
//  2. FP64 refinement of the right factor V by matrix products: two
//     Newton-Schulz steps V <- V - V (V^T V - I)/2, then steps of
//     simultaneous Jacobi rotations B = G V, C = B^T B, t_ab from the 2 x 2
//     problem of columns (a, b), V <- V (I + T - T^T), each followed by three
//     Newton-Schulz steps, until max cos < d eps (quadratic convergence).
// The column products of B keep each pair's rounding relative to
// sigma_a sigma_b, so small singular values keep relative accuracy.
// dyn: dynamic shared memory (dyn_bytes); matrices are column-major with
// leading dimension d.


// C = A * B (+ beta C) for d x d column-major matrices (ld d); C must not
// alias A or B.  transA: use A^T.
__device__ void mm_d(int d, const double* A, bool transA, const double* B, double* C,
                     double alpha, double beta) {
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
    const int i = e % d, j = e / d;
    double s = 0.0;
    if (transA)
      for (int k = 0; k < d; ++k) s = fma(A[k + i * d], B[k + j * d], s);
    else
      for (int k = 0; k < d; ++k) s = fma(A[i + k * d], B[k + j * d], s);
    C[e] = (beta == 0.0) ? alpha * s : fma(alpha, s, beta * C[e]);
  }
  __syncthreads();
}

// Jacobi rotation tangent t of the 2 x 2 problem [[aa, g], [g, bb]] (the
// one-sided Jacobi angle of two columns with squared norms aa, bb and inner
// product g); 0 when g = 0.
__device__ __forceinline__ double pair_rotation(double aa, double bb, double g) {
  if (g == 0.0) return 0.0;
  const double zeta = (bb - aa) / (2.0 * g);
  return (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
}

// Simultaneous first-order rotations (V <- V (I + T - T^T)) are applied only
// where |t| <= kRotCap; larger rotations (relative gap of the pair's singular
// values below ~cos / kRotCap, e.g. a degenerate cluster) are done exactly,
// one pair at a time, after the simultaneous steps.  A first-order step
// leaves V non-orthogonal by O(t^2) <= 2.5e-3, which three Newton-Schulz
// steps take below rounding (2.5e-3 -> ~1e-5 -> ~1.5e-10 -> ~3e-20).
constexpr double kRotCap = 0.05;
constexpr int kMaxPairs = 512;

// Newton-Schulz step: V <- V - V (V^T V - I) / 2, using R and T as scratch.
__device__ void ns_step(int d, double*& V, double*& T, double* R) {
  mm_d(d, V, true, V, R, 1.0, 0.0);
  for (int i = threadIdx.x; i < d; i += blockDim.x) R[i + i * d] -= 1.0;
  __syncthreads();
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) T[e] = V[e];
  __syncthreads();
  mm_d(d, V, false, R, T, -0.5, 1.0);
  double* t = V; V = T; T = t;
}

// Where the d x d matrices of one small LREP live: L1, L2 in the job's work
// array; G, V, B, S in dynamic shared memory when 4 d^2 doubles fit, else in
// the work array too; the FP32 copies of phase 1 alias B and S.
struct SmallMats {
  double *L1, *L2, *G, *V, *B, *S;
  float *G32, *V32;
};

__device__ SmallMats small_place(const SmallJob& J, double* dyn, int dyn_bytes) {
  const size_t dd = (size_t)J.d * J.d;
  SmallMats m;
  m.L1 = J.work;
  m.L2 = J.work + dd;
  if (4 * dd * sizeof(double) <= (size_t)dyn_bytes) {
    m.G = dyn; m.V = dyn + dd; m.B = dyn + 2 * dd; m.S = dyn + 3 * dd;
    m.G32 = reinterpret_cast<float*>(m.B);
    m.V32 = reinterpret_cast<float*>(m.S);
  } else {
    m.G = J.work + 2 * dd; m.V = J.work + 3 * dd; m.B = J.work + 4 * dd; m.S = J.work + 5 * dd;
    // phase 1 still runs in shared memory when its FP32 copies fit
    const bool fit32 = 2 * dd * sizeof(float) <= (size_t)dyn_bytes;
    m.G32 = fit32 ? reinterpret_cast<float*>(dyn) : reinterpret_cast<float*>(m.B);
    m.V32 = fit32 ? reinterpret_cast<float*>(dyn) + dd : reinterpret_cast<float*>(m.S);
  }
  return m;
}

// Phase 1 of the small LREP (biorthogonality check of S, K^ = L1 L1^T,
// M^ = L2 L2^T, G = L1^T L2, FP32 one-sided Jacobi of G) leaving G in
// FP64 and the FP32 right factor in m.V32.  Returns false (info 1 or 2
// written) when a Cholesky factor fails.
__device__ bool small_phase1(const SmallJob& J, const SmallMats& mm, int* sweeps_out) {
  const int d = J.d;
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ int s_flag;
  __shared__ int s_conv;
  __shared__ double red[32];
  double* L1 = mm.L1;
  double* L2 = mm.L2;
  double* G = mm.G;
  float* G32 = mm.G32;
  float* V32 = mm.V32;
  if (tid == 0) s_flag = 0;
  // biorthogonality of the current basis (safeguard input)
  if (J.S) {
    double m = 0.0;
    for (int e = tid; e < d * d; e += nt) {
      const int i = e % d, j = e / d;
      m = fmax(m, fabs(J.S[i + (size_t)j * J.ld_in] - (i == j ? 1.0 : 0.0)));
    }
    m = block_max(m, red);
    if (tid == 0) *J.biorth_err = m;
  }
  for (int e = tid; e < d * d; e += nt) {
    const int i = e % d, j = e / d;
    L1[e] = 0.5 * (J.Khat[i + (size_t)j * J.ld_in] + J.Khat[j + (size_t)i * J.ld_in]);
    L2[e] = 0.5 * (J.Mhat[i + (size_t)j * J.ld_in] + J.Mhat[j + (size_t)i * J.ld_in]);
  }
  __syncthreads();
  if (!chol_lower(L1, d, &s_flag)) {
    if (tid == 0) *J.info = 1;
    return false;
  }
  if (!chol_lower(L2, d, &s_flag)) {
    if (tid == 0) *J.info = 2;
    return false;
  }
  // G = L1^T L2 (both lower triangular)
  for (int e = tid; e < d * d; e += nt) {
    const int i = e % d, j = e / d;
    double s = 0.0;
    for (int k = max(i, j); k < d; ++k) s = fma(L1[k + i * d], L2[k + j * d], s);
    G[e] = s;
    G32[e] = (float)s;
    V32[e] = (i == j) ? 1.0f : 0.0f;
  }
  __syncthreads();
  // ---- phase 1: FP32 one-sided Jacobi
  const int dp = d + (d & 1), m = dp - 1;
  const float tol32 = 2.0f * sqrtf((float)d) * 1.1920929e-7f;
  const int npairs = dp / 2;
  int gsz = 32;
  while (gsz > 16 && npairs > nt / gsz) gsz >>= 1;
  const int ngroups = nt / gsz, gid = tid / gsz, glane = tid % gsz;
  const int warp_gid0 = (tid >> 5) * (32 / gsz);  // first group of this warp
  int sweeps = 0;
  for (int sweep = 0; sweep < 30; ++sweep) {
    ++sweeps;
    if (tid == 0) s_conv = 1;
    __syncthreads();
    for (int r = 0; r < m; ++r) {
      // the pairs of the round in lane groups of gsz lanes (16 or 32: one
      // group per pair when they fit); every lane of a working warp runs the
      // same trip count (inactive groups idle through the shuffles)
      for (int base = 0; base < npairs; base += ngroups) {
        // warps whose groups all lie past the last pair skip the round (the
        // shuffles below stay within a warp); the kernel is issue-bound
        if (base + warp_gid0 >= npairs) continue;
        const int p = base + gid;
        int a = 0, b = 0;
        if (p < npairs) {
          if (p == 0) {
            a = r;
            b = m;
          } else {  // (r + p) mod m and (r - p) mod m for 0 <= r < m, 0 < p < m
            a = r + p;
            if (a >= m) a -= m;
            b = r - p;
            if (b < 0) b += m;
          }
          if (a > b) { const int t = a; a = b; b = t; }
        }
        const bool live = p < npairs && b < d;
        float al = 0.f, be = 0.f, ga = 0.f;
        if (live)
          for (int i = glane; i < d; i += gsz) {
            const float x = G32[i + a * d], y = G32[i + b * d];
            al = fmaf(x, x, al); be = fmaf(y, y, be); ga = fmaf(x, y, ga);
          }
        for (int o = gsz >> 1; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        if (live && fabsf(ga) > tol32 * sqrtf(al * be)) {
          const float zeta = (be - al) / (2.0f * ga);
          const float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
          const float c = rsqrtf(1.f + t * t), s = c * t;
          for (int i = glane; i < d; i += gsz) {
            const float x = G32[i + a * d], y = G32[i + b * d];
            G32[i + a * d] = c * x - s * y;
            G32[i + b * d] = s * x + c * y;
            const float u = V32[i + a * d], v = V32[i + b * d];
            V32[i + a * d] = c * u - s * v;
            V32[i + b * d] = s * u + c * v;
          }
          if (glane == 0) s_conv = 0;
        }
      }
      __syncthreads();
    }
    const int conv = s_conv;
    __syncthreads();
    if (conv) break;
  }
  *sweeps_out = sweeps;
  return true;
}

__device__ void small_lrep_body(const SmallJob& J, double* dyn, int dyn_bytes) {
  const int d = J.d;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  __shared__ double red[32];
  __shared__ double sig[SMALL_MAXD];
  __shared__ int perm[SMALL_MAXD];
  __shared__ int flip[SMALL_MAXD];
  __shared__ int s_npairs, s_rot;
  __shared__ unsigned char pa[kMaxPairs], pb[kMaxPairs];
  const SmallMats mm = small_place(J, dyn, dyn_bytes);
  double* L1 = mm.L1;
  double* L2 = mm.L2;
  double* G = mm.G;
  double* V = mm.V;
  double* B = mm.B;
  double* S = mm.S;
  const float* V32 = mm.V32;
  int sweeps = 0;
  if (!small_phase1(J, mm, &sweeps)) return;
  // ---- phase 2: FP64 refinement of V
  for (int e = tid; e < d * d; e += nt) V[e] = (double)V32[e];
  __syncthreads();
  ns_step(d, V, B, S);
  ns_step(d, V, B, S);
  const double tol = (double)d * 2.220446049250313e-16;
  int converged = 0;
  for (int it = 0; it < 6; ++it) {
    mm_d(d, G, false, V, B, 1.0, 0.0);            // B = G V
    // S = B^T B (upper part), then rotation parameters in place (upper)
    double cmax = 0.0;
    for (int e = tid; e < d * d; e += nt) {
      const int i = e % d, j = e / d;
      if (i > j) continue;
      double s = 0.0;
      for (int k = 0; k < d; ++k) s = fma(B[k + i * d], B[k + j * d], s);
      S[e] = s;
    }
    if (tid == 0) s_npairs = 0;
    __syncthreads();
    // pairs whose 2 x 2 rotation is large (nearly equal singular values) are
    // left to the exact sequential pass below and kept out of cmax
    for (int e = tid; e < d * d; e += nt) {
      const int i = e % d, j = e / d;
      if (i >= j) continue;
      const double aa = S[i + i * d], bb = S[j + j * d], g = S[e];
      if (fabs(pair_rotation(aa, bb, g)) > kRotCap) {
        const int q = atomicAdd(&s_npairs, 1);
        if (q < kMaxPairs) { pa[q] = (unsigned char)i; pb[q] = (unsigned char)j; }
      } else {
        cmax = fmax(cmax, fabs(g) / sqrt(aa * bb));
      }
    }
    cmax = block_max(cmax, red);
    if (cmax <= tol) {
      converged = 1;
      break;
    }
    // Omega = T - T^T into the lower/upper of S (diagonal 0)
    for (int e = tid; e < d * d; e += nt) {
      const int i = e % d, j = e / d;
      if (i >= j) continue;
      const double aa = S[i + i * d], bb = S[j + j * d], g = S[e];
      double t = pair_rotation(aa, bb, g);
      if (fabs(t) > kRotCap) t = 0.0;
      S[e] = t;  // upper: +t
      S[j + i * d] = -t;  // lower: -t (distinct element, no race)
    }
    __syncthreads();  // the diagonal is still read above
    for (int i = tid; i < d; i += nt) S[i + i * d] = 0.0;
    __syncthreads();
    for (int e = tid; e < d * d; e += nt) B[e] = V[e];
    __syncthreads();
    mm_d(d, V, false, S, B, 1.0, 1.0);            // B = V + V Omega
    { double* t = V; V = B; B = t; }
    ns_step(d, V, B, S);
    ns_step(d, V, B, S);
    ns_step(d, V, B, S);
  }
  if (!converged) mm_d(d, G, false, V, B, 1.0, 0.0);
  // exact FP64 rotations of the nearly degenerate pairs (one warp, in order)
  const int np = min(s_npairs, kMaxPairs);
  if (np > 0) {
    int left = 1;
    for (int sw = 0; sw < 10 && left; ++sw) {
      if (tid == 0) s_rot = 0;
      __syncthreads();
      if (wid == 0) {
        for (int q = 0; q < np; ++q) {
          const int a = pa[q], b = pb[q];
          double al = 0.0, be = 0.0, ga = 0.0;
          for (int i = lane; i < d; i += 32) {
            const double x = B[i + a * d], y = B[i + b * d];
            al = fma(x, x, al); be = fma(y, y, be); ga = fma(x, y, ga);
          }
          al = warp_sum(al); be = warp_sum(be); ga = warp_sum(ga);
          if (fabs(ga) > tol * sqrt(al * be)) {
            const double t = pair_rotation(al, be, ga);
            const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
            for (int i = lane; i < d; i += 32) {
              const double x = B[i + a * d], y = B[i + b * d];
              B[i + a * d] = c * x - sn * y;
              B[i + b * d] = sn * x + c * y;
              const double u = V[i + a * d], v = V[i + b * d];
              V[i + a * d] = c * u - sn * v;
              V[i + b * d] = sn * u + c * v;
            }
            if (lane == 0) s_rot = 1;
          }
          __syncwarp();
        }
      }
      __syncthreads();
      left = s_rot;
      __syncthreads();  // every thread has read s_rot before it is reset
    }
    converged = converged && !left && s_npairs <= kMaxPairs;
  }
  // singular values (column norms of B = G V), ascending order (ties by index)
  for (int j = wid; j < d; j += nw) {
    double s = 0.0;
    for (int i = lane; i < d; i += 32) s = fma(B[i + j * d], B[i + j * d], s);
    s = warp_sum(s);
    if (lane == 0) sig[j] = sqrt(s);
  }
  __syncthreads();
  for (int j = tid; j < d; j += nt) {
    int rk = 0;
    for (int k = 0; k < d; ++k) rk += (sig[k] < sig[j]) || (sig[k] == sig[j] && k < j);
    perm[rk] = j;
  }
  __syncthreads();
  // X^ = L2 V S^-1/2,  Y^ = L1 W S^-1/2 with W = B / S
  for (int e = tid; e < d * d; e += nt) {
    const int r = e % d, i = e / d;
    const int j = perm[i];
    const double s = sig[j];
    double x = 0.0, y = 0.0;
    for (int k = 0; k <= r; ++k) {
      x = fma(L2[r + k * d], V[k + j * d], x);
      y = fma(L1[r + k * d], B[k + j * d], y);
    }
    J.Xh[r + (size_t)i * J.ldo] = x / sqrt(s);
    J.Yh[r + (size_t)i * J.ldo] = y / (s * sqrt(s));
  }
  for (int i = tid; i < d; i += nt) J.lam[i] = sig[perm[i]];
  __syncthreads();
  // sign of each Ritz pair follows its previous iterate (X^[j, j] >= 0)
  const int wa = min(J.w_prev, d);
  for (int j = tid; j < d; j += nt) flip[j] = (j < wa) && (J.Xh[j + (size_t)j * J.ldo] < 0.0);
  __syncthreads();
  for (int e = tid; e < d * d; e += nt) {
    const int r = e % d, i = e / d;
    if (flip[i]) {
      J.Xh[r + (size_t)i * J.ldo] = -J.Xh[r + (size_t)i * J.ldo];
      J.Yh[r + (size_t)i * J.ldo] = -J.Yh[r + (size_t)i * J.ldo];
    }
  }
  if (tid == 0) {
    *J.info = converged ? 0 : 3;
    if (J.sweeps) *J.sweeps = sweeps;
  }
}

__global__ void __launch_bounds__(SMALL_T) small_lrep_kernel(const SmallJob* __restrict__ jobs,
                                                             int dyn_bytes) {
  extern __shared__ double dyn[];
  const SmallJob J = jobs[blockIdx.x];
  small_lrep_body(J, dyn, dyn_bytes);
}

__global__ void __launch_bounds__(SMALL_T) small_lrep_one_kernel(SmallJob J, int dyn_bytes) {
  extern __shared__ double dyn[];
  small_lrep_body(J, dyn, dyn_bytes);
}

// ---------------------------------------------------------------- wide path
// One small LREP spread over the GPU (single solves, d >= kWideMin): phase 1
// (Cholesky factors, G, FP32 Jacobi) stays in one CTA; the FP64 refinement
// of V and the Ritz coefficients run as grid kernels (every d x d product
// over ceil(d/16)^2 CTAs), so the FP64 work uses many SMs instead of one.
// Same arithmetic as the one-CTA path: two Newton-Schulz steps, up to six
// steps of simultaneous rotations (+ three Newton-Schulz steps each), exact
// sequential rotations of the nearly degenerate pairs, then X^, Y^.
// Work layout (doubles, after L1, L2): G, V, T, R, B, S (d^2 each), then the
// control block.
struct WideCtl {
  unsigned long long cmax[8];  // max cos per rotation step (double bits)
  int fail;                    // Cholesky failed: every later kernel returns
  int stop;                    // fail or converged: refinement kernels return
  int conv;                    // rotation steps converged
  int npairs;                  // nearly degenerate pairs of the last step
  int sweeps;
  unsigned char pa[kMaxPairs], pb[kMaxPairs];
};
constexpr int kWideMin = 40;

struct WideMats {
  double *L1, *L2, *G, *V, *T, *R, *B, *S;
  WideCtl* ctl;
  int* perm;
  double* sig;
};

__host__ __device__ inline WideMats wide_place(double* work, int d) {
  const size_t dd = (size_t)d * d;
  WideMats w;
  w.L1 = work; w.L2 = work + dd; w.G = work + 2 * dd; w.V = work + 3 * dd;
  w.T = work + 4 * dd; w.R = work + 5 * dd; w.B = work + 6 * dd; w.S = work + 7 * dd;
  w.ctl = reinterpret_cast<WideCtl*>(work + 8 * dd);
  w.sig = work + 8 * dd + (sizeof(WideCtl) + 7) / 8;
  w.perm = reinterpret_cast<int*>(w.sig + d);
  return w;
}

// phase 1 is latency bound (one pair rotation per warp per round): twice the
// one-CTA kernel's warps
constexpr int FRONT_T = 1024;

__global__ void __launch_bounds__(FRONT_T) small_front_kernel(SmallJob J, int dyn_bytes) {
  extern __shared__ double dyn[];
  const int d = J.d;
  const WideMats w = wide_place(J.work, d);
  if (threadIdx.x == 0) {
    for (int i = 0; i < 8; ++i) w.ctl->cmax[i] = 0ull;
    w.ctl->fail = 0; w.ctl->stop = 0; w.ctl->conv = 0; w.ctl->npairs = 0;
  }
  // phase 1 with G, V, B, S in shared memory when they fit (B, S hold the
  // FP32 copies), else in the T..S slots of the work array
  // G (FP64) in the work array; the FP32 copies of phase 1 in shared
  // memory when they fit (d <= 166), else in the B, S slots
  SmallMats m;
  const size_t dd = (size_t)d * d;
  m.L1 = w.L1; m.L2 = w.L2; m.G = w.G; m.V = w.V; m.B = w.B; m.S = w.S;
  const bool fit32 = 2 * dd * sizeof(float) <= (size_t)dyn_bytes;
  m.G32 = fit32 ? reinterpret_cast<float*>(dyn) : reinterpret_cast<float*>(w.B);
  m.V32 = fit32 ? reinterpret_cast<float*>(dyn) + dd : reinterpret_cast<float*>(w.S);
  int sweeps = 0;
  const bool ok = small_phase1(J, m, &sweeps);
  if (!ok) {
    if (threadIdx.x == 0) { w.ctl->fail = 1; w.ctl->stop = 1; }
    return;
  }
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) w.V[e] = (double)m.V32[e];
  if (threadIdx.x == 0) w.ctl->sweeps = sweeps;
}

// C = alpha op(A) B + beta D + gamma I (d x d, ld d); 16 x 16 tile per CTA.
__global__ void __launch_bounds__(256) sq_gemm_kernel(int d, const double* __restrict__ A,
                                                      int transA, const double* __restrict__ B,
                                                      double* __restrict__ C, double alpha,
                                                      const double* __restrict__ D, double beta,
                                                      double gamma, const int* __restrict__ skip) {
  if (*skip) return;
  __shared__ double As[16][17], Bs[16][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i = blockIdx.x * 16 + tx, j = blockIdx.y * 16 + ty;
  double acc = 0.0;
  for (int k0 = 0; k0 < d; k0 += 16) {
    // As[kk][ii] = op(A)[blockIdx.x*16 + ii][k0 + kk]; Bs[jj][kk] = B[k0 + kk][blockIdx.y*16 + jj]
    {
      const int ii = tx, kk = ty;
      const int r = blockIdx.x * 16 + ii, k = k0 + kk;
      double a = 0.0;
      if (r < d && k < d) a = transA ? A[k + (size_t)r * d] : A[r + (size_t)k * d];
      As[kk][ii] = a;
      const int kb = k0 + tx, cb = blockIdx.y * 16 + ty;
      Bs[ty][tx] = (kb < d && cb < d) ? B[kb + (size_t)cb * d] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) acc = fma(As[kk][tx], Bs[ty][kk], acc);
    __syncthreads();
  }
  if (i < d && j < d) {
    double v = alpha * acc;
    if (D) v = fma(beta, D[i + (size_t)j * d], v);
    if (i == j) v += gamma;
    C[i + (size_t)j * d] = v;
  }
}

// Rotation step: from S = B^T B (full, ld d) the tangents t of the pairs
// (Omega, upper +t / lower -t, zero diagonal, |t| <= kRotCap), the largest
// cosine of the capped pairs into ctl->cmax[it], the other pairs into the
// degenerate list.
__global__ void __launch_bounds__(256) sq_rot_kernel(int d, const double* __restrict__ S,
                                                     double* __restrict__ Om, WideCtl* ctl,
                                                     int it) {
  if (ctl->stop) return;
  __shared__ double red[8];
  double cmax = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d * d; e += gridDim.x * blockDim.x) {
    const int i = e % d, j = e / d;
    if (i == j) { Om[e] = 0.0; continue; }
    const int a = min(i, j), b = max(i, j);
    const double aa = S[a + (size_t)a * d], bb = S[b + (size_t)b * d], g = S[a + (size_t)b * d];
    double t = pair_rotation(aa, bb, g);
    if (fabs(t) > kRotCap) {
      t = 0.0;
      if (i < j) {
        const int q = atomicAdd(&ctl->npairs, 1);
        if (q < kMaxPairs) { ctl->pa[q] = (unsigned char)a; ctl->pb[q] = (unsigned char)b; }
      }
    } else if (i < j) {
      cmax = fmax(cmax, fabs(g) / sqrt(aa * bb));
    }
    Om[e] = (i < j) ? t : -t;
  }
  for (int o = 16; o > 0; o >>= 1) cmax = fmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) cmax = fmax(cmax, red[w]);
    atomicMax(&ctl->cmax[it], (unsigned long long)__double_as_longlong(cmax));
  }
}

// after sq_rot_kernel(it): converged when the largest capped cosine is
// below tol; otherwise clear the pair list for the next step
__global__ void sq_check_kernel(WideCtl* ctl, int it, double tol, int last) {
  if (ctl->stop) return;
  if (__longlong_as_double((long long)ctl->cmax[it]) <= tol) {
    ctl->stop = 1;
    ctl->conv = 1;
  } else if (!last) {
    ctl->npairs = 0;
  }
}

__global__ void sq_copy_kernel(int cnt, const double* __restrict__ src, double* __restrict__ dst,
                               const int* __restrict__ skip) {
  if (*skip) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += gridDim.x * blockDim.x)
    dst[e] = src[e];
}

// exact rotations of the degenerate pairs (B = G V, V), singular values and
// their ascending order, eigenvalues (one CTA)
__global__ void __launch_bounds__(SMALL_T) sq_final_kernel(SmallJob J, double tol) {
  const int d = J.d;
  const WideMats w = wide_place(J.work, d);
  WideCtl* ctl = w.ctl;
  if (ctl->fail) return;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5,
            nw = nt >> 5;
  __shared__ int s_rot;
  double* B = w.B;
  double* V = w.V;
  const int np = min(ctl->npairs, kMaxPairs);
  int left = 0;
  if (np > 0) {
    left = 1;
    for (int sw = 0; sw < 10 && left; ++sw) {
      if (tid == 0) s_rot = 0;
      __syncthreads();
      if (wid == 0) {
        for (int q = 0; q < np; ++q) {
          const int a = ctl->pa[q], b = ctl->pb[q];
          double al = 0.0, be = 0.0, ga = 0.0;
          for (int i = lane; i < d; i += 32) {
            const double x = B[i + a * d], y = B[i + b * d];
            al = fma(x, x, al); be = fma(y, y, be); ga = fma(x, y, ga);
          }
          al = warp_sum(al); be = warp_sum(be); ga = warp_sum(ga);
          if (fabs(ga) > tol * sqrt(al * be)) {
            const double t = pair_rotation(al, be, ga);
            const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
            for (int i = lane; i < d; i += 32) {
              const double x = B[i + a * d], y = B[i + b * d];
              B[i + a * d] = c * x - sn * y;
              B[i + b * d] = sn * x + c * y;
              const double u = V[i + a * d], v = V[i + b * d];
              V[i + a * d] = c * u - sn * v;
              V[i + b * d] = sn * u + c * v;
            }
            if (lane == 0) s_rot = 1;
          }
          __syncwarp();
        }
      }
      __syncthreads();
      left = s_rot;
      __syncthreads();
    }
  }
  for (int j = wid; j < d; j += nw) {
    double s = 0.0;
    for (int i = lane; i < d; i += 32) s = fma(B[i + j * d], B[i + j * d], s);
    s = warp_sum(s);
    if (lane == 0) w.sig[j] = sqrt(s);
  }
  __syncthreads();
  for (int j = tid; j < d; j += nt) {
    int rk = 0;
    const double sj = w.sig[j];
    for (int k = 0; k < d; ++k) rk += (w.sig[k] < sj) || (w.sig[k] == sj && k < j);
    w.perm[rk] = j;
  }
  __syncthreads();
  for (int i = tid; i < d; i += nt) J.lam[i] = w.sig[w.perm[i]];
  if (tid == 0) {
    *J.info = (ctl->conv && !left && ctl->npairs <= kMaxPairs) ? 0 : 3;
    if (J.sweeps) *J.sweeps = ctl->sweeps;
  }
}

// X^ = L2 V S^-1/2, Y^ = L1 W S^-1/2 with W = B / S (grid)
__global__ void __launch_bounds__(256) sq_assemble_kernel(SmallJob J) {
  const int d = J.d;
  const WideMats w = wide_place(J.work, d);
  if (w.ctl->fail) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d * d; e += gridDim.x * blockDim.x) {
    const int r = e % d, i = e / d;
    const int j = w.perm[i];
    const double s = w.sig[j];
    double x = 0.0, y = 0.0;
    for (int k = 0; k <= r; ++k) {
      x = fma(w.L2[r + k * d], w.V[k + j * d], x);
      y = fma(w.L1[r + k * d], w.B[k + j * d], y);
    }
    J.Xh[r + (size_t)i * J.ldo] = x / sqrt(s);
    J.Yh[r + (size_t)i * J.ldo] = y / (s * sqrt(s));
  }
}

// sign of each Ritz pair follows its previous iterate (X^[j, j] >= 0)
__global__ void __launch_bounds__(256) sq_flip_kernel(SmallJob J) {
  const int d = J.d;
  const WideMats w = wide_place(J.work, d);
  if (w.ctl->fail) return;
  const int wa = min(J.w_prev, d);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d * wa; e += gridDim.x * blockDim.x) {
    const int r = e % d, i = e / d;
    if (J.Xh[i + (size_t)i * J.ldo] < 0.0 && r != i) {
      J.Xh[r + (size_t)i * J.ldo] = -J.Xh[r + (size_t)i * J.ldo];
      J.Yh[r + (size_t)i * J.ldo] = -J.Yh[r + (size_t)i * J.ldo];
    }
  }
}
__global__ void sq_flip_diag_kernel(SmallJob J) {
  const int d = J.d;
  const WideMats w = wide_place(J.work, d);
  if (w.ctl->fail) return;
  const int wa = min(J.w_prev, d);
  for (int i = threadIdx.x; i < wa; i += blockDim.x)
    if (J.Xh[i + (size_t)i * J.ldo] < 0.0) {
      J.Xh[i + (size_t)i * J.ldo] = -J.Xh[i + (size_t)i * J.ldo];
      J.Yh[i + (size_t)i * J.ldo] = -J.Yh[i + (size_t)i * J.ldo];
    }
}

constexpr int kSmallDynBytes = 216 * 1024;

cudaError_t small_smem_setup() {
  static const cudaError_t once = [] {
    cudaError_t e = cudaFuncSetAttribute(
        small_lrep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmallDynBytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(small_lrep_one_kernel,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, kSmallDynBytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(small_front_kernel,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, kSmallDynBytes);
    return e;
  }();
  return once;
}

cudaError_t small_lrep_wide(const SmallJob& J, cudaStream_t st) {
  const int d = J.d;
  const WideMats w = wide_place(J.work, d);
  const int* fail = &w.ctl->fail;
  const int* stop = &w.ctl->stop;
  const double tol = (double)d * 2.220446049250313e-16;
  const dim3 g((d + 15) / 16, (d + 15) / 16);
  const unsigned ge = (unsigned)std::min(256, (d * d + 255) / 256);
  small_front_kernel<<<1, FRONT_T, kSmallDynBytes, st>>>(J, kSmallDynBytes); LREP_COUNT_LAUNCH();
  auto gemm = [&](const double* A, int tA, const double* B, double* C, double alpha,
                  const double* D, double beta, double gamma, const int* skip) {
    sq_gemm_kernel<<<g, 256, 0, st>>>(d, A, tA, B, C, alpha, D, beta, gamma, skip);
    LREP_COUNT_LAUNCH();
  };
  auto copy = [&](const double* src, double* dst, const int* skip) {
    sq_copy_kernel<<<ge, 256, 0, st>>>(d * d, src, dst, skip); LREP_COUNT_LAUNCH();
  };
  // Newton-Schulz: R = V^T V - I, T = V - V R / 2, V = T
  auto ns = [&](const int* skip) {
    gemm(w.V, 1, w.V, w.R, 1.0, nullptr, 0.0, -1.0, skip);
    gemm(w.V, 0, w.R, w.T, -0.5, w.V, 1.0, 0.0, skip);
    copy(w.T, w.V, skip);
  };
  ns(fail);
  ns(fail);
  for (int it = 0; it < 6; ++it) {
    gemm(w.G, 0, w.V, w.B, 1.0, nullptr, 0.0, 0.0, stop);   // B = G V
    gemm(w.B, 1, w.B, w.S, 1.0, nullptr, 0.0, 0.0, stop);   // S = B^T B
    sq_rot_kernel<<<ge, 256, 0, st>>>(d, w.S, w.R, w.ctl, it); LREP_COUNT_LAUNCH();
    sq_check_kernel<<<1, 1, 0, st>>>(w.ctl, it, tol, it == 5); LREP_COUNT_LAUNCH();
    gemm(w.V, 0, w.R, w.T, 1.0, w.V, 1.0, 0.0, stop);       // T = V + V Omega
    copy(w.T, w.V, stop);
    ns(stop);
    ns(stop);
    ns(stop);
  }
  gemm(w.G, 0, w.V, w.B, 1.0, nullptr, 0.0, 0.0, fail);     // B = G V
  sq_final_kernel<<<1, SMALL_T, 0, st>>>(J, tol); LREP_COUNT_LAUNCH();
  sq_assemble_kernel<<<ge, 256, 0, st>>>(J); LREP_COUNT_LAUNCH();
  sq_flip_kernel<<<ge, 256, 0, st>>>(J); LREP_COUNT_LAUNCH();
  sq_flip_diag_kernel<<<1, 256, 0, st>>>(J); LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

// ---------------------------------------------------------------- eq. hat_pq
__global__ void __launch_bounds__(256) small_pq_kernel(PqJob J) {
  const int d = J.d, na = J.na, end = J.end;
  const int tid = threadIdx.x, nt = blockDim.x;
  double* Pa = J.work;                 // d x na
  double* Qa = Pa + (size_t)d * na;
  double* T = Qa + (size_t)d * na;     // end x na coefficients (2 blocks)
  double* T2 = T + (size_t)d * na;
  __shared__ double refp[64], refq[64];
  // entering vectors X^_j - E_j, Y^_j - E_j
  for (int e = tid; e < d * na; e += nt) {
    const int r = e % d, c = e / d;
    const int j = J.act[c];
    const double ej = (j < J.w_prev && r == j) ? 1.0 : 0.0;
    Pa[e] = J.Xh[r + (size_t)j * J.ld] - ej;
    Qa[e] = J.Yh[r + (size_t)j * J.ld] - ej;
  }
  __syncthreads();
  for (int c = tid; c < na; c += nt) {
    double sp = 0.0, sq = 0.0;
    for (int r = 0; r < d; ++r) {
      sp = fma(Pa[r + c * d], Pa[r + c * d], sp);
      sq = fma(Qa[r + c * d], Qa[r + c * d], sq);
    }
    refp[c] = sqrt(sp);
    refq[c] = sqrt(sq);
  }
  // T = Y^[:, :end]^T Pa, T2 = X^[:, :end]^T Qa
  for (int e = tid; e < end * na; e += nt) {
    const int k = e % end, c = e / end;
    double s = 0.0, s2 = 0.0;
    for (int r = 0; r < d; ++r) {
      s = fma(J.Yh[r + (size_t)k * J.ld], Pa[r + c * d], s);
      s2 = fma(J.Xh[r + (size_t)k * J.ld], Qa[r + c * d], s2);
    }
    T[k + c * end] = s;
    T2[k + c * end] = s2;
  }
  __syncthreads();
  // projected: P^ = Pa - X^ T, Q^ = Qa - Y^ T2 (written to the outputs)
  for (int e = tid; e < d * na; e += nt) {
    const int r = e % d, c = e / d;
    double p = Pa[e], q = Qa[e];
    for (int k = 0; k < end; ++k) {
      p = fma(-J.Xh[r + (size_t)k * J.ld], T[k + c * end], p);
      q = fma(-J.Yh[r + (size_t)k * J.ld], T2[k + c * end], q);
    }
    J.Ph[r + (size_t)c * J.ldo] = p;
    J.Qh[r + (size_t)c * J.ldo] = q;
  }
  __syncthreads();
  // Alg. 1 on the columns, one warp, compacting kept pairs in place
  if (tid < 32) {
    const int lane = tid;
    int kept = 0;
    for (int c = 0; c < na; ++c) {
      double* p = J.Ph + (size_t)c * J.ldo;
      double* q = J.Qh + (size_t)c * J.ldo;
      for (int j = 0; j < kept; ++j) {
        const double* pj = J.Ph + (size_t)j * J.ldo;
        const double* qj = J.Qh + (size_t)j * J.ldo;
        double r = 0.0;
        for (int i = lane; i < d; i += 32) r = fma(qj[i], p[i], r);
        r = warp_sum(r);
        for (int i = lane; i < d; i += 32) p[i] = fma(-r, pj[i], p[i]);
        __syncwarp();
        double s = 0.0;
        for (int i = lane; i < d; i += 32) s = fma(pj[i], q[i], s);
        s = warp_sum(s);
        for (int i = lane; i < d; i += 32) q[i] = fma(-s, qj[i], q[i]);
        __syncwarp();
      }
      double eta = 0.0;
      for (int i = lane; i < d; i += 32) eta = fma(p[i], q[i], eta);
      eta = warp_sum(eta);
      if (!isfinite(eta) || !(fabs(eta) > J.tau * refp[c] * refq[c])) continue;
      const double root = sqrt(fabs(eta));
      const double rr = (eta > 0.0 ? root : -root);
      double* po = J.Ph + (size_t)kept * J.ldo;
      double* qo = J.Qh + (size_t)kept * J.ldo;
      for (int i = lane; i < d; i += 32) {
        const double pv = p[i] / rr, qv = q[i] / root;
        po[i] = pv;
        qo[i] = qv;
      }
      __syncwarp();
      ++kept;
    }
    if (lane == 0) *J.count = kept;
  }
}

// ------------------------------------------------- Alg. 1, coefficient form
// The coefficient vectors and the Sxy block live in dynamic shared memory
// when 5 m^2 + 3 m doubles fit (m <= 67), else in the global work array.
__global__ void __launch_bounds__(512)
biorth_coef_kernel(int m, const double* __restrict__ G2, int ld2,
                   const double* __restrict__ refw2, const double* __restrict__ refz2,
                   double tau, double* __restrict__ A, double* __restrict__ B, int ldc,
                   double* __restrict__ work, int* __restrict__ count, int dyn_bytes) {
  extern __shared__ double sh[];
  const size_t mm = (size_t)m * m;
  const bool in_smem = (5 * mm + 3 * (size_t)m) * sizeof(double) <= (size_t)dyn_bytes;
  double* a = sh;          // m
  double* b = a + m;       // m
  double* u = b + m;       // m
  double *Uc, *Vc, *Ac, *Bc, *S;
  int lda;
  if (in_smem) {
    Uc = u + m; Vc = Uc + mm; Ac = Vc + mm; Bc = Ac + mm; S = Bc + mm; lda = m;
  } else {
    Uc = work; Vc = Uc + mm; Ac = A; Bc = B; S = nullptr; lda = ldc;
  }
  __shared__ int s_kept, s_take;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
  if (in_smem)
    for (int e = tid; e < (int)mm; e += nt) {
      const int t = e % m, k = e / m;
      S[e] = G2[t + (size_t)(m + k) * ld2];
    }
#define SXY(t, k) (in_smem ? S[(t) + (size_t)(k) * m] : G2[(t) + (size_t)(m + (k)) * ld2])
  if (tid == 0) s_kept = 0;
  __syncthreads();
  for (int l = 0; l < m; ++l) {
    const int kept = s_kept;
    if (tid < 32) {
      for (int i = lane; i < m; i += 32) { a[i] = (i == l); b[i] = (i == l); }
      __syncwarp();
      for (int j = 0; j < kept; ++j) {
        double r = 0.0;
        for (int i = lane; i < m; i += 32) r = fma(Uc[i + (size_t)j * m], a[i], r);
        r = warp_sum(r);
        for (int i = lane; i < m; i += 32) a[i] = fma(-r, Ac[i + (size_t)j * lda], a[i]);
        double s2 = 0.0;
        for (int i = lane; i < m; i += 32) s2 = fma(Vc[i + (size_t)j * m], b[i], s2);
        s2 = warp_sum(s2);
        for (int i = lane; i < m; i += 32) b[i] = fma(-s2, Bc[i + (size_t)j * lda], b[i]);
        __syncwarp();
      }
    }
    __syncthreads();
    for (int t = tid; t < m; t += nt) {
      double acc = 0.0;
      for (int k = 0; k < m; ++k) acc = fma(SXY(t, k), b[k], acc);
      u[t] = acc;
    }
    __syncthreads();
    if (tid < 32) {
      double eta = 0.0;
      for (int i = lane; i < m; i += 32) eta = fma(a[i], u[i], eta);
      eta = warp_sum(eta);
      const double rw = refw2 ? sqrt(refw2[l]) : sqrt(G2[l + (size_t)l * ld2]);
      const double rz = refz2 ? sqrt(refz2[l]) : sqrt(G2[(m + l) + (size_t)(m + l) * ld2]);
      const int take = isfinite(eta) && (fabs(eta) > tau * rw * rz);
      if (take) {
        const double root = sqrt(fabs(eta));
        const double rr = eta > 0.0 ? root : -root;
        for (int i = lane; i < m; i += 32) {
          a[i] /= rr;
          b[i] /= root;
          u[i] /= root;
          Ac[i + (size_t)kept * lda] = a[i];
          Bc[i + (size_t)kept * lda] = b[i];
          Uc[i + (size_t)kept * m] = u[i];
        }
      }
      if (lane == 0) s_take = take;
    }
    __syncthreads();
    if (s_take) {
      for (int s3 = tid; s3 < m; s3 += nt) {
        double v = 0.0;
        for (int t = 0; t < m; ++t) v = fma(SXY(t, s3), a[t], v);
        Vc[s3 + (size_t)kept * m] = v;
      }
      __syncthreads();
      if (tid == 0) s_kept = kept + 1;
    }
    __syncthreads();
  }
#undef SXY
  const int kept = s_kept;
  for (int e = tid; e < (int)mm; e += nt) {
    const int i = e % m, j = e / m;
    const double va = (j < kept) ? Ac[i + (size_t)j * lda] : 0.0;
    const double vb = (j < kept) ? Bc[i + (size_t)j * lda] : 0.0;
    A[i + (size_t)j * ldc] = va;
    B[i + (size_t)j * ldc] = vb;
  }
  if (tid == 0) *count = kept;
}

// Alg. 1 in coefficient form through the LDU factorisation of S = W^T Z
// without pivoting: the biorthogonal pair P = W A, Q = Z B with upper
// triangular A, B and P^T Q = I is unique, and its pivots are the etas of
// Alg. 1 (the Schur complement of the kept leading pairs).  Right-looking
// elimination in shared memory, all threads on each rank-1 update of the
// trailing block; a pair whose pivot fails the discard test is skipped (no
// update), as Alg. 1 skips it.  Then A = L^-T D_a^-1 and B = U^-1 D_b^-1
// over the kept indices (D_a D_b = D, D_b = sqrt|eta|), one column per warp
// by column-oriented back substitution with the vector held in registers
// (lane i % 32, slot i / 32).  For m <= kLuMaxM (S fits in shared memory)
// and S close to the identity (see biorth_coef).
constexpr int kLuMaxM = 160;
constexpr int kLuSlots = (kLuMaxM + 31) / 32;

__global__ void __launch_bounds__(1024)
biorth_lu_kernel(int m, const double* __restrict__ G2, int ld2,
                 const double* __restrict__ refw2, const double* __restrict__ refz2,
                 double tau, double* __restrict__ A, double* __restrict__ B, int ldc,
                 int* __restrict__ count) {
  extern __shared__ double S[];  // m x m, S[i + j m]
  __shared__ int keep[kLuMaxM], pos[kLuMaxM];
  __shared__ int s_kept;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < m * m; e += nt) {
    const int i = e % m, j = e / m;
    S[e] = G2[i + (size_t)(m + j) * ld2];
  }
  __syncthreads();
  for (int l = 0; l < m; ++l) {
    if (tid == 0) {
      const double eta = S[l + l * m];
      const double rw = refw2 ? sqrt(refw2[l]) : sqrt(G2[l + (size_t)l * ld2]);
      const double rz = refz2 ? sqrt(refz2[l]) : sqrt(G2[(m + l) + (size_t)(m + l) * ld2]);
      keep[l] = isfinite(eta) && (fabs(eta) > tau * rw * rz);
    }
    __syncthreads();
    if (keep[l]) {
      const double inv = 1.0 / S[l + l * m];
      const int r = m - l - 1;
      for (int e = tid; e < r * r; e += nt) {
        const int i = l + 1 + e % r, j = l + 1 + e / r;
        S[i + j * m] = fma(-S[i + l * m] * inv, S[l + j * m], S[i + j * m]);
      }
      __syncthreads();
      for (int e = tid; e < r; e += nt) {
        S[(l + 1 + e) + l * m] *= inv;  // L(i, l)
        S[l + (l + 1 + e) * m] *= inv;  // U(l, j)
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    int k = 0;
    for (int l = 0; l < m; ++l) pos[l] = keep[l] ? k++ : -1;
    s_kept = k;
  }
  __syncthreads();
  const int kept = s_kept;
  // columns past the kept ones are zero
  for (int e = tid; e < m * (m - kept); e += nt) {
    const int i = e % m, j = kept + e / m;
    A[i + (size_t)j * ldc] = 0.0;
    B[i + (size_t)j * ldc] = 0.0;
  }
  // task t < m: A column of index t; t >= m: B column of index t - m
  const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
  for (int t = warp; t < 2 * m; t += nw) {
    const bool isB = t >= m;
    const int lk = isB ? t - m : t;
    if (!keep[lk]) continue;
    double xv[kLuSlots];
#pragma unroll
    for (int sl = 0; sl < kLuSlots; ++sl) xv[sl] = (sl * 32 + lane == lk) ? 1.0 : 0.0;
    for (int j = lk; j > 0; --j) {
      if (!keep[j]) continue;
      double own = 0.0;
#pragma unroll
      for (int sl = 0; sl < kLuSlots; ++sl)
        if (sl == (j >> 5)) own = xv[sl];
      const double xj = __shfl_sync(0xffffffffu, own, j & 31);
      // L^T x = e: x_i -= L(j, i) x_j;  U y = e: y_i -= U(i, j) y_j  (i < j)
#pragma unroll
      for (int sl = 0; sl < kLuSlots; ++sl) {
        const int i = sl * 32 + lane;
        if (i < j && keep[i]) {
          const double c = isB ? S[i + j * m] : S[j + i * m];
          xv[sl] = fma(-c, xj, xv[sl]);
        }
      }
    }
    const double eta = S[lk + lk * m];
    const double root = sqrt(fabs(eta));
    const double scl = isB ? root : (eta > 0.0 ? root : -root);
    double* out = (isB ? B : A) + (size_t)pos[lk] * ldc;
#pragma unroll
    for (int sl = 0; sl < kLuSlots; ++sl) {
      const int i = sl * 32 + lane;
      if (i < m) out[i] = (i <= lk && keep[i]) ? xv[sl] / scl : 0.0;
    }
  }
  if (tid == 0) *count = kept;
}

__global__ void biorth_error_kernel(int d, const double* __restrict__ S, int lds,
                                    double* __restrict__ out) {
  __shared__ double red[32];
  double m = 0.0;
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
    const int i = e % d, j = e / d;
    m = fmax(m, fabs(S[i + (size_t)j * lds] - (i == j ? 1.0 : 0.0)));
  }
  m = block_max(m, red);
  if (threadIdx.x == 0) *out = m;
}

// One thread: L L^T = G (r x r), then Cinv = L^-T.
__global__ void chol_upper_inverse_kernel(int r, const double* __restrict__ G, int ldg,
                                          double* __restrict__ Cinv, int ldc,
                                          double* __restrict__ L, int* __restrict__ info) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int j = 0; j < r; ++j)
    for (int i = 0; i < r; ++i) L[i + j * r] = (i >= j) ? 0.5 * (G[i + j * ldg] + G[j + i * ldg]) : 0.0;
  for (int j = 0; j < r; ++j) {
    double v = L[j + j * r];
    for (int k = 0; k < j; ++k) v -= L[j + k * r] * L[j + k * r];
    if (!(v > 0.0) || !isfinite(v)) { *info = 1; return; }
    const double piv = sqrt(v);
    L[j + j * r] = piv;
    for (int i = j + 1; i < r; ++i) {
      double s = L[i + j * r];
      for (int k = 0; k < j; ++k) s -= L[i + k * r] * L[j + k * r];
      L[i + j * r] = s / piv;
    }
  }
  // Linv (lower) by forward substitution on unit vectors; Cinv = Linv^T
  for (int c = 0; c < r; ++c) {
    for (int i = 0; i < r; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) s -= L[i + k * r] * Cinv[c + k * ldc];
      Cinv[c + i * ldc] = (i < c) ? 0.0 : s / L[i + i * r];
    }
  }
  *info = 0;
}

}  // namespace

cudaError_t chol_upper_inverse(int r, const double* G, int ldg, double* Cinv,
                               int ldc, double* work, int* info, cudaStream_t st) {
  if (r <= 0) return cudaSuccess;
  chol_upper_inverse_kernel<<<1, 32, 0, st>>>(r, G, ldg, Cinv, ldc, work, info); LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

size_t small_work_elems(int d) {
  return (size_t)8 * d * d + (sizeof(WideCtl) + 7) / 8 + 2 * (size_t)d + 64;
}

cudaError_t small_lrep_batched(const SmallJob* jobs_dev, int njobs, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  cudaError_t e = small_smem_setup();
  if (e != cudaSuccess) return e;
  small_lrep_kernel<<<njobs, SMALL_T, kSmallDynBytes, st>>>(jobs_dev, kSmallDynBytes); LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

int small_wide_min() { return kWideMin; }

cudaError_t small_lrep_one(const SmallJob& job, cudaStream_t st) {
  if (job.d <= 0 || job.d > SMALL_MAXD) return cudaErrorInvalidValue;
  cudaError_t e = small_smem_setup();
  if (e != cudaSuccess) return e;
  if (job.d >= kWideMin) return small_lrep_wide(job, st);
  small_lrep_one_kernel<<<1, SMALL_T, kSmallDynBytes, st>>>(job, kSmallDynBytes); LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

size_t pq_work_elems(int d, int na) { return (size_t)4 * d * (na > 0 ? na : 1); }

cudaError_t small_pq(const PqJob& job, cudaStream_t st) {
  if (job.na > 64 || job.d > SMALL_MAXD) return cudaErrorInvalidValue;
  small_pq_kernel<<<1, 256, 0, st>>>(job); LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

size_t biorth_coef_work_elems(int m) { return (size_t)2 * m * m; }

cudaError_t biorth_coef(int m, const double* G2, int ld2, const double* ref_w2,
                        const double* ref_z2, double tau, double* A, double* B,
                        int ldc, double* work, int* count, cudaStream_t st,
                        bool near_identity) {
  if (m <= 0) return cudaSuccess;
  constexpr int kCoefDyn = 200 * 1024;
  static const cudaError_t attr = cudaFuncSetAttribute(
      biorth_coef_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kCoefDyn);
  if (attr != cudaSuccess) return attr;
  if ((size_t)3 * m * sizeof(double) > (size_t)kCoefDyn) return cudaErrorInvalidValue;
  // The LU form serves the passes over bases that are already nearly
  // biorthogonal (S close to I: the safeguard's pass over U, V and every
  // second pass).  A first pass over new directions (the W, Z of eq.
  // update_W/Z, a random start block) keeps the MGS coefficient form, which
  // takes every projection coefficient afresh from the original Gram; the
  // Schur-complement updates of the LU form accumulate rounding in the
  // trailing block, and on ill-conditioned W^T Z that stalled a 64^3 stencil
  // solve at residual 1.4e-8.
  if (m <= kLuMaxM && near_identity) {
    constexpr int kLuDyn = kLuMaxM * kLuMaxM * (int)sizeof(double);
    static const cudaError_t lu_attr = cudaFuncSetAttribute(
        biorth_lu_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kLuDyn);
    if (lu_attr != cudaSuccess) return lu_attr;
    biorth_lu_kernel<<<1, 1024, (size_t)m * m * sizeof(double), st>>>(
        m, G2, ld2, ref_w2, ref_z2, tau, A, B, ldc, count); LREP_COUNT_LAUNCH();
    return cudaGetLastError();
  }
  biorth_coef_kernel<<<1, 512, kCoefDyn, st>>>(m, G2, ld2, ref_w2, ref_z2, tau, A, B,
                                               ldc, work, count, kCoefDyn); LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t biorth_error(int d, const double* S, int lds, double* out, cudaStream_t st) {
  biorth_error_kernel<<<1, 512, 0, st>>>(d, S, lds, out); LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

}  // namespace lrep
