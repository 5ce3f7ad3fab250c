// FP64 block kernels of the BOSP hot path: the dense operator product
// (Step 3 / Step 6 "mv"), tall-skinny Grams (eq. hat_H, eq. update_W/Z),
// block updates (eq. eigenVector-pullback, eq. update_W/Z), the residual
// norms of eq. tol and column utilities.
//
// GB300 notes: FP64 is issued on the CUDA cores at a fraction of the
// bf16 tensor rate, so these kernels are arithmetic-bound at the FP64 rate
// for the dense product and HBM-bound for the tall-skinny work; every
// reduction over n uses a fixed slab partition and a fixed summation order,
// so results do not depend on scheduling.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace lrep {

// =====================================================================
// Dense symmetric product Y = A X.  Because A is symmetric, row i of A is
// column i (contiguous): Y[i, j] = sum_k A[k, i] X[k, j].  A CTA owns a
// 64-row x 16-column output tile and a K range; 128 threads each hold a
// 4 x 2 register tile.
// =====================================================================
namespace {
constexpr int DM = 64, DN = 16, DK = 32, DT = 128;

__global__ void __launch_bounds__(DT)
dense_apply_kernel(int64_t n, int c, const double* __restrict__ A, int64_t lda,
                   const double* __restrict__ X, int64_t ldx,
                   double* __restrict__ Y, int64_t ldy, int64_t kchunk,
                   int partial, const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ double As[DK][DM + 1];
  __shared__ double Xs[DK][DN + 1];
  const int t = threadIdx.x;
  const int64_t i0 = (int64_t)blockIdx.x * DM;
  const int j0 = blockIdx.y * DN;
  const int64_t kb = (int64_t)blockIdx.z * kchunk;
  const int64_t ke = min(n, kb + kchunk);
  const int ty = t >> 3, tx = t & 7;
  double acc[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
  for (int64_t k0 = kb; k0 < ke; k0 += DK) {
#pragma unroll
    for (int s = 0; s < (DK * DM) / DT; ++s) {
      const int e = t + s * DT;
      const int kk = e % DK, ii = e / DK;
      const int64_t k = k0 + kk, i = i0 + ii;
      As[kk][ii] = (k < ke && i < n) ? A[k + i * lda] : 0.0;
    }
#pragma unroll
    for (int s = 0; s < (DK * DN) / DT; ++s) {
      const int e = t + s * DT;
      const int kk = e % DK, jj = e / DK;
      const int64_t k = k0 + kk;
      const int j = j0 + jj;
      Xs[kk][jj] = (k < ke && j < c) ? X[k + (int64_t)j * ldx] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < DK; ++kk) {
      double a[4], b[2];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty * 4 + r];
#pragma unroll
      for (int q = 0; q < 2; ++q) b[q] = Xs[kk][tx * 2 + q];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 2; ++q) acc[r][q] = fma(a[r], b[q], acc[r][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t i = i0 + ty * 4 + r;
    if (i >= n) continue;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int j = j0 + tx * 2 + q;
      if (j >= c) continue;
      if (partial)
        Y[(int64_t)blockIdx.z * n * c + (int64_t)j * n + i] = acc[r][q];
      else
        Y[i + (int64_t)j * ldy] = acc[r][q];
    }
  }
}

__global__ void splitk_reduce_kernel(int64_t n, int c, int splits,
                                     const double* __restrict__ P,
                                     double* __restrict__ Y, int64_t ldy,
                                     const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t tot = n * c;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += P[(int64_t)z * tot + e];
    const int64_t j = e / n, i = e % n;
    Y[i + j * ldy] = s;
  }
}

int dense_splits(int64_t n, int c) {
  const int64_t tiles = ((n + DM - 1) / DM) * ((c + DN - 1) / DN);
  int64_t s = (2 * kNumSMs + tiles - 1) / tiles;
  const int64_t kmax = (n + 1023) / 1024;  // keep >= 1024 K per split
  s = std::min<int64_t>(s, std::max<int64_t>(kmax, 1));
  return (int)std::max<int64_t>(s, 1);
}
}  // namespace

size_t dense_apply_ws_elems(int64_t n, int c) {
  const int s = dense_splits(n, c);
  return s > 1 ? (size_t)s * n * c : 0;
}

cudaError_t dense_apply_f64(int64_t n, int c, const double* A, int64_t lda,
                            const double* X, int64_t ldx, double* Y,
                            int64_t ldy, double* ws, size_t ws_elems,
                            const int* skip, cudaStream_t st) {
  if (n <= 0 || c <= 0) return cudaSuccess;
  int s = dense_splits(n, c);
  if (s > 1 && (ws == nullptr || ws_elems < (size_t)s * n * c)) s = 1;
  int64_t kchunk = (n + s - 1) / s;
  kchunk = ((kchunk + DK - 1) / DK) * DK;
  s = (int)((n + kchunk - 1) / kchunk);
  dim3 grid((unsigned)((n + DM - 1) / DM), (unsigned)((c + DN - 1) / DN), (unsigned)s);
  dense_apply_kernel<<<grid, DT, 0, st>>>(n, c, A, lda, X, ldx, s > 1 ? ws : Y,
                                          ldy, kchunk, s > 1, skip); LREP_COUNT_LAUNCH();
  if (s > 1) {
    const int64_t tot = n * c;
    const int blocks = (int)std::min<int64_t>((tot + 255) / 256, 8 * kNumSMs);
    splitk_reduce_kernel<<<blocks, 256, 0, st>>>(n, c, s, ws, Y, ldy, skip); LREP_COUNT_LAUNCH();
  }
  return cudaGetLastError();
}

// =====================================================================
// Tall-skinny Gram G = A^T B: CTA = one 32 x 32 output tile x one row slab;
// 256 threads, 2 x 2 outputs each; partials reduced in slab order.
// =====================================================================
namespace {
constexpr int GT = 32, GK = 32;

__global__ void __launch_bounds__(256)
gram_kernel(int64_t n, Segs A, Segs B, int a, int b, int tiles_b,
            int64_t slab_rows, double* __restrict__ part) {
  __shared__ double As[GK][GT + 1];
  __shared__ double Bs[GK][GT + 1];
  const int tile = blockIdx.x;
  const int ta = tile / tiles_b, tb = tile % tiles_b;
  const int slab = blockIdx.y;
  const int64_t r0 = (int64_t)slab * slab_rows;
  const int64_t r1 = min(n, r0 + slab_rows);
  const int t = threadIdx.x;
  const int ti = t & 15, tj = t >> 4;
  // column pointers of this tile (each thread loads 4 of A's and 4 of B's
  // 32 x 32 elements per step: column = e / 32, row = e % 32)
  double acc[2][2] = {{0, 0}, {0, 0}};
  for (int64_t k0 = r0; k0 < r1; k0 += GK) {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int e = t + s * 256;
      const int rr = e & 31, cc = e >> 5;
      const int64_t row = k0 + rr;
      const int ca = ta * GT + cc, cb = tb * GT + cc;
      double va = 0.0, vb = 0.0;
      if (row < r1) {
        if (ca < a) va = A.col(ca)[row];
        if (cb < b) vb = B.col(cb)[row];
      }
      As[rr][cc] = va;
      Bs[rr][cc] = vb;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < GK; ++kk) {
      const double a0 = As[kk][ti * 2], a1 = As[kk][ti * 2 + 1];
      const double b0 = Bs[kk][tj * 2], b1 = Bs[kk][tj * 2 + 1];
      acc[0][0] = fma(a0, b0, acc[0][0]);
      acc[0][1] = fma(a0, b1, acc[0][1]);
      acc[1][0] = fma(a1, b0, acc[1][0]);
      acc[1][1] = fma(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
  const int64_t ab = (int64_t)a * b;
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int i = ta * GT + ti * 2 + p, j = tb * GT + tj * 2 + q;
      if (i < a && j < b) part[(int64_t)slab * ab + (int64_t)j * a + i] = acc[p][q];
    }
}

__global__ void gram_reduce_kernel(int a, int b, int slabs,
                                   const double* __restrict__ part,
                                   double* __restrict__ G, int64_t ldg) {
  const int64_t ab = (int64_t)a * b;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ab;
       e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < slabs; ++z) s += part[(int64_t)z * ab + e];
    const int64_t j = e / a, i = e % a;
    G[i + j * ldg] = s;
  }
}

int gram_slabs(int64_t n, int a, int b) {
  const int tiles = ((a + GT - 1) / GT) * ((b + GT - 1) / GT);
  int64_t s = (4 * kNumSMs + tiles - 1) / tiles;
  s = std::min<int64_t>(s, (n + 127) / 128);
  return (int)std::max<int64_t>(s, 1);
}
}  // namespace

size_t gram_ws_elems(int64_t n, int a, int b) {
  return (size_t)gram_slabs(n, a, b) * a * b;
}

cudaError_t gram_f64(int64_t n, const Segs& A, const Segs& B, double* G,
                     int64_t ldg, double* ws, size_t ws_elems, cudaStream_t st) {
  const int a = A.total(), b = B.total();
  if (a <= 0 || b <= 0) return cudaSuccess;
  int slabs = gram_slabs(n, a, b);
  if (ws_elems < (size_t)slabs * a * b) return cudaErrorInvalidValue;
  int64_t slab_rows = (n + slabs - 1) / slabs;
  slab_rows = std::max<int64_t>(((slab_rows + GK - 1) / GK) * GK, GK);
  slabs = (int)std::max<int64_t>((n + slab_rows - 1) / slab_rows, 1);
  const int tiles_b = (b + GT - 1) / GT;
  const int tiles = ((a + GT - 1) / GT) * tiles_b;
  dim3 grid(tiles, slabs);
  gram_kernel<<<grid, 256, 0, st>>>(n, A, B, a, b, tiles_b, slab_rows, ws); LREP_COUNT_LAUNCH();
  const int64_t ab = (int64_t)a * b;
  const int blocks = (int)std::min<int64_t>((ab + 255) / 256, 4 * kNumSMs);
  gram_reduce_kernel<<<blocks, 256, 0, st>>>(a, b, slabs, ws, G, ldg); LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

// Same Gram with the number of row slabs capped (for a fixed-size caller
// scratch of ws_elems doubles); fewer slabs change only the summation
// partition.
cudaError_t gram_f64_capped(int64_t n, const Segs& A, const Segs& B, double* G,
                            int64_t ldg, double* ws, size_t ws_elems, cudaStream_t st) {
  const int a = A.total(), b = B.total();
  if (a <= 0 || b <= 0) return cudaSuccess;
  const size_t ab = (size_t)a * b;
  if (ws_elems < ab) return cudaErrorInvalidValue;
  int slabs = gram_slabs(n, a, b);
  slabs = (int)std::min<size_t>((size_t)slabs, ws_elems / ab);
  int64_t slab_rows = (n + slabs - 1) / slabs;
  slab_rows = std::max<int64_t>(((slab_rows + GK - 1) / GK) * GK, GK);
  slabs = (int)std::max<int64_t>((n + slab_rows - 1) / slab_rows, 1);
  const int tiles_b = (b + GT - 1) / GT;
  const int tiles = ((a + GT - 1) / GT) * tiles_b;
  gram_kernel<<<dim3(tiles, slabs), 256, 0, st>>>(n, A, B, a, b, tiles_b, slab_rows, ws); LREP_COUNT_LAUNCH();
  const int blocks = (int)std::min<int64_t>(((int64_t)ab + 255) / 256, 4 * kNumSMs);
  gram_reduce_kernel<<<blocks, 256, 0, st>>>(a, b, slabs, ws, G, ldg); LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

// =====================================================================
// Block update C = alpha C + beta A B, A n x k (segmented), B k x c.
// CTA = UM rows x UN columns with UM * UN = 2048; 256 threads, each one row
// and 8 columns; UN = 8, 16 or 32 follows c, so thin updates (c = 8 in a
// block of 8) do no work on padding columns.
// =====================================================================
namespace {
constexpr int UK = 16;

template <int UN>
__global__ void __launch_bounds__(256)
update_kernel(int64_t n, int c, int k, double alpha, Segs A,
              const double* __restrict__ B, int64_t ldb, double beta,
              double* __restrict__ C, int64_t ldc) {
  constexpr int UM = 2048 / UN;
  constexpr int G = UN / 8;  // column groups of 8
  __shared__ double As[UK][UM];
  __shared__ double Bs[UK][UN + 1];
  const int t = threadIdx.x;
  const int64_t i0 = (int64_t)blockIdx.x * UM;
  const int j0 = blockIdx.y * UN;
  const int r = t % UM, g = t / UM;
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int k0 = 0; k0 < k; k0 += UK) {
#pragma unroll
    for (int s = 0; s < (UK * UM) / 256; ++s) {
      const int e = t + s * 256;
      const int rr = e % UM, kk = e / UM;
      const int64_t row = i0 + rr;
      const int col = k0 + kk;
      As[kk][rr] = (row < n && col < k) ? A.col(col)[row] : 0.0;
    }
    for (int e = t; e < UK * UN; e += 256) {
      const int kk = e % UK, jj = e / UK;
      const int col = k0 + kk, j = j0 + jj;
      Bs[kk][jj] = (col < k && j < c) ? B[col + (int64_t)j * ldb] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < UK; ++kk) {
      const double a = As[kk][r];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] = fma(a, Bs[kk][g * 8 + q], acc[q]);
    }
    __syncthreads();
  }
  static_assert(G * UM == 256, "one row and 8 columns per thread");
  const int64_t row = i0 + r;
  if (row >= n) return;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int j = j0 + g * 8 + q;
    if (j >= c) continue;
    double* cp = C + row + (int64_t)j * ldc;
    const double v = beta * acc[q];
    *cp = (alpha == 0.0) ? v : fma(alpha, *cp, v);
  }
}

template <int UN>
void launch_update(int64_t n, int c, int k, double alpha, const Segs& A, const double* B,
                   int64_t ldb, double beta, double* C, int64_t ldc, cudaStream_t st) {
  constexpr int UM = 2048 / UN;
  dim3 grid((unsigned)((n + UM - 1) / UM), (unsigned)((c + UN - 1) / UN));
  update_kernel<UN><<<grid, 256, 0, st>>>(n, c, k, alpha, A, B, ldb, beta, C, ldc);
  LREP_COUNT_LAUNCH();
}
}  // namespace

cudaError_t update_f64(int64_t n, int c, double alpha, const Segs& A,
                       const double* B, int64_t ldb, double beta, double* C,
                       int64_t ldc, cudaStream_t st) {
  if (n <= 0 || c <= 0) return cudaSuccess;
  const int k = A.total();
  if (c <= 8)
    launch_update<8>(n, c, k, alpha, A, B, ldb, beta, C, ldc, st);
  else if (c <= 16)
    launch_update<16>(n, c, k, alpha, A, B, ldb, beta, C, ldc, st);
  else
    launch_update<32>(n, c, k, alpha, A, B, ldb, beta, C, ldc, st);
  return cudaGetLastError();
}

// =====================================================================
// Residual norms (eq. tol): partial sums of ||KX - lam Y||^2,
// ||MY - lam X||^2, ||X||^2, ||Y||^2 per (column, slab); the last block
// reduces them in slab order.
// =====================================================================
namespace {
__global__ void __launch_bounds__(256)
residual_kernel(int64_t n, int w, const double* __restrict__ X,
                const double* __restrict__ Y, const double* __restrict__ KX,
                const double* __restrict__ MY, const double* __restrict__ BX,
                const double* __restrict__ BY, int64_t ld,
                const double* __restrict__ lam, double* __restrict__ eps,
                double* __restrict__ part, unsigned int* counter,
                int64_t slab_rows) {
  __shared__ double red[32];
  const int col = blockIdx.y, slab = blockIdx.x, slabs = gridDim.x;
  const double l = lam[col];
  const int64_t r0 = (int64_t)slab * slab_rows, r1 = min(n, r0 + slab_rows);
  const int64_t off = (int64_t)col * ld;
  double s1 = 0, s2 = 0, s3 = 0, s4 = 0;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    const double x = X[off + i], y = Y[off + i];
    const double bx = BX ? BX[off + i] : x, by = BY ? BY[off + i] : y;
    const double a = KX[off + i] - l * by, b = MY[off + i] - l * bx;
    s1 = fma(a, a, s1); s2 = fma(b, b, s2); s3 = fma(x, x, s3); s4 = fma(y, y, s4);
  }
  s1 = block_sum(s1, red); s2 = block_sum(s2, red);
  s3 = block_sum(s3, red); s4 = block_sum(s4, red);
  if (threadIdx.x == 0) {
    double* p = part + ((int64_t)col * slabs + slab) * 4;
    p[0] = s1; p[1] = s2; p[2] = s3; p[3] = s4;
  }
  if (!arrive_last(counter)) return;
  for (int c = threadIdx.x; c < w; c += blockDim.x) {
    double t1 = 0, t2 = 0, t3 = 0, t4 = 0;
    for (int z = 0; z < slabs; ++z) {
      const double* p = part + ((int64_t)c * slabs + z) * 4;
      t1 += ld_cg(p); t2 += ld_cg(p + 1); t3 += ld_cg(p + 2); t4 += ld_cg(p + 3);
    }
    eps[c] = sqrt(t1 + t2) / ((1.0 + lam[c]) * sqrt(t3 + t4));
  }
}
}  // namespace

size_t residual_ws_elems(int64_t n, int w) {
  return (size_t)reduction_slabs(n, 2048, 64) * w * 4;
}

cudaError_t residuals_f64(int64_t n, int w, const double* X, const double* Y,
                          const double* KX, const double* MY, int64_t ld,
                          const double* lam, double* eps, double* part,
                          unsigned int* counter, cudaStream_t st, const double* BX,
                          const double* BY) {
  if (w <= 0) return cudaSuccess;
  const int slabs = reduction_slabs(n, 2048, 64);
  const int64_t slab_rows = (n + slabs - 1) / slabs;
  dim3 grid(slabs, w);
  residual_kernel<<<grid, 256, 0, st>>>(n, w, X, Y, KX, MY, BX, BY, ld, lam, eps, part,
                                        counter, slab_rows); LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

// =====================================================================
// Column utilities
// =====================================================================
namespace {
__global__ void gather_combine_kernel(int64_t n, int nb, const int* __restrict__ idx,
                                      const double* __restrict__ s1,
                                      const double* __restrict__ P1, double s2,
                                      const double* __restrict__ P2,
                                      const double* __restrict__ s3,
                                      const double* __restrict__ P3,
                                      int64_t ld_in, double* __restrict__ out,
                                      int64_t ld_out) {
  const int b = blockIdx.y;
  const int j = idx[b];
  const double a1 = s1 ? s1[b] : 1.0;
  const double a3 = (P3 && s3) ? s3[b] : 1.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v = a1 * P1[i + (int64_t)j * ld_in];
    if (P2) v = fma(s2, P2[i + (int64_t)j * ld_in], v);
    if (P3) v = fma(a3, P3[i + (int64_t)b * ld_out], v);
    out[i + (int64_t)b * ld_out] = v;
  }
}

__global__ void __launch_bounds__(256)
colnorm_kernel(int64_t n, int c, const double* __restrict__ A, int64_t lda,
               double* __restrict__ out, double* __restrict__ part,
               unsigned int* counter, int64_t slab_rows) {
  __shared__ double red[32];
  const int col = blockIdx.y, slab = blockIdx.x, slabs = gridDim.x;
  const int64_t r0 = (int64_t)slab * slab_rows, r1 = min(n, r0 + slab_rows);
  double s = 0;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    const double x = A[i + (int64_t)col * lda];
    s = fma(x, x, s);
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[(int64_t)col * slabs + slab] = s;
  if (!arrive_last(counter)) return;
  for (int j = threadIdx.x; j < c; j += blockDim.x) {
    double t = 0;
    for (int z = 0; z < slabs; ++z) t += ld_cg(part + (int64_t)j * slabs + z);
    out[j] = t;
  }
}

__global__ void copy_cols_kernel(int64_t n, const double* __restrict__ src,
                                 int64_t lds, double* __restrict__ dst, int64_t ldd) {
  const int j = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i + j * ldd] = src[i + j * lds];
}

__global__ void __launch_bounds__(256)
fix_sign_kernel(int64_t n, double* __restrict__ X, double* __restrict__ Y, int64_t ld) {
  __shared__ double sv[256];
  __shared__ int64_t si[256];
  const int j = blockIdx.x;
  double* x = X + (int64_t)j * ld;
  double* y = Y + (int64_t)j * ld;
  double best = -1.0;
  int64_t bi = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double a = fabs(x[i]);
    if (a > best) { best = a; bi = i; }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double b2 = sv[threadIdx.x + o];
      const int64_t i2 = si[threadIdx.x + o];
      if (b2 > sv[threadIdx.x] || (b2 == sv[threadIdx.x] && i2 < si[threadIdx.x])) {
        sv[threadIdx.x] = b2;
        si[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  const double sgn = (x[si[0]] < 0.0) ? -1.0 : 1.0;
  __syncthreads();
  if (sgn < 0.0)
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      x[i] = -x[i];
      y[i] = -y[i];
    }
}

__global__ void uv_kernel(int64_t n, const double* __restrict__ X,
                          const double* __restrict__ Y, int64_t ld,
                          double* __restrict__ U, double* __restrict__ V, int64_t ldo) {
  const int j = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double x = X[i + j * ld], y = Y[i + j * ld];
    U[i + j * ldo] = y + x;
    V[i + j * ldo] = y - x;
  }
}

__global__ void km_kernel(int64_t n, double* __restrict__ A, double* __restrict__ B,
                          int64_t ld) {
  const int64_t tot = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n, j = e / n;
    const double a = A[i + j * ld], b = B[i + j * ld];
    A[i + j * ld] = a - b;
    B[i + j * ld] = a + b;
  }
}

// Philox4x32-10 (Salmon et al., SC'11): S-box multipliers and Weyl key
// increments from the published definition.
__device__ __forceinline__ void philox10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

__global__ void philox_normal_kernel(int64_t n, int64_t total, uint32_t k0,
                                     uint32_t k1, uint32_t sid,
                                     double* __restrict__ out, int64_t ld) {
  const int64_t npair = (total + 1) / 2;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < npair;
       t += (int64_t)gridDim.x * blockDim.x) {
    uint32_t c[4] = {(uint32_t)(t & 0xffffffffu), (uint32_t)((uint64_t)t >> 32), sid, 0u};
    philox10(c, k0, k1);
    const double u1 = ((double)c[0] + 0.5) * (1.0 / 4294967296.0);
    const double u2 = ((double)c[1] + 0.5) * (1.0 / 4294967296.0);
    const double rad = sqrt(-2.0 * log(u1));
    double s, co;
    sincospi(2.0 * u2, &s, &co);
    const int64_t e0 = 2 * t, e1 = 2 * t + 1;
    out[(e0 % n) + (e0 / n) * ld] = rad * co;
    if (e1 < total) out[(e1 % n) + (e1 / n) * ld] = rad * s;
  }
}

unsigned grid1d(int64_t n, int per = 256, int cap = 4 * kNumSMs) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + per - 1) / per, cap));
}
}  // namespace

cudaError_t gather_combine(int64_t n, int nb, const int* idx, const double* s1,
                           const double* P1, double s2, const double* P2,
                           const double* s3, const double* P3, int64_t ld_in,
                           double* out, int64_t ld_out, cudaStream_t st) {
  if (nb <= 0) return cudaSuccess;
  dim3 grid(grid1d(n, 256, 2 * kNumSMs), nb);
  gather_combine_kernel<<<grid, 256, 0, st>>>(n, nb, idx, s1, P1, s2, P2, s3, P3,
                                              ld_in, out, ld_out); LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

size_t colnorm_ws_elems(int64_t n, int c) {
  return (size_t)reduction_slabs(n, 2048, 64) * c;
}

cudaError_t colnorm2_f64(int64_t n, int c, const double* A, int64_t lda,
                         double* out, double* part, unsigned int* counter,
                         cudaStream_t st) {
  if (c <= 0) return cudaSuccess;
  const int slabs = reduction_slabs(n, 2048, 64);
  const int64_t slab_rows = (n + slabs - 1) / slabs;
  colnorm_kernel<<<dim3(slabs, c), 256, 0, st>>>(n, c, A, lda, out, part, counter,
                                                 slab_rows); LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t copy_cols(int64_t n, int c, const double* src, int64_t lds,
                      double* dst, int64_t ldd, cudaStream_t st) {
  if (c <= 0 || n <= 0) return cudaSuccess;
  copy_cols_kernel<<<dim3(grid1d(n, 256, 64), c), 256, 0, st>>>(n, src, lds, dst, ldd); LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t fix_sign(int64_t n, int c, double* X, double* Y, int64_t ld,
                     cudaStream_t st) {
  if (c <= 0) return cudaSuccess;
  fix_sign_kernel<<<c, 256, 0, st>>>(n, X, Y, ld); LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t uv_from_xy(int64_t n, int c, const double* X, const double* Y,
                       int64_t ld, double* U, double* V, int64_t ldo,
                       cudaStream_t st) {
  if (c <= 0) return cudaSuccess;
  uv_kernel<<<dim3(grid1d(n, 256, 64), c), 256, 0, st>>>(n, X, Y, ld, U, V, ldo); LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t km_from_ab(int64_t n, double* A, double* B, int64_t ld, cudaStream_t st) {
  km_kernel<<<grid1d(n * n, 256, 8 * kNumSMs), 256, 0, st>>>(n, A, B, ld); LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t philox_normal(int64_t n, int c, uint64_t seed, int stream_id,
                          double* out, int64_t ld, cudaStream_t st) {
  const int64_t total = n * (int64_t)c;
  if (total <= 0) return cudaSuccess;
  philox_normal_kernel<<<grid1d((total + 1) / 2, 256, 8 * kNumSMs), 256, 0, st>>>(
      n, total, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32),
      (uint32_t)stream_id, out, ld); LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

}  // namespace lrep
