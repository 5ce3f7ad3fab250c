// Matrix-free operator products (7-point stencil, CSR) and the vector
// kernels of the block CG used for eq. block_GS (one independent CG per
// column; per-column alpha, beta; columns stop when ||r|| <= tol ||b||).
//
// CG control stays on the device: each kernel reads the `done` flag and
// returns at once when every column has converged, so the host can
// enqueue the iteration budget without a read-back per step.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace lrep {
namespace {

// ------------------------------------------------------------- stencil
// Y = coef * Lap_h X + d .* X, zero values outside the grid.  2.5-D
// blocking: a CTA owns a 32 x 8 tile of one xy plane of one column and
// marches along z over a chunk of planes; the z-1 / z+1 neighbours stay in
// registers and the current plane (with a one-point halo) is staged in
// shared memory, so each value is read from memory about once.
constexpr int STX = 32, STY = 8;

template <typename T>
__global__ void __launch_bounds__(STX * STY)
stencil_kernel(int nx, int ny, int nz, double coef_d, const double* __restrict__ d,
               const double* __restrict__ X, int64_t ldx, double* __restrict__ Y,
               int64_t ldy, int zchunk, int tiles_x, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const T coef = (T)coef_d;
  __shared__ T s[STY + 2][STX + 2];
  const int tx = threadIdx.x % STX, ty = threadIdx.x / STX;
  const int tile = blockIdx.x;
  const int i0 = (tile % tiles_x) * STX, j0 = (tile / tiles_x) * STY;
  const int i = i0 + tx, j = j0 + ty;
  const bool in = (i < nx) && (j < ny);
  const int z0 = blockIdx.y * zchunk;
  const int z1 = min(nz, z0 + zchunk);
  const int64_t plane = (int64_t)nx * ny;
  const double* x = X + (int64_t)blockIdx.z * ldx;
  double* y = Y + (int64_t)blockIdx.z * ldy;
  const int64_t p0 = (int64_t)j * nx + i;
  T below = (in && z0 > 0) ? (T)x[p0 + (int64_t)(z0 - 1) * plane] : (T)0;
  T cur = (in && z0 < nz) ? (T)x[p0 + (int64_t)z0 * plane] : (T)0;
  for (int z = z0; z < z1; ++z) {
    const int64_t pz = (int64_t)z * plane;
    const T above = (in && z + 1 < nz) ? (T)x[p0 + pz + plane] : (T)0;
    s[ty + 1][tx + 1] = cur;
    // halo: left/right columns by the first/last lane of each row, top/
    // bottom rows by the first/last warp
    if (tx == 0) s[ty + 1][0] = (i0 > 0 && j < ny) ? (T)x[pz + (int64_t)j * nx + i0 - 1] : (T)0;
    if (tx == STX - 1)
      s[ty + 1][STX + 1] =
          (i0 + STX < nx && j < ny) ? (T)x[pz + (int64_t)j * nx + i0 + STX] : (T)0;
    if (ty == 0) s[0][tx + 1] = (j0 > 0 && i < nx) ? (T)x[pz + (int64_t)(j0 - 1) * nx + i] : (T)0;
    if (ty == STY - 1)
      s[STY + 1][tx + 1] =
          (j0 + STY < ny && i < nx) ? (T)x[pz + (int64_t)(j0 + STY) * nx + i] : (T)0;
    __syncthreads();
    if (in) {
      const T lap = s[ty + 1][tx] + s[ty + 1][tx + 2] + s[ty][tx + 1] + s[ty + 2][tx + 1] +
                    below + above - (T)6 * cur;
      y[p0 + pz] = (double)fma(coef, lap, (T)d[p0 + pz] * cur);
    }
    __syncthreads();
    below = cur;
    cur = above;
  }
}

// z-marching form for the float32 CG products: the 32 x 8 tile of the
// 2.5-D form, four columns per thread, but no shared memory and no
// barriers: the x and y neighbours are the tile's own loads of the same
// plane (L1 hits), the z neighbours stay in registers, and the warps march
// independently with the next planes' loads in flight.  Loads are narrowed
// to float32 by truncation on the integer units and the result widened
// exactly (a hardware conversion is a float64 instruction on GB300, ~2 per
// clock per SM).  The float64 products stay on the 2.5-D form, which is
// bound by the FP64 pipe on GB300 (~8 FP64 operations per point and column)
// either way.
constexpr int SZC = 4;  // columns per thread

__global__ void __launch_bounds__(STX * STY, 5)
stencil_z_f32_kernel(int nx, int ny, int nz, float coef, const double* __restrict__ d,
                     int c, const double* __restrict__ X, int64_t ldx,
                     double* __restrict__ Y, int64_t ldy, int zchunk, int tiles_x,
                     const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int tx = threadIdx.x % STX, ty = threadIdx.x / STX;
  const int tile = blockIdx.x;
  const int i = (tile % tiles_x) * STX + tx, j = (tile / tiles_x) * STY + ty;
  if (i >= nx || j >= ny) return;
  const int z0 = blockIdx.y * zchunk, z1 = min(nz, z0 + zchunk);
  const int c0 = blockIdx.z * SZC;
  const int64_t plane = (int64_t)nx * ny;
  const bool xl = i > 0, xr = i + 1 < nx, yl = j > 0, yr = j + 1 < ny;
  const double* x[SZC];
  double* y[SZC];
  float below[SZC], cur[SZC];
  const int64_t p0 = (int64_t)j * nx + i + (int64_t)z0 * plane;
#pragma unroll
  for (int q = 0; q < SZC; ++q) {
    const int col = min(c0 + q, c - 1);
    x[q] = X + (int64_t)col * ldx + p0;
    y[q] = Y + (int64_t)col * ldy + p0;
    below[q] = z0 > 0 ? f64_to_f32_rz(__ldg(x[q] - plane)) : 0.f;
    cur[q] = f64_to_f32_rz(__ldg(x[q]));
  }
  const double* dz = d + p0;
  const int ncol = min(SZC, c - c0);
#pragma unroll 2
  for (int z = z0; z < z1; ++z) {
    const bool up = z + 1 < nz;
    const float dp = f64_to_f32_rz(__ldg(dz));
#pragma unroll
    for (int q = 0; q < SZC; ++q) {
      const double* xq = x[q];
      const float above = up ? f64_to_f32_rz(__ldg(xq + plane)) : 0.f;
      const float s4 = (xl ? f64_to_f32_rz(__ldg(xq - 1)) : 0.f) +
                       (xr ? f64_to_f32_rz(__ldg(xq + 1)) : 0.f) +
                       (yl ? f64_to_f32_rz(__ldg(xq - nx)) : 0.f) +
                       (yr ? f64_to_f32_rz(__ldg(xq + nx)) : 0.f);
      const float lap = s4 + below[q] + above - 6.f * cur[q];
      if (q < ncol) *y[q] = f32_to_f64(fmaf(coef, lap, dp * cur[q]));
      below[q] = cur[q];
      cur[q] = above;
      x[q] = xq + plane;
      y[q] += plane;
    }
    dz += plane;
  }
}

// ----------------------------------------------------------------- CSR
// One thread per row; the row's entries are read once and applied to up to
// 8 columns per pass.
__global__ void __launch_bounds__(256)
csr_kernel(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
           const double* __restrict__ v, int c, const double* __restrict__ X,
           int64_t ldx, double* __restrict__ Y, int64_t ldy,
           const int* __restrict__ skip) {
  if (skip && *skip) return;
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < n;
       row += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = rp[row], e = rp[row + 1];
    for (int c0 = 0; c0 < c; c0 += 8) {
      double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      const int cw = min(8, c - c0);
      for (int64_t q = b; q < e; ++q) {
        const int64_t col = ci[q];
        const double a = v[q];
#pragma unroll
        for (int t = 0; t < 8; ++t)
          if (t < cw) acc[t] = fma(a, X[col + (int64_t)(c0 + t) * ldx], acc[t]);
      }
#pragma unroll
      for (int t = 0; t < 8; ++t)
        if (t < cw) Y[row + (int64_t)(c0 + t) * ldy] = acc[t];
    }
  }
}

// ------------------------------------------------------------------ CG
__global__ void __launch_bounds__(256)
cg_init_kernel(int64_t n, int nb, const double* __restrict__ B, int64_t ldb,
               double* __restrict__ X, double* __restrict__ R, double* __restrict__ P,
               int64_t ld, double tol, CgState s, int64_t slab_rows) {
  __shared__ double red[32];
  const int col = blockIdx.y, slab = blockIdx.x, slabs = gridDim.x;
  const int64_t r0 = (int64_t)slab * slab_rows, r1 = min(n, r0 + slab_rows);
  double acc = 0.0;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    const double b = B[i + (int64_t)col * ldb];
    X[i + (int64_t)col * ld] = 0.0;
    R[i + (int64_t)col * ld] = b;
    P[i + (int64_t)col * ld] = b;
    acc = fma(b, b, acc);
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) s.part[(int64_t)col * slabs + slab] = acc;
  if (!arrive_last(s.counter + 2)) return;
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int c = threadIdx.x; c < nb; c += blockDim.x) {
    double rho = 0.0;
    for (int z = 0; z < slabs; ++z) rho += ld_cg(s.part + (int64_t)c * slabs + z);
    s.rho[c] = rho;
    s.stop[c] = tol * tol * rho;
    const int act = (rho > tol * tol * rho) && isfinite(rho);
    s.active[c] = act;
    s.alpha[c] = 0.0;
    s.beta[c] = 0.0;
    if (act) atomicOr(&any, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) *s.done = any ? 0 : 1;
}

__global__ void __launch_bounds__(256)
cg_alpha_kernel(int64_t n, int nb, const double* __restrict__ P,
                const double* __restrict__ Q, int64_t ld, CgState s, int64_t slab_rows) {
  if (*s.done) return;
  __shared__ double red[32];
  const int col = blockIdx.y, slab = blockIdx.x, slabs = gridDim.x;
  const int64_t r0 = (int64_t)slab * slab_rows, r1 = min(n, r0 + slab_rows);
  double acc = 0.0;
  if (s.active[col])
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x)
      acc = fma(P[i + (int64_t)col * ld], Q[i + (int64_t)col * ld], acc);
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) s.part[(int64_t)col * slabs + slab] = acc;
  if (!arrive_last(s.counter)) return;
  if (threadIdx.x == 0 && s.iters) *s.iters += 1;
  for (int c = threadIdx.x; c < nb; c += blockDim.x) {
    double pq = 0.0;
    for (int z = 0; z < slabs; ++z) pq += ld_cg(s.part + (int64_t)c * slabs + z);
    if (s.active[c] && pq > 0.0 && isfinite(pq)) {
      s.alpha[c] = s.rho[c] / pq;
    } else {
      s.alpha[c] = 0.0;
      s.active[c] = 0;
    }
  }
}

__global__ void __launch_bounds__(256)
cg_update_kernel(int64_t n, int nb, double* __restrict__ X, double* __restrict__ R,
                 const double* __restrict__ P, const double* __restrict__ Q,
                 int64_t ld, CgState s, int64_t slab_rows) {
  if (*s.done) return;
  __shared__ double red[32];
  const int col = blockIdx.y, slab = blockIdx.x, slabs = gridDim.x;
  const int64_t r0 = (int64_t)slab * slab_rows, r1 = min(n, r0 + slab_rows);
  const double a = s.alpha[col];
  double acc = 0.0;
  if (a != 0.0)
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      const int64_t o = i + (int64_t)col * ld;
      X[o] = fma(a, P[o], X[o]);
      const double r = fma(-a, Q[o], R[o]);
      R[o] = r;
      acc = fma(r, r, acc);
    }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) s.part[(int64_t)col * slabs + slab] = acc;
  if (!arrive_last(s.counter + 1)) return;
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int c = threadIdx.x; c < nb; c += blockDim.x) {
    if (s.active[c]) {
      double rn = 0.0;
      for (int z = 0; z < slabs; ++z) rn += ld_cg(s.part + (int64_t)c * slabs + z);
      s.beta[c] = rn / s.rho[c];
      s.rho[c] = rn;
      if (!(rn > s.stop[c]) || !isfinite(rn)) s.active[c] = 0;
    }
    if (s.active[c]) atomicOr(&any, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) *s.done = any ? 0 : 1;
}

__global__ void cg_pdir_kernel(int64_t n, const double* __restrict__ R,
                               double* __restrict__ P, int64_t ld, CgState s) {
  if (*s.done) return;
  const int col = blockIdx.y;
  if (!s.active[col]) return;
  const double b = s.beta[col];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = i + (int64_t)col * ld;
    P[o] = fma(b, P[o], R[o]);
  }
}

// cg_alpha_kernel with Q formed first from the split-K partials of the
// tensor-core product (inactive columns: Q is not needed and not formed).
// The fp32 partials are summed in fp32, in split order, and converted once:
// on GB300 every float64 operation (conversions included) runs at ~2 per
// clock per SM, and the seven float64 additions per entry made this kernel
// ALU-bound; the fp32 sum adds ~2^-22 relative error to a product that
// carries ~2^-16.
__global__ void __launch_bounds__(256)
cg_sum_alpha_kernel(int64_t n, int nb, const float* __restrict__ part, int splits,
                    const double* __restrict__ P, double* __restrict__ Q, int64_t ld,
                    CgState s, int64_t slab_rows) {
  if (*s.done) return;
  __shared__ double red[32];
  const int col = blockIdx.y, slab = blockIdx.x, slabs = gridDim.x;
  const int64_t r0 = (int64_t)slab * slab_rows, r1 = min(n, r0 + slab_rows);
  double acc = 0.0;
  if (s.active[col])
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      float qf = 0.0f;
      for (int z = 0; z < splits; ++z) qf += part[((int64_t)z * nb + col) * n + i];
      const double q = f32_to_f64(qf);
      Q[i + (int64_t)col * ld] = q;
      acc = fma(P[i + (int64_t)col * ld], q, acc);
    }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) s.part[(int64_t)col * slabs + slab] = acc;
  if (!arrive_last(s.counter)) return;
  if (threadIdx.x == 0 && s.iters) *s.iters += 1;
  for (int c = threadIdx.x; c < nb; c += blockDim.x) {
    double pq = 0.0;
    for (int z = 0; z < slabs; ++z) pq += ld_cg(s.part + (int64_t)c * slabs + z);
    if (s.active[c] && pq > 0.0 && isfinite(pq)) {
      s.alpha[c] = s.rho[c] / pq;
    } else {
      s.alpha[c] = 0.0;
      s.active[c] = 0;
    }
  }
}

// cg_pdir_kernel that also writes the bf16 split of the new direction p:
// with f = fp32(p) (one float64 conversion), hi = bf16(f), lo = bf16(f - hi)
// (f - hi is exact in fp32).  hi + lo is within ~2^-17 of p, as for a
// split taken from the float64 value directly, at one float64 operation
// per entry instead of four.
__global__ void cg_pdir_split_kernel(int64_t n, const double* __restrict__ R,
                                     double* __restrict__ P, int64_t ld, CgState s,
                                     __nv_bfloat16* __restrict__ hi,
                                     __nv_bfloat16* __restrict__ lo, int64_t ldb) {
  if (*s.done) return;
  const int col = blockIdx.y;
  if (!s.active[col]) return;
  const double b = s.beta[col];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = i + (int64_t)col * ld;
    const double pv = fma(b, P[o], R[o]);
    P[o] = pv;
    const float f = f64_to_f32(pv);
    const __nv_bfloat16 h = __float2bfloat16_rn(f);
    hi[i + (int64_t)col * ldb] = h;
    lo[i + (int64_t)col * ldb] = __float2bfloat16_rn(f - __bfloat162float(h));
  }
}

// ------------------------------------------------- one-launch CG step
// cg_sum_alpha + cg_update + cg_pdir_split in one cooperative launch: the
// CTA of (slab, column) keeps its rows of p and q (later r) in registers
// across the three phases, and the two reductions of the step (p.q for
// alpha, r.r for beta) are barriers over the column's CTAs instead of
// kernel boundaries.  Every CTA reads its column's state (active, rho,
// stop) at entry and derives alpha and beta from the column's partials in
// a fixed order; CTA (0, 0) alone writes the new state of every column,
// after every column has passed its second barrier, so no state is read
// after it is rewritten.  Same arithmetic as the three kernels, with the
// per-thread row order of this kernel's slabs.
constexpr int kCoopRows = 8;                        // rows per thread
constexpr int kCoopMaxCols = 120;                   // column barriers in CgState.counter
constexpr long long kBarrierCycles = 4000000000ll;  // ~2 s of SM clock

// Wait until *count >= target (thread 0 of the CTA); bounded: on expiry
// *err is set to 6 and false returned.
__device__ __forceinline__ bool wait_count(const unsigned int* count, unsigned int target,
                                           int* err) {
  const long long t0 = clock64();
  while (*(const volatile unsigned int*)count < target) {
    if (clock64() - t0 > kBarrierCycles) {
      if (err) atomicExch(err, 6);
      return false;
    }
    __nanosleep(100);
  }
  return true;
}

// Barrier over the CTAs that share `count` (one arrival per CTA per
// barrier; the k-th barrier of the CG solve waits for k * members).
__device__ __forceinline__ bool group_barrier(unsigned int* count, unsigned int target,
                                              int* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(count, 1u);
    ok = wait_count(count, target, err) ? 1 : 0;
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

__global__ void __launch_bounds__(256, 4)
cg_step_coop_kernel(int64_t n, int nb, const float* __restrict__ part, int splits,
                    double* __restrict__ X, double* __restrict__ R, double* __restrict__ P,
                    int64_t ld, CgState s, __nv_bfloat16* __restrict__ hi,
                    __nv_bfloat16* __restrict__ lo, int64_t ldb, int64_t slab_rows, int epoch,
                    int* err) {
  if (*s.done) return;
  __shared__ double red[32];
  __shared__ double sh_coef;
  const int col = blockIdx.y, slab = blockIdx.x, slabs = gridDim.x;
  unsigned int* bar = s.counter + 8;  // one barrier counter per column
  const unsigned int t1 = (unsigned int)(2 * epoch + 1) * slabs, t2 = t1 + slabs;
  const int64_t r0 = (int64_t)slab * slab_rows, r1 = min(n, r0 + slab_rows);
  const int64_t cx = (int64_t)col * ld;
  const bool act0 = s.active[col] != 0;
  const double rho = s.rho[col], stop = s.stop[col];
  double* part1 = s.part;                        // p.q partials
  double* part2 = s.part + (int64_t)nb * slabs;  // r.r partials
  double pr[kCoopRows], qr[kCoopRows];
  // phase 1: q = A p from the split-K partials (split order, every row's
  // partial of one split in flight together), p.q
  float qf[kCoopRows];
#pragma unroll
  for (int k = 0; k < kCoopRows; ++k) qf[k] = 0.0f;
  if (act0)
    for (int z = 0; z < splits; ++z) {
      const float* pz = part + ((int64_t)z * nb + col) * n;
#pragma unroll
      for (int k = 0; k < kCoopRows; ++k) {
        const int64_t i = r0 + threadIdx.x + (int64_t)k * blockDim.x;
        if (i < r1) qf[k] += pz[i];
      }
    }
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < kCoopRows; ++k) {
    const int64_t i = r0 + threadIdx.x + (int64_t)k * blockDim.x;
    pr[k] = 0.0;
    qr[k] = 0.0;
    if (act0 && i < r1) {
      qr[k] = f32_to_f64(qf[k]);
      pr[k] = P[i + cx];
      acc = fma(pr[k], qr[k], acc);
    }
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) part1[(int64_t)col * slabs + slab] = acc;
  if (!group_barrier(bar + col, t1, err)) return;
  // alpha (thread 0: one float64 division per CTA)
  if (threadIdx.x == 0) {
    double pq = 0.0;
    for (int z = 0; z < slabs; ++z) pq += ld_cg(part1 + (int64_t)col * slabs + z);
    sh_coef = (act0 && pq > 0.0 && isfinite(pq)) ? rho / pq : 0.0;
  }
  __syncthreads();
  const double alpha = sh_coef;
  const bool act1 = alpha != 0.0;
  // phase 2: x += alpha p, r -= alpha q, r.r
  double acc2 = 0.0;
  if (act1) {
#pragma unroll
    for (int k = 0; k < kCoopRows; ++k) {
      const int64_t i = r0 + threadIdx.x + (int64_t)k * blockDim.x;
      if (i < r1) {
        const int64_t o = i + cx;
        X[o] = fma(alpha, pr[k], X[o]);
        const double r = fma(-alpha, qr[k], R[o]);
        R[o] = r;
        qr[k] = r;
        acc2 = fma(r, r, acc2);
      }
    }
  }
  acc2 = block_sum(acc2, red);
  if (threadIdx.x == 0) part2[(int64_t)col * slabs + slab] = acc2;
  if (!group_barrier(bar + col, t2, err)) return;
  // beta (thread 0), -1 when the column stops
  if (threadIdx.x == 0) {
    double rn = 0.0;
    for (int z = 0; z < slabs; ++z) rn += ld_cg(part2 + (int64_t)col * slabs + z);
    sh_coef = (act1 && rn > stop && isfinite(rn)) ? rn / rho : -1.0;
  }
  __syncthreads();
  const double beta = sh_coef;
  // phase 3: p = r + beta p and its bf16 split
  if (beta >= 0.0) {
#pragma unroll
    for (int k = 0; k < kCoopRows; ++k) {
      const int64_t i = r0 + threadIdx.x + (int64_t)k * blockDim.x;
      if (i < r1) {
        const double pv = fma(beta, pr[k], qr[k]);
        P[i + cx] = pv;
        const float f = f64_to_f32(pv);
        const __nv_bfloat16 h = __float2bfloat16_rn(f);
        hi[i + (int64_t)col * ldb] = h;
        lo[i + (int64_t)col * ldb] = __float2bfloat16_rn(f - __bfloat162float(h));
      }
    }
  }
  // the new state of every column (CTA (0, 0) only, once every column has
  // passed its second barrier)
  if (slab == 0 && col == 0) {
    __shared__ int any, all_ok;
    if (threadIdx.x == 0) {
      any = 0;
      all_ok = 1;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < nb; c += blockDim.x)
      if (!wait_count(bar + c, t2, err)) atomicExch(&all_ok, 0);
    __syncthreads();
    if (!all_ok) return;
    __threadfence();
    for (int c = threadIdx.x; c < nb; c += blockDim.x) {
      if (!s.active[c]) {
        s.alpha[c] = 0.0;
        continue;
      }
      double q = 0.0, r = 0.0;
      for (int z = 0; z < slabs; ++z) q += ld_cg(part1 + (int64_t)c * slabs + z);
      if (!(q > 0.0 && isfinite(q))) {
        s.alpha[c] = 0.0;
        s.active[c] = 0;
        continue;
      }
      s.alpha[c] = s.rho[c] / q;
      for (int z = 0; z < slabs; ++z) r += ld_cg(part2 + (int64_t)c * slabs + z);
      s.beta[c] = r / s.rho[c];
      s.rho[c] = r;
      if (!(r > s.stop[c]) || !isfinite(r)) s.active[c] = 0;
      if (s.active[c]) atomicOr(&any, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      *s.done = any ? 0 : 1;
      if (s.iters) *s.iters += 1;
    }
  }
}

int cg_slabs(int64_t n) { return reduction_slabs(n, 2048, 64); }
unsigned grid_rows(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 2 * kNumSMs));
}
}  // namespace

cudaError_t stencil_apply_f64(int nx, int ny, int nz, double coef_h2,
                              const double* d, int c, const double* X,
                              int64_t ldx, double* Y, int64_t ldy,
                              const int* skip, cudaStream_t st) {
  return stencil_apply(false, nx, ny, nz, coef_h2, d, c, X, ldx, Y, ldy, skip, st);
}

cudaError_t stencil_apply(bool f32, int nx, int ny, int nz, double coef_h2, const double* d,
                          int c, const double* X, int64_t ldx, double* Y, int64_t ldy,
                          const int* skip, cudaStream_t st) {
  if (c <= 0) return cudaSuccess;
  const int tiles_x = (nx + STX - 1) / STX, tiles_y = (ny + STY - 1) / STY;
  const int tiles = tiles_x * tiles_y;
  // z chunks: enough CTAs for ~4 per SM over all columns, >= 8 planes each
  int zchunks = (int)std::max<int64_t>(1, (4 * kNumSMs + (int64_t)tiles * c - 1) / ((int64_t)tiles * c));
  zchunks = std::min(zchunks, std::max(1, nz / 8));
  const int zchunk = (nz + zchunks - 1) / zchunks;
  zchunks = (nz + zchunk - 1) / zchunk;
  if (f32) {
    // z chunks (of >= 4 planes): fewest waves of the resident slots times
    // (planes per chunk + the 2 planes a chunk loads before its first)
    const int cgrp = (c + SZC - 1) / SZC;
    static const int64_t slots = [] {
      int per = 0, dev = 0, sms = kNumSMs;
      if (cudaGetDevice(&dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, stencil_z_f32_kernel, STX * STY,
                                                        0) != cudaSuccess ||
          per < 1)
        return (int64_t)4 * kNumSMs;
      return (int64_t)per * sms;
    }();
    const int64_t unit = (int64_t)tiles * cgrp;
    int zc = 1;
    int64_t best = -1;
    for (int t = 1; t <= std::max(1, nz / 4); ++t) {
      const int tch = (nz + t - 1) / t;
      const int64_t w = unit * ((nz + tch - 1) / tch);
      const int64_t cost = ((w + slots - 1) / slots) * (tch + 2);
      if (best < 0 || cost < best) {
        best = cost;
        zc = t;
      }
    }
    const int zch = (nz + zc - 1) / zc;
    zc = (nz + zch - 1) / zch;
    stencil_z_f32_kernel<<<dim3(tiles, zc, cgrp), STX * STY, 0, st>>>(
        nx, ny, nz, (float)coef_h2, d, c, X, ldx, Y, ldy, zch, tiles_x, skip);
  } else {
    stencil_kernel<double><<<dim3(tiles, zchunks, c), STX * STY, 0, st>>>(
        nx, ny, nz, coef_h2, d, X, ldx, Y, ldy, zchunk, tiles_x, skip);
  }
  LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t csr_apply_f64(int64_t n, const int64_t* rp, const int32_t* ci,
                          const double* v, int c, const double* X, int64_t ldx,
                          double* Y, int64_t ldy, const int* skip,
                          cudaStream_t st) {
  if (c <= 0) return cudaSuccess;
  const unsigned gx = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((n + 255) / 256, 8 * kNumSMs));
  csr_kernel<<<gx, 256, 0, st>>>(n, rp, ci, v, c, X, ldx, Y, ldy, skip); LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

// two partial sets: the one-launch CG step keeps p.q and r.r apart
size_t cg_part_elems(int64_t n, int nb) { return (size_t)2 * cg_slabs(n) * nb; }

bool cg_step_coop_fits(int64_t n, int nb, const CgState& s) {
  if (nb < 1 || nb > kCoopMaxCols || s.slabs < 1) return false;
  const int64_t sr = (n + s.slabs - 1) / s.slabs;
  if (sr > (int64_t)kCoopRows * 256) return false;
  int dev = 0, sms = 0, per = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, cg_step_coop_kernel, 256, 0) !=
          cudaSuccess)
    return false;
  return coop != 0 && (int64_t)s.slabs * nb <= (int64_t)per * sms;
}

cudaError_t cg_step_coop(int64_t n, int nb, const float* part, int splits, double* X,
                         double* R, double* P, int64_t ld, CgState& s, void* hi, void* lo,
                         int64_t ldb, int epoch, int* err, cudaStream_t st) {
  int64_t sr = (n + s.slabs - 1) / s.slabs;
  __nv_bfloat16* h = (__nv_bfloat16*)hi;
  __nv_bfloat16* l = (__nv_bfloat16*)lo;
  void* args[] = {&n,  &nb, &part, &splits, &X,   &R,     &P,  &ld,
                  &s,  &h,  &l,    &ldb,    &sr, &epoch, &err};
  const cudaError_t e = cudaLaunchCooperativeKernel((const void*)cg_step_coop_kernel,
                                                    dim3(s.slabs, nb), dim3(256), args, 0, st);
  LREP_COUNT_LAUNCH();
  return e;
}

cudaError_t cg_init(int64_t n, int nb, const double* B, int64_t ldb, double* X,
                    double* R, double* P, int64_t ld, double tol, CgState& s,
                    cudaStream_t st) {
  const int slabs = cg_slabs(n);
  s.slabs = slabs;
  const int64_t sr = (n + slabs - 1) / slabs;
  cg_init_kernel<<<dim3(slabs, nb), 256, 0, st>>>(n, nb, B, ldb, X, R, P, ld, tol, s, sr); LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t cg_alpha(int64_t n, int nb, const double* P, const double* Q,
                     int64_t ld, CgState& s, cudaStream_t st) {
  const int64_t sr = (n + s.slabs - 1) / s.slabs;
  cg_alpha_kernel<<<dim3(s.slabs, nb), 256, 0, st>>>(n, nb, P, Q, ld, s, sr); LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t cg_update(int64_t n, int nb, double* X, double* R, const double* P,
                      const double* Q, int64_t ld, CgState& s, cudaStream_t st) {
  const int64_t sr = (n + s.slabs - 1) / s.slabs;
  cg_update_kernel<<<dim3(s.slabs, nb), 256, 0, st>>>(n, nb, X, R, P, Q, ld, s, sr); LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t cg_pdir(int64_t n, int nb, const double* R, double* P, int64_t ld,
                    CgState& s, cudaStream_t st) {
  cg_pdir_kernel<<<dim3(grid_rows(n), nb), 256, 0, st>>>(n, R, P, ld, s); LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t cg_sum_alpha(int64_t n, int nb, const float* part, int splits, const double* P,
                         double* Q, int64_t ld, CgState& s, cudaStream_t st) {
  const int64_t sr = (n + s.slabs - 1) / s.slabs;
  cg_sum_alpha_kernel<<<dim3(s.slabs, nb), 256, 0, st>>>(n, nb, part, splits, P, Q, ld, s, sr);
  LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t cg_pdir_split(int64_t n, int nb, const double* R, double* P, int64_t ld,
                          CgState& s, void* hi, void* lo, int64_t ldb, cudaStream_t st) {
  cg_pdir_split_kernel<<<dim3(grid_rows(n), nb), 256, 0, st>>>(
      n, R, P, ld, s, (__nv_bfloat16*)hi, (__nv_bfloat16*)lo, ldb);
  LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

}  // namespace lrep
