// FP64-accurate dense operator products Y = A X on the bf16 tensor cores by
// error-free slicing (the scheme of Ozaki, Ogita, Oishi and Rump, with
// per-row / per-column power-of-two scales as in its integer-unit variants).
//
// Every float64 value is written as a scale times seven base-2^8 digits:
//   A_ik = 2^e_i   sum_{s=1..7} a_ik^(s) 2^(-8s)   (|a^(1)| <= 256, else <= 128)
//   X_kj = 2^f_j   sum_{t=1..7} x_kj^(t) 2^(-8t)
// where 2^e_i bounds row i of A and 2^f_j column j of X, and the digits are
// the balanced base-256 digits of the nearest integer to A_ik 2^(56 - e_i),
// so the truncation error is at most 2^-57 of the scale.  Digits are integers of at most 9 bits and are
// exact in bfloat16, and so are their products in the fp32 accumulator as
// long as every partial sum stays below 2^24.  The product keeps the 28 digit
// pairs with s + t <= 8 and groups them by level L = s + t:
//   Y_ij = 2^(e_i + f_j) sum_{L=2..8} 2^(-8L) S_L,  S_L = sum_{s+t=L} sum_k a^(s) x^(t).
// The dropped pairs (s + t >= 9) weigh at most ~2^-55.4 per term.
//
// Kernel layout (one CTA per 128 rows and one k-range; M = 128, N = 7C,
// C = 16 or 32 columns; one TMA warp, one MMA warp, C/4 epilogue warps):
//  * The X digit planes of one k-tile sit side by side as a 7C-row bf16
//    operand, so the MMA of A digit s against the first (8 - s) X planes
//    writes its pairs straight into the accumulator columns of their levels
//    (column block L - 2 = s + t - 2); one MMA per A digit and 16 k.
//  * Levels 2..5 must be exact: after every 64-k tile the epilogue warps
//    read them from tensor memory (all partial sums < 2^24 by the digit
//    bounds: at most (L + 1) 2^14 per k), convert to int32, add to
//    per-thread integer sums and zero the columns.  Levels 6..8 weigh
//    <= 2^-48 and stay in the fp32 accumulator for the whole k-range: their
//    rounding errors land below 2^-53 of the result's scale.
//  * Two accumulator regions alternate between k-tiles so that the drain of
//    one overlaps the MMAs of the next.  TMA stages the A digit tiles (one
//    16 KB tile per digit) through a ring and the X digit tile of each
//    k-tile through a second, two-deep ring.
//  * Split-K partials are written in float64 and summed in a fixed order.
// Every mbarrier wait is bounded (about 2 s of SM clock); on expiry the CTA
// records an error code, waits (bounded) for its own TMA copies and MMAs,
// frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "oz.h"
#include "tc.h"
#include "tcgen05.cuh"

namespace lrep {
namespace {

using namespace tc5;

// TMA load of one digit tile: entries [x, x + 64) of rows [y, y + 128) of
// digit plane z (3-D tensor map; rows or entries past the planes' extent
// arrive as zeros and are not read from memory)
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t mbar,
                                            int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
      "l"((uint64_t)map), "r"(mbar), "r"(x), "r"(y), "r"(z)
      : "memory");
}

constexpr int S = kOzSlices;  // digits per value
constexpr int EXACT = 4;      // levels 2..5 drained exactly per k-tile
constexpr int BM = 128, BK = 64;
constexpr int TILE_A = BM * BK * 2;  // one A digit tile: 16 KB
constexpr int MAX_PER = 64;          // k-tiles per split (4096 k)

template <int C>
struct Cfg {
  static constexpr int CTAS = (C == 16) ? 2 : 1;      // resident CTAs per SM
  static constexpr int DRAIN = 4 * (C / 16);           // epilogue warps (16 columns each)
  static constexpr int THREADS = 32 * (2 + DRAIN);
  static constexpr int TILE_B = S * C * BK * 2;        // X digit planes of one k-tile
  static constexpr int NSA = (C == 16) ? 5 : 10;       // A digit stages
  static constexpr int REGION = S * C;                 // TMEM columns per region (7 levels)
  static constexpr int TMEM_COLS = (2 * REGION <= 256) ? 256 : 512;
  static constexpr int SMEM = 1024 + 2 * TILE_B + NSA * TILE_A + 512;
};

template <int C>
__global__ void __launch_bounds__(Cfg<C>::THREADS, Cfg<C>::CTAS)
oz_gemm_kernel(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mX,
               int rows_pad, int kt_per_split, int kt_total, const int* __restrict__ sig,
               const int* __restrict__ tau, double* __restrict__ part, int* __restrict__ err,
               const int* __restrict__ skip) {
  using G = Cfg<C>;
  if (skip && *skip) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* bufB = base;                    // 2 x TILE_B
  uint8_t* bufA = base + 2 * G::TILE_B;    // NSA x TILE_A
  uint64_t* bars = (uint64_t*)(bufA + G::NSA * TILE_A);
  uint64_t* fullA = bars;
  uint64_t* emptyA = bars + G::NSA;
  uint64_t* fullB = bars + 2 * G::NSA;
  uint64_t* emptyB = fullB + 2;
  uint64_t* tfull = emptyB + 2;
  uint64_t* tempty = tfull + 2;
  uint64_t* done = tempty + 2;
  volatile uint32_t* tmem_slot = (volatile uint32_t*)(done + 1);
  // [0] A tiles issued, [1] X tiles issued, [2] A tiles consumed, [3] X tiles consumed
  volatile int* cnt = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile_m = blockIdx.x, split = blockIdx.y;
  const int kt0 = split * kt_per_split;
  const int nk = min(kt_total, kt0 + kt_per_split) - kt0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < G::NSA; ++s) {
      mbar_init(smem_u32(&fullA[s]), 1);
      mbar_init(smem_u32(&emptyA[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&fullB[b]), 1);
      mbar_init(smem_u32(&emptyB[b]), 1);
      mbar_init(smem_u32(&tfull[b]), 1);
      mbar_init(smem_u32(&tempty[b]), 32 * G::DRAIN);
    }
    mbar_init(smem_u32(done), 1);
    for (int i = 0; i < 4; ++i) cnt[i] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32((const void*)tmem_slot), G::TMEM_COLS);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      int ia = 0, ib = 0;
      bool ok = true;
      for (int j = 0; j < nk && ok; ++j) {
        const int b = j & 1;
        if (j >= 2 && !mbar_wait(smem_u32(&emptyB[b]), ((j >> 1) - 1) & 1, err, 11)) break;
        const int k = (kt0 + j) * BK;
        const uint32_t fb = smem_u32(&fullB[b]);
        mbar_expect_tx(fb, G::TILE_B);
        tma_load_2d(smem_u32(bufB + b * G::TILE_B), &mX, fb, k, 0);
        ib = j + 1;
        for (int s = 0; s < S; ++s) {
          const int q = j * S + s, st = q % G::NSA;
          if (q >= G::NSA && !mbar_wait(smem_u32(&emptyA[st]), ((q / G::NSA) - 1) & 1, err, 12)) {
            ok = false;
            break;
          }
          const uint32_t fa = smem_u32(&fullA[st]);
          mbar_expect_tx(fa, TILE_A);
          tma_load_3d(smem_u32(bufA + st * TILE_A), &mA, fa, k, tile_m * BM, s);
          ia = q + 1;
        }
      }
      cnt[0] = ia;
      cnt[1] = ib;
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      int ca = 0, cb = 0;
      bool ok = true;
      for (int j = 0; j < nk && ok; ++j) {
        const int g = j & 1;
        if (j >= 2 && !mbar_wait(smem_u32(&tempty[g]), ((j >> 1) - 1) & 1, err, 13)) break;
        if (!mbar_wait(smem_u32(&fullB[g]), (j >> 1) & 1, err, 14)) break;
        fence_after();
        const uint32_t bb = smem_u32(bufB + g * G::TILE_B);
        for (int s = 0; s < S; ++s) {
          const int q = j * S + s, st = q % G::NSA;
          if (!mbar_wait(smem_u32(&fullA[st]), (q / G::NSA) & 1, err, 15)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t aa = smem_u32(bufA + st * TILE_A);
          const uint32_t d = tmem + (uint32_t)(g * G::REGION + s * C);
          const uint32_t id = idesc_bf16(BM, (S - s) * C);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk)
            mma_bf16(d, sdesc(aa + kk * 32), sdesc(bb + kk * 32), id,
                     (j < 2 && s == 0 && kk == 0) ? 0u : 1u);
          mma_commit(smem_u32(&emptyA[st]));
          ca = q + 1;
        }
        if (!ok) break;
        mma_commit(smem_u32(&emptyB[g]));
        cb = j + 1;
        mma_commit(smem_u32(&tfull[g]));
      }
      cnt[2] = ca;
      cnt[3] = cb;
      mma_commit(smem_u32(done));  // fires once every MMA issued above has completed
    }
    __syncwarp();
  } else {  // warps 2..: accumulator drain, one output row and 16 columns per thread
    const int q4 = warp & 3;            // TMEM lane quarter this warp may access
    const int c0 = ((warp - 2) >> 2) * 16;
    const uint32_t lanes = (uint32_t)(q4 * 32) << 16;
    int acc[EXACT][16];
#pragma unroll
    for (int b = 0; b < EXACT; ++b)
#pragma unroll
      for (int q = 0; q < 16; ++q) acc[b][q] = 0;
    bool ok = true;
    for (int j = 0; j < nk; ++j) {
      const int g = j & 1;
      if (!mbar_wait(smem_u32(&tfull[g]), (j >> 1) & 1, err, 16)) {
        ok = false;
        break;
      }
      fence_after();
      const uint32_t rg = tmem + lanes + (uint32_t)(g * G::REGION + c0);
#pragma unroll
      for (int b = 0; b < EXACT; ++b) {
        uint32_t v[16];
        tmem_ld16(rg + (uint32_t)(b * C), v);
        tmem_ld_wait();
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[b][q] += __float2int_rn(__uint_as_float(v[q]));
      }
#pragma unroll
      for (int b = 0; b < EXACT; ++b) tmem_zero16(rg + (uint32_t)(b * C));
      tmem_st_wait();
      fence_before();
      mbar_arrive(smem_u32(&tempty[g]));
    }
    if (ok) {
      // levels 6..8 of both regions, combined in fp32 (weights 1, 2^-8, 2^-16
      // relative to 2^-48: the rounding stays ~2^-72 of S_6), then
      // Y_ij = 2^(e_i + f_j) (sum_{L=2..5} 2^-8L S_L + 2^-48 low)
      const int row = tile_m * BM + q4 * 32 + lane;
      const int nreg = nk >= 2 ? 2 : 1;
      float low[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) low[q] = 0.0f;
#pragma unroll
      for (int b = S - 1; b >= EXACT; --b) {  // smallest weights first
        const float wgt = ldexpf(1.0f, -8 * (b - EXACT));
        for (int g = 0; g < nreg; ++g) {
          uint32_t v[16];
          tmem_ld16(tmem + lanes + (uint32_t)(g * G::REGION + b * C + c0), v);
          tmem_ld_wait();
#pragma unroll
          for (int q = 0; q < 16; ++q) low[q] += __uint_as_float(v[q]) * wgt;
        }
      }
      const int e = sig[row];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        // levels 2..5 as one exact integer: |V| < 2^41 k < 2^53 for the
        // <= MAX_PER * 64 k of a split, so the conversion below is exact
        const long long V = ((long long)acc[0][q] << 24) + ((long long)acc[1][q] << 16) +
                            ((long long)acc[2][q] << 8) + (long long)acc[3][q];
        const int sc = e + tau[c0 + q];
        double y;
        if (sc - 48 > -1022 && sc - 40 < 1023) {  // scales as normal doubles (4 FP64 ops)
          const double s40 = __longlong_as_double((long long)(1023 + sc - 40) << 52);
          const double s48 = __longlong_as_double((long long)(1023 + sc - 48) << 52);
          y = fma((double)V, s40, (double)low[q] * s48);
        } else {
          y = ldexp((double)V + (double)low[q] * 0x1p-8, sc - 40);
        }
        part[((int64_t)split * C + c0 + q) * rows_pad + row] = y;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // every MMA this CTA issued has completed; no TMA copy is left in flight
    mbar_drain(smem_u32(done), 0, err, 17);
    for (int q = cnt[2]; q < cnt[0]; ++q)
      if (!mbar_drain(smem_u32(&fullA[q % G::NSA]), (q / G::NSA) & 1, err, 18)) break;
    for (int j = cnt[3]; j < cnt[1]; ++j)
      if (!mbar_drain(smem_u32(&fullB[j & 1]), (j >> 1) & 1, err, 19)) break;
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, G::TMEM_COLS);
}

// ---------------------------------------------------------------- slicing
// A float64 x with scale exponent e (|x| < 2^e) becomes N = round(x 2^(56-e))
// (|N| <= 2^56) written as balanced base-256 digits d_1..d_7
// (N = sum_s d_s 2^(8 (7 - s)), d_2..d_7 in [-128, 127], |d_1| <= 256),
// stored as bf16.  Integer arithmetic on the bit pattern only (the FP64
// pipe is the GPU's scarcest unit); non-finite x gives NaN digits.
constexpr uint64_t kAbs = 0x7FFFFFFFFFFFFFFFull, kInf = 0x7FF0000000000000ull;

__device__ __forceinline__ uint16_t small_int_to_bf16(int d) {
  // |d| <= 256 has at most 8 significant bits: the upper half of the fp32
  // pattern is exact
  return (uint16_t)(__float_as_uint((float)d) >> 16);
}

// e with max < 2^e <= 2 max for the largest finite |entry| given by its bit
// pattern (biased exponent E: e = E - 1022, a subnormal max counts as E = 1)
__device__ __forceinline__ int scale_exponent(uint64_t maxbits) {
  return maxbits ? max((int)(maxbits >> 52), 1) - 1022 : 0;
}

__device__ __forceinline__ void write_digits(uint64_t bits, int e, uint16_t* out,
                                             int64_t sstride) {
  const uint64_t a = bits & kAbs;
  if (a >= kInf) {
#pragma unroll
    for (int s = 0; s < S; ++s) out[(int64_t)s * sstride] = 0x7FC0;
    return;
  }
  // |x| = mant 2^(E - 1075); N = round(|x| 2^(56 - e)) = round(mant 2^sh)
  const int E = (int)(a >> 52);
  const int64_t mant = (int64_t)(a & 0xFFFFFFFFFFFFFull) | (E ? (1ll << 52) : 0ll);
  const int sh = max(E, 1) - 1075 + 56 - e;  // <= 3 since |x| < 2^e
  int64_t N;
  if (sh >= 0)
    N = mant << sh;
  else if (sh > -63)
    N = (mant + (1ll << (-sh - 1))) >> (-sh);  // round half away from zero
  else
    N = 0;
  if (bits >> 63) N = -N;
  int d[S];
#pragma unroll
  for (int s = S - 1; s > 0; --s) {
    d[s] = (int)(((N + 128) & 255) - 128);
    N = (N - d[s]) >> 8;  // exact
  }
  d[0] = (int)N;
#pragma unroll
  for (int s = 0; s < S; ++s) out[(int64_t)s * sstride] = small_int_to_bf16(d[s]);
}

constexpr int kChunk = 8192;  // entries of one column per CTA

// largest finite |entry| of each column of a segmented n x ncols block, as
// bit patterns (atomicMax; maxbits zero on entry)
__global__ void __launch_bounds__(256)
oz_colmax_kernel(Segs src, int64_t n, int ncols, unsigned long long* __restrict__ maxbits) {
  const int j = blockIdx.y;
  if (j >= ncols) return;
  const uint64_t* col = (const uint64_t*)src.col(j);
  const int64_t k0 = (int64_t)blockIdx.x * kChunk, k1 = min(n, k0 + kChunk);
  uint64_t m = 0;
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    const uint64_t a = col[k] & kAbs;
    if (a < kInf && a > m) m = a;
  }
  __shared__ uint64_t red[8];
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t t = __shfl_xor_sync(0xffffffffu, m, o);
    m = t > m ? t : m;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = red[w] > m ? red[w] : m;
    if (m) atomicMax(&maxbits[j], (unsigned long long)m);
  }
}

// digit planes of the columns: plane s, column j, entry k at
// dst[s * sstride + j * ld + k]; columns ncols..gridDim.y-1 and entries
// n..ld-1 zero; expo[j] = the column's scale exponent
__global__ void __launch_bounds__(256)
oz_coldigits_kernel(Segs src, int64_t n, int ncols, int64_t ld,
                    const unsigned long long* __restrict__ maxbits, uint16_t* __restrict__ dst,
                    int64_t sstride, int* __restrict__ expo) {
  const int j = blockIdx.y;
  const bool live = j < ncols;
  const int e = live ? scale_exponent(maxbits[j]) : 0;
  if (blockIdx.x == 0 && threadIdx.x == 0 && expo) expo[j] = e;
  const uint64_t* col = live ? (const uint64_t*)src.col(j) : nullptr;
  const int64_t k0 = (int64_t)blockIdx.x * kChunk, k1 = min(ld, k0 + kChunk);
  uint16_t* out = dst + (int64_t)j * ld;
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x)
    write_digits((live && k < n) ? col[k] : 0ull, e, out + k, sstride);
}

// Both passes in one CTA per column when a column fits one chunk (ld <=
// kChunk): the block's maximum, then the digits (a second read that hits
// the cache).  Same exponents and digits as oz_colmax_kernel followed by
// oz_coldigits_kernel.
__global__ void __launch_bounds__(256)
oz_colslice_kernel(Segs src, int64_t n, int ncols, int64_t ld, uint16_t* __restrict__ dst,
                   int64_t sstride, int* __restrict__ expo) {
  const int j = blockIdx.y;
  const bool live = j < ncols;
  const uint64_t* col = live ? (const uint64_t*)src.col(j) : nullptr;
  uint64_t m = 0;
  if (live)
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
      const uint64_t a = col[k] & kAbs;
      if (a < kInf && a > m) m = a;
    }
  __shared__ uint64_t red[8];
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t t = __shfl_xor_sync(0xffffffffu, m, o);
    m = t > m ? t : m;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  m = red[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = red[w] > m ? red[w] : m;
  const int e = live ? scale_exponent(m) : 0;
  if (threadIdx.x == 0 && expo) expo[j] = e;
  uint16_t* out = dst + (int64_t)j * ld;
  for (int64_t k = threadIdx.x; k < ld; k += blockDim.x)
    write_digits((live && k < n) ? col[k] : 0ull, e, out + k, sstride);
}

// Transposing slicer for a tall left operand: rows r of a segmented n x k
// block become digit rows dst[s * sstride + r * ldk + kk] (per-row scale
// expo[r]); rows n..gridDim.x*kRows-1 and entries k..ldk-1 zero.
constexpr int kRows = 32;
__global__ void __launch_bounds__(256)
oz_rowslice_kernel(Segs src, int64_t n, int k, int64_t ldk, uint16_t* __restrict__ dst,
                   int64_t sstride, int* __restrict__ expo) {
  extern __shared__ uint64_t tile[];  // kRows x k, row-major
  const int64_t r0 = (int64_t)blockIdx.x * kRows;
  for (int e = threadIdx.x; e < kRows * k; e += blockDim.x) {
    const int rr = e % kRows, kk = e / kRows;  // consecutive threads: consecutive rows
    const int64_t r = r0 + rr;
    tile[rr * k + kk] = (r < n) ? ((const uint64_t*)src.col(kk))[r] : 0ull;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ int rexp[kRows];
  for (int rr = warp; rr < kRows; rr += (int)(blockDim.x >> 5)) {
    uint64_t m = 0;
    for (int kk = lane; kk < k; kk += 32) {
      const uint64_t a = tile[rr * k + kk] & kAbs;
      if (a < kInf && a > m) m = a;
    }
    for (int o = 16; o > 0; o >>= 1) {
      const uint64_t t = __shfl_xor_sync(0xffffffffu, m, o);
      m = t > m ? t : m;
    }
    if (lane == 0) {
      rexp[rr] = scale_exponent(m);
      if (expo) expo[r0 + rr] = rexp[rr];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kRows * ldk; e += blockDim.x) {
    const int rr = (int)(e / ldk), kk = (int)(e % ldk);
    write_digits(kk < k ? tile[rr * k + kk] : 0ull, rexp[rr],
                 dst + (r0 + rr) * ldk + kk, sstride);
  }
}

// Y[i, j] = alpha Y[i, j] + beta sum_z part[z][j][i] (fixed order; alpha = 0
// does not read Y)
__global__ void oz_reduce_kernel(int64_t nrows, int c, int C, int splits, int64_t rows_pad,
                                 const double* __restrict__ part, double* __restrict__ Y,
                                 int64_t ldy, double alpha, double beta,
                                 const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t tot = nrows * c;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / nrows, i = e % nrows;
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += part[((int64_t)z * C + j) * rows_pad + i];
    Y[i + j * ldy] = (alpha == 0.0) ? beta * s : fma(alpha, Y[i + j * ldy], beta * s);
  }
}

// k-tiles per split: fewest waves x (tiles per CTA + pipeline fill), at most
// MAX_PER (keeps the per-split integer level sums exact)
int oz_per(int64_t row_tiles, int64_t kt, int ctas_per_sm) {
  const int64_t slots = (int64_t)ctas_per_sm * kNumSMs;
  int64_t best = -1, best_cost = 0;
  for (int64_t per = 1; per <= std::min<int64_t>(kt, MAX_PER); ++per) {
    const int64_t s = (kt + per - 1) / per;
    const int64_t waves = (row_tiles * s + slots - 1) / slots;
    const int64_t cost = waves * (per + 2);
    if (best < 0 || cost <= best_cost) {
      best = per;
      best_cost = cost;
    }
  }
  return (int)best;
}

bool make_map(CUtensorMap* map, const void* base, int64_t inner, int64_t outer, int64_t ld,
              int box_outer) {
  return tc_make_map(map, base, inner, outer, ld, BK, box_outer);
}

// signature of cuTensorMapEncodeTiled (driver API, obtained at run time)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Descriptor of left-operand digit planes: plane s, row r, entry kk at
// base[(s * rows + r) * ldk + kk] (ldk a multiple of 8), read in boxes of
// 64 entries x 128 rows x 1 plane with the 128-byte swizzle.  Rows past
// `rows` (a Gram with fewer than 128 columns) and entries past ldk (a short
// contraction) are filled with zeros by the copy, so the planes are stored
// without padding to the tile.
bool make_planes_map(CUtensorMap* map, const void* base, int64_t ldk, int64_t rows) {
  static const EncodeTiledFn fn = [] {
    cudaDriverEntryPointQueryResult q;
    void* f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (EncodeTiledFn)f;
    return (EncodeTiledFn) nullptr;
  }();
  if (!fn || ldk % 8 != 0 || rows <= 0) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)ldk, (cuuint64_t)rows, (cuuint64_t)S};
  const cuuint64_t strides[2] = {(cuuint64_t)ldk * 2, (cuuint64_t)(rows * ldk * 2)};
  const cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)BM, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides,
            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

Segs segs_sub(const Segs& s, int j0, int cnt) {
  Segs o{};
  o.nseg = 0;
  for (int q = 0; q < s.nseg && cnt > 0; ++q) {
    if (j0 >= s.cols[q]) {
      j0 -= s.cols[q];
      continue;
    }
    const int take = std::min(cnt, s.cols[q] - j0);
    o.ptr[o.nseg] = s.ptr[q] + (int64_t)j0 * s.ld[q];
    o.ld[o.nseg] = s.ld[q];
    o.cols[o.nseg] = take;
    o.nseg++;
    cnt -= take;
    j0 = 0;
  }
  return o;
}

unsigned grid1(int64_t tot) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((tot + 255) / 256, 8 * kNumSMs));
}

// digit planes of the c columns of X (k entries each, padded to ldk) for a
// group of width C, into xs / tau (maxbits: C words of scratch)
cudaError_t slice_columns(const Segs& X, int64_t k, int c, int C, int64_t ldk, uint16_t* xs,
                          int* tau, unsigned long long* maxbits, cudaStream_t st) {
  if (ldk <= kChunk) {  // one CTA per column: both passes in one launch
    oz_colslice_kernel<<<dim3(1, (unsigned)C), 256, 0, st>>>(X, k, c, ldk, xs,
                                                            (int64_t)C * ldk, tau);
    LREP_COUNT_LAUNCH();
    return cudaGetLastError();
  }
  cudaError_t e = cudaMemsetAsync(maxbits, 0, sizeof(unsigned long long) * C, st);
  if (e != cudaSuccess) return e;
  const unsigned chunks_n = (unsigned)std::max<int64_t>(1, (k + kChunk - 1) / kChunk);
  const unsigned chunks_ld = (unsigned)std::max<int64_t>(1, (ldk + kChunk - 1) / kChunk);
  oz_colmax_kernel<<<dim3(chunks_n, (unsigned)c), 256, 0, st>>>(X, k, c, maxbits);
  LREP_COUNT_LAUNCH();
  oz_coldigits_kernel<<<dim3(chunks_ld, (unsigned)C), 256, 0, st>>>(X, k, c, ldk, maxbits, xs,
                                                                    (int64_t)C * ldk, tau);
  LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

// one column group: Y[:, 0:c] = alpha Y + beta A X for the sliced left
// operand A (digit planes behind the 3-D map mapA, row exponents sig for
// rows_pad rows) and the c <= C columns of X
template <int C>
cudaError_t oz_group(const CUtensorMap& mapA, int64_t rows, int64_t rows_pad, int64_t ldk,
                     const int* sig, const Segs& X, int64_t k, int c, double* Y, int64_t ldy,
                     double alpha, double beta, uint8_t* ws, int* err, const int* skip,
                     cudaStream_t st) {
  using G = Cfg<C>;
  uint16_t* xs = (uint16_t*)ws;
  uint8_t* q = ws + (((size_t)S * C * ldk * 2 + 255) & ~(size_t)255);
  int* tau = (int*)q;
  unsigned long long* maxbits = (unsigned long long*)(q + 256);
  double* part = (double*)(q + 1024);
  cudaError_t e = slice_columns(X, k, c, C, ldk, xs, tau, maxbits, st);
  if (e != cudaSuccess) return e;
  CUtensorMap mx;
  if (!make_map(&mx, xs, ldk, (int64_t)S * C, ldk, S * C)) return cudaErrorInvalidValue;
  const int64_t kt = ldk / BK, rt = rows_pad / BM;
  const int per = oz_per(rt, kt, G::CTAS);
  const int splits = (int)((kt + per - 1) / per);
  static const cudaError_t attr = cudaFuncSetAttribute(
      oz_gemm_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
  if (attr != cudaSuccess) return attr;
  dim3 grid((unsigned)rt, (unsigned)splits);
  oz_gemm_kernel<C><<<grid, G::THREADS, G::SMEM, st>>>(mapA, mx, (int)rows_pad, per, (int)kt,
                                                       sig, tau, part, err, skip);
  LREP_COUNT_LAUNCH();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  oz_reduce_kernel<<<grid1(rows * c), 256, 0, st>>>(rows, c, C, splits, rows_pad, part, Y, ldy,
                                                    alpha, beta, skip);
  LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

size_t group_ws_bytes(int64_t rows, int64_t k, int C, int ctas) {
  const int64_t ldk = oz_ldk(k), rp = oz_rows_pad(rows);
  const int64_t kt = ldk / BK, rt = rp / BM;
  const int per = oz_per(rt, kt, ctas);
  const int64_t splits = (kt + per - 1) / per;
  return (((size_t)S * C * ldk * 2 + 255) & ~(size_t)255) + 1024 +
         (size_t)splits * C * rp * sizeof(double) + 256;
}

size_t groups_ws_bytes(int64_t rows, int64_t k, int c) {
  size_t b = group_ws_bytes(rows, k, 16, Cfg<16>::CTAS);
  if (c > 16) b = std::max(b, group_ws_bytes(rows, k, 32, Cfg<32>::CTAS));
  return b;
}

// all column groups of Y = alpha Y + beta A X
cudaError_t oz_groups(const CUtensorMap& mapA, int64_t rows, int64_t rows_pad, int64_t ldk,
                      const int* sig, const Segs& X, int64_t k, int c, double* Y, int64_t ldy,
                      double alpha, double beta, uint8_t* ws, int* err, const int* skip,
                      cudaStream_t st) {
  for (int j0 = 0; j0 < c;) {
    const int left = c - j0;
    const Segs Xg = segs_sub(X, j0, std::min(left, 32));
    cudaError_t e;
    if (left <= 16) {
      e = oz_group<16>(mapA, rows, rows_pad, ldk, sig, Xg, k, left, Y + (int64_t)j0 * ldy, ldy,
                       alpha, beta, ws, err, skip, st);
      j0 += left;
    } else {
      const int g = std::min(left, 32);
      e = oz_group<32>(mapA, rows, rows_pad, ldk, sig, Xg, k, g, Y + (int64_t)j0 * ldy, ldy,
                       alpha, beta, ws, err, skip, st);
      j0 += g;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

int64_t oz_ldk(int64_t n) { return ((n + BK - 1) / BK) * BK; }
int64_t oz_rows_pad(int64_t n) { return ((n + BM - 1) / BM) * BM; }

size_t oz_operand_bytes(int64_t n) {
  return (size_t)S * oz_rows_pad(n) * oz_ldk(n) * 2 + (size_t)oz_rows_pad(n) * sizeof(int) +
         (size_t)oz_rows_pad(n) * 8 + 512;
}

cudaError_t oz_slice_operator(int64_t n, const double* A, int64_t lda, OzOperand* o,
                              cudaStream_t st) {
  o->n = n;
  o->ldk = oz_ldk(n);
  o->rows_pad = oz_rows_pad(n);
  const size_t planes = (size_t)S * o->rows_pad * o->ldk;
  o->sig = (int*)((uint8_t*)o->slices + planes * 2);
  unsigned long long* maxbits =
      (unsigned long long*)align256((size_t)(o->sig + o->rows_pad));
  // row i of the symmetric A is its column i
  cudaError_t e = slice_columns(seg1(A, lda, (int)n), n, (int)n, (int)o->rows_pad, o->ldk,
                                (uint16_t*)o->slices, o->sig, maxbits, st);
  if (e != cudaSuccess) return e;
  if (!make_planes_map(&o->map, o->slices, o->ldk, o->rows_pad)) return cudaErrorInvalidValue;
  return cudaSuccess;
}

size_t oz_ws_bytes(int64_t n, int c) { return groups_ws_bytes(n, n, c); }

cudaError_t oz_apply(const OzOperand& A, int c, const double* X, int64_t ldx, double* Y,
                     int64_t ldy, void* ws, size_t ws_bytes, int* err, const int* skip,
                     cudaStream_t st) {
  if (c <= 0) return cudaSuccess;
  if (ws_bytes < oz_ws_bytes(A.n, c)) return cudaErrorInvalidValue;
  uint8_t* w = (uint8_t*)align256((size_t)ws);
  return oz_groups(A.map, A.n, A.rows_pad, A.ldk, A.sig, seg1(X, ldx, c), A.n, c, Y, ldy, 0.0,
                   1.0, w, err, skip, st);
}

// ------------------------------------------------ tall-skinny Gram / update
size_t oz_gram_ws_bytes(int64_t n, int a, int b) {
  const int64_t rp = oz_rows_pad(a), ldk = oz_ldk(n);
  return align256((size_t)S * rp * ldk * 2) + align256((size_t)rp * 12) + 512 +
         groups_ws_bytes(a, n, b);
}

cudaError_t oz_gram(int64_t n, const Segs& A, const Segs& B, double* G, int64_t ldg, void* ws,
                    size_t ws_bytes, int* err, cudaStream_t st) {
  const int a = A.total(), b = B.total();
  if (a <= 0 || b <= 0) return cudaSuccess;
  if (ws_bytes < oz_gram_ws_bytes(n, a, b)) return cudaErrorInvalidValue;
  const int64_t rp = oz_rows_pad(a), ldk = oz_ldk(n);
  uint8_t* w = (uint8_t*)align256((size_t)ws);
  uint16_t* planes = (uint16_t*)w;
  w += align256((size_t)S * rp * ldk * 2);
  int* sig = (int*)w;
  unsigned long long* maxbits = (unsigned long long*)(w + align256((size_t)rp * 4));
  w += align256((size_t)rp * 12) + 512;
  // rows of A^T = columns of A: planes of exactly a rows (the copy fills
  // the tile's rows a..127 with zeros); the exponents of those rows are 0
  cudaError_t e = slice_columns(A, n, a, a, ldk, planes, sig, maxbits, st);
  if (e == cudaSuccess && rp > a)
    e = cudaMemsetAsync(sig + a, 0, (size_t)(rp - a) * sizeof(int), st);
  if (e != cudaSuccess) return e;
  CUtensorMap map;
  if (!make_planes_map(&map, planes, ldk, a)) return cudaErrorInvalidValue;
  return oz_groups(map, a, rp, ldk, sig, B, n, b, G, ldg, 0.0, 1.0, w, err, nullptr, st);
}

size_t oz_update_ws_bytes(int64_t n, int k, int c) {
  const int64_t rp = oz_rows_pad(n), ldk = oz_ldk(k);
  return align256((size_t)S * rp * ldk * 2) + align256((size_t)rp * 4) + 512 +
         groups_ws_bytes(n, k, c);
}

cudaError_t oz_update(int64_t n, int k, int c, double alpha, const Segs& A, const double* B,
                      int64_t ldb, double beta, double* C, int64_t ldc, void* ws,
                      size_t ws_bytes, int* err, cudaStream_t st) {
  if (c <= 0 || n <= 0) return cudaSuccess;
  if (k <= 0 || beta == 0.0) return cudaErrorInvalidValue;
  if (ws_bytes < oz_update_ws_bytes(n, k, c)) return cudaErrorInvalidValue;
  const int64_t rp = oz_rows_pad(n), ldk = oz_ldk(k);
  uint8_t* w = (uint8_t*)align256((size_t)ws);
  uint16_t* planes = (uint16_t*)w;
  w += align256((size_t)S * rp * ldk * 2);
  int* sig = (int*)w;
  w += align256((size_t)rp * 4) + 512;
  const size_t smem = (size_t)kRows * k * sizeof(uint64_t);
  static const cudaError_t attr = cudaFuncSetAttribute(
      oz_rowslice_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (attr != cudaSuccess) return attr;
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  // left planes with the contraction padded to 8 entries, not to the
  // 64-entry tile: the copy fills entries k8..63 of the last k-tile with zeros
  const int64_t k8 = ((int64_t)k + 7) / 8 * 8;
  oz_rowslice_kernel<<<(unsigned)(rp / kRows), 256, smem, st>>>(A, n, k, k8, planes, rp * k8,
                                                                sig);
  LREP_COUNT_LAUNCH();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  CUtensorMap map;
  if (!make_planes_map(&map, planes, k8, rp)) return cudaErrorInvalidValue;
  return oz_groups(map, n, rp, ldk, sig, seg1(B, ldb, c), k, c, C, ldc, alpha, beta, w, err,
                   nullptr, st);
}

}  // namespace lrep
