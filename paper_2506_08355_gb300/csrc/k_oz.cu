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
          tma_load_2d(smem_u32(bufA + st * TILE_A), &mA, fa, k, s * rows_pad + tile_m * BM);
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
    mbar_wait(smem_u32(done), 0, err, 17);
    for (int q = cnt[2]; q < cnt[0]; ++q)
      if (!mbar_wait(smem_u32(&fullA[q % G::NSA]), (q / G::NSA) & 1, err, 18)) break;
    for (int j = cnt[3]; j < cnt[1]; ++j)
      if (!mbar_wait(smem_u32(&fullB[j & 1]), (j >> 1) & 1, err, 19)) break;
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, G::TMEM_COLS);
}

// One CTA per column j of a column-major block (entries k = 0..n-1 of column
// j contiguous, leading dimension lds): the exponent e with max_k |src_kj| <
// 2^e (0 for a zero column) and the base-2^8 digits of src_kj / 2^e:
// N = round(src_kj 2^(56 - e)) (|N| <= 2^56), written as balanced digits
// N = sum_s d_s 2^(8 (7 - s)), d_2..d_7 in [-128, 127] and |d_1| <= 256,
// stored as bf16 at dst[(s - 1) * sstride + j * ld + k].  Columns j >= ncols
// and entries n <= k < ld are written as zeros, non-finite entries as NaN
// digits.  Everything runs in integer arithmetic on the float64 bit pattern
// (the FP64 pipe is the GPU's scarcest unit).
__device__ __forceinline__ uint16_t small_int_to_bf16(int d) {
  // |d| <= 256 has at most 8 significant bits: the upper half of the fp32
  // pattern is exact
  return (uint16_t)(__float_as_uint((float)d) >> 16);
}

__global__ void __launch_bounds__(256)
oz_slice_kernel(int64_t n, int ncols, const double* __restrict__ src, int64_t lds,
                uint16_t* __restrict__ dst, int64_t ld, int64_t sstride,
                int* __restrict__ expo) {
  constexpr uint64_t kAbs = 0x7FFFFFFFFFFFFFFFull, kInf = 0x7FF0000000000000ull;
  const int j = blockIdx.x;
  const bool live = j < ncols;
  const uint64_t* col = (const uint64_t*)(src + (int64_t)j * lds);
  uint64_t m = 0;  // largest finite |entry| (bit patterns of non-negative doubles order like them)
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
  // e: max < 2^e <= 2 max (biased exponent field E of max: e = E - 1022;
  // a subnormal max counts as E = 1)
  int e = 0;
  if (m > 0) e = max((int)(m >> 52), 1) - 1022;
  if (threadIdx.x == 0 && expo) expo[j] = e;
  uint16_t* out = dst + (int64_t)j * ld;
  for (int64_t k = threadIdx.x; k < ld; k += blockDim.x) {
    const uint64_t bits = (live && k < n) ? col[k] : 0ull;
    const uint64_t a = bits & kAbs;
    if (a >= kInf) {
#pragma unroll
      for (int s = 0; s < S; ++s) out[(int64_t)s * sstride + k] = 0x7FC0;
      continue;
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
    for (int s = 0; s < S; ++s) out[(int64_t)s * sstride + k] = small_int_to_bf16(d[s]);
  }
}

__global__ void oz_reduce_kernel(int64_t n, int c, int C, int splits, int64_t rows_pad,
                                 const double* __restrict__ part, double* __restrict__ Y,
                                 int64_t ldy, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t tot = n * c;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / n, i = e % n;
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += part[((int64_t)z * C + j) * rows_pad + i];
    Y[i + j * ldy] = s;
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

template <int C>
cudaError_t oz_group(const OzOperand& A, int c, const double* X, int64_t ldx, double* Y,
                     int64_t ldy, uint8_t* ws, int* err, const int* skip, cudaStream_t st) {
  using G = Cfg<C>;
  const int64_t ldk = A.ldk, rp = A.rows_pad, n = A.n;
  __nv_bfloat16* xs = (__nv_bfloat16*)ws;
  int* tau = (int*)(ws + (size_t)S * C * ldk * 2);
  double* part = (double*)(ws + (((size_t)S * C * ldk * 2 + 4 * 32 + 255) & ~(size_t)255));
  oz_slice_kernel<<<C, 256, 0, st>>>(n, c, X, ldx, (uint16_t*)xs, ldk, (int64_t)C * ldk, tau);
  LREP_COUNT_LAUNCH();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  CUtensorMap mx;
  if (!make_map(&mx, xs, ldk, (int64_t)S * C, ldk, S * C)) return cudaErrorInvalidValue;
  const int64_t kt = ldk / BK, rt = rp / BM;
  const int per = oz_per(rt, kt, G::CTAS);
  const int splits = (int)((kt + per - 1) / per);
  static const cudaError_t attr = cudaFuncSetAttribute(
      oz_gemm_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
  if (attr != cudaSuccess) return attr;
  dim3 grid((unsigned)rt, (unsigned)splits);
  oz_gemm_kernel<C><<<grid, G::THREADS, G::SMEM, st>>>(A.map, mx, (int)rp, per, (int)kt, A.sig, tau,
                                                 part, err, skip);
  LREP_COUNT_LAUNCH();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t tot = n * c;
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((tot + 255) / 256, 8 * kNumSMs));
  oz_reduce_kernel<<<g, 256, 0, st>>>(n, c, C, splits, rp, part, Y, ldy, skip);
  LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

size_t group_ws_bytes(int64_t n, int C, int ctas) {
  const int64_t ldk = oz_ldk(n), rp = oz_rows_pad(n);
  const int64_t kt = ldk / BK, rt = rp / BM;
  const int per = oz_per(rt, kt, ctas);
  const int64_t splits = (kt + per - 1) / per;
  return (((size_t)S * C * ldk * 2 + 4 * 32 + 255) & ~(size_t)255) +
         (size_t)splits * C * rp * sizeof(double) + 256;
}

}  // namespace

int64_t oz_ldk(int64_t n) { return ((n + BK - 1) / BK) * BK; }
int64_t oz_rows_pad(int64_t n) { return ((n + BM - 1) / BM) * BM; }

size_t oz_operand_bytes(int64_t n) {
  return (size_t)S * oz_rows_pad(n) * oz_ldk(n) * 2 + (size_t)oz_rows_pad(n) * sizeof(int) + 256;
}

cudaError_t oz_slice_operator(int64_t n, const double* A, int64_t lda, OzOperand* o,
                              cudaStream_t st) {
  o->n = n;
  o->ldk = oz_ldk(n);
  o->rows_pad = oz_rows_pad(n);
  const size_t planes = (size_t)S * o->rows_pad * o->ldk;
  o->sig = (int*)((uint8_t*)o->slices + planes * 2);
  // row i of the symmetric A is its column i
  oz_slice_kernel<<<(unsigned)o->rows_pad, 256, 0, st>>>(
      n, (int)n, A, lda, (uint16_t*)o->slices, o->ldk, o->rows_pad * o->ldk, o->sig);
  LREP_COUNT_LAUNCH();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (!make_map(&o->map, o->slices, o->ldk, (int64_t)S * o->rows_pad, o->ldk, BM))
    return cudaErrorInvalidValue;
  return cudaSuccess;
}

size_t oz_ws_bytes(int64_t n, int c) {
  size_t b = group_ws_bytes(n, 16, Cfg<16>::CTAS);
  if (c > 16) b = std::max(b, group_ws_bytes(n, 32, Cfg<32>::CTAS));
  return b;
}

cudaError_t oz_apply(const OzOperand& A, int c, const double* X, int64_t ldx, double* Y,
                     int64_t ldy, void* ws, size_t ws_bytes, int* err, const int* skip,
                     cudaStream_t st) {
  if (c <= 0) return cudaSuccess;
  if (ws_bytes < oz_ws_bytes(A.n, c)) return cudaErrorInvalidValue;
  uint8_t* w = (uint8_t*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  for (int j0 = 0; j0 < c;) {
    const int left = c - j0;
    cudaError_t e;
    if (left <= 16) {
      e = oz_group<16>(A, left, X + (int64_t)j0 * ldx, ldx, Y + (int64_t)j0 * ldy, ldy, w, err,
                       skip, st);
      j0 += left;
    } else {
      const int g = std::min(left, 32);
      e = oz_group<32>(A, g, X + (int64_t)j0 * ldx, ldx, Y + (int64_t)j0 * ldy, ldy, w, err,
                       skip, st);
      j0 += g;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace lrep
