// Tensor-core operator product for the inexact CG solves of eq. block_GS:
//   Y (n x c, fp64) ~= A X = (A_hi + A_lo)(X_hi + X_lo)
//                   ~= A_hi X_hi + A_hi X_lo + A_lo X_hi
// with A (symmetric K or M) split once into bfloat16 hi + lo parts and X
// split per call.  The three products accumulate in one fp32 tensor-memory
// accumulator (tcgen05.mma kind::f16, M = 128 rows, N = columns rounded up
// to 16).  Operand tiles (64 k-values = 128 bytes per row, 128-byte
// swizzle) are staged by TMA through a 3-stage mbarrier pipeline (two CTAs
// per SM); one thread issues TMA, one issues MMA, and four warps drain the
// accumulator with tcgen05.ld.  Split-K partials (fp32) are summed in a fixed order in
// fp64.  Relative error ~ 2^-16 plus fp32 accumulation, far below the CG
// tolerance (1e-2) that these products serve.
//
// Every mbarrier wait is bounded (about 2 s of SM clock); on expiry the CTA
// records an error code, drains its own TMA copies (bounded), frees its
// tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "tc.h"
#include "tcgen05.cuh"

namespace lrep {
namespace {

constexpr int BM = 128;              // output rows per CTA = TMEM lanes
constexpr int BK = 64;               // k per stage: 64 bf16 = 128 B (one swizzle row)
constexpr int STAGES = 3;             // 3 x ~36 KB: two CTAs per SM
constexpr int TILE_A = BM * BK * 2;  // 16 KB

using namespace tc5;

__global__ void __launch_bounds__(128, 2)
bf16x3_kernel(const __grid_constant__ CUtensorMap mAhi, const __grid_constant__ CUtensorMap mAlo,
              const __grid_constant__ CUtensorMap mXhi, const __grid_constant__ CUtensorMap mXlo,
              int n, int c, int N, int kt_per_split, int kt_total, int tmem_cols,
              float* __restrict__ part, int* __restrict__ err, const int* __restrict__ skip) {
  if (skip && *skip) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tile_x = N * BK * 2;  // X tile bytes
  const int stage_bytes = ((2 * TILE_A + 2 * tile_x) + 1023) & ~1023;
  uint64_t* bars = (uint64_t*)(base + STAGES * stage_bytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + STAGES;
  uint64_t* done = bars + 2 * STAGES;
  volatile uint32_t* tmem_slot = (volatile uint32_t*)(bars + 2 * STAGES + 1);
  volatile int* counts = (volatile int*)(tmem_slot + 1);  // [0] issued [1] consumed

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile_m = blockIdx.x, split = blockIdx.y;
  const int kt0 = split * kt_per_split;
  const int nk = min(kt_total, kt0 + kt_per_split) - kt0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(done), 1);
    counts[0] = 0;
    counts[1] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32((const void*)tmem_slot)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;
  const uint32_t expect = (uint32_t)(2 * TILE_A + 2 * tile_x);

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      int it = 0;
      for (; it < nk; ++it) {
        const int s = it % STAGES;
        if (it >= STAGES &&
            !mbar_wait(smem_u32(&empty[s]), ((it / STAGES) - 1) & 1, err, 1))
          break;
        if (*(volatile int*)err) break;
        uint8_t* st = base + s * stage_bytes;
        const uint32_t fb = smem_u32(&full[s]);
        mbar_expect_tx(fb, expect);
        const int k = (kt0 + it) * BK;
        tma_load_2d(smem_u32(st), &mAhi, fb, k, tile_m * BM);
        tma_load_2d(smem_u32(st + TILE_A), &mAlo, fb, k, tile_m * BM);
        tma_load_2d(smem_u32(st + 2 * TILE_A), &mXhi, fb, k, 0);
        tma_load_2d(smem_u32(st + 2 * TILE_A + tile_x), &mXlo, fb, k, 0);
      }
      counts[0] = it;
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) |
                             ((uint32_t)(N >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
      int it = 0;
      for (; it < nk; ++it) {
        const int s = it % STAGES;
        if (!mbar_wait(smem_u32(&full[s]), (it / STAGES) & 1, err, 2)) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        uint8_t* st = base + s * stage_bytes;
        const uint32_t ahi = smem_u32(st), alo = smem_u32(st + TILE_A);
        const uint32_t xhi = smem_u32(st + 2 * TILE_A), xlo = smem_u32(st + 2 * TILE_A + tile_x);
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint32_t off = kk * 32;  // 16 bf16 along k
          mma_bf16(tmem, sdesc(ahi + off), sdesc(xhi + off), idesc, (it | kk) ? 1u : 0u);
          mma_bf16(tmem, sdesc(ahi + off), sdesc(xlo + off), idesc, 1u);
          mma_bf16(tmem, sdesc(alo + off), sdesc(xhi + off), idesc, 1u);
        }
        mma_commit(smem_u32(&empty[s]));
      }
      counts[1] = it;
      mma_commit(smem_u32(done));
    }
    __syncwarp();
  }
  // epilogue: TMEM lane = output row; warp w owns lanes 32w..32w+31
  const bool ok = mbar_drain(smem_u32(done), 0, err, 3);
  asm volatile("tcgen05.fence::after_thread_sync;");
  const int row = tile_m * BM + warp * 32 + lane;
  if (ok) {
    for (int j0 = 0; j0 < N; j0 += 16) {
      uint32_t v[16];
      const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)j0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32"
          " {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
            "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
            "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(ta));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < n) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int j = j0 + q;
          if (j < c) part[((int64_t)split * c + j) * n + row] = __uint_as_float(v[q]);
        }
      }
    }
  }
  __syncthreads();
  // drain TMA copies that were issued but not consumed (error path only)
  if (threadIdx.x == 0) {
    for (int it = counts[1]; it < counts[0]; ++it)
      if (!mbar_drain(smem_u32(&full[it % STAGES]), (it / STAGES) & 1, err, 4)) break;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(tmem_cols));
}

// ---------------------------------------------------------------------------
// Symmetric form: A = A^T, so only the tiles A_IJ with I <= J (128 x 128) are
// read, and each off-diagonal tile serves both Y_I += A_IJ X_J and
// Y_J += A_IJ^T X_I (the second MMA reads the same shared-memory tile as an
// MN-major operand: no transposed copy).  HBM traffic is about half the
// matrix.
//
// Work: items are super-blocks of b x b tiles (super-rows S <= C; an
// off-diagonal item keeps 2b fp32 accumulators in tensor memory, b for its
// rows I and b for its columns J; a diagonal item b).  The tiles of all
// items, in item order, are split evenly over the persistent CTAs; the run
// of one item inside one CTA's range is a segment, whose accumulators are
// written once to its own partial slots (the host lists, per super-row,
// the slots that hold its rows).  The fixed-order float64 sum of the slots
// keeps results deterministic.
//
// Pipelines: the two planes (hi, lo) of a tile are separate 32 KB stages of
// a 5- or 6-deep ring, the tile's X boxes (X_J and X_I, hi and lo) a 2-deep
// ring; operator boxes three tiles ahead are prefetched into L2.  One
// thread issues TMA, one issues MMA, four warps drain and zero the
// accumulators of each segment.
constexpr int SYM_TILE = 128;
constexpr int SYM_BOX = BM * BK * 2;  // one 128 x 64 bf16 box: 16 KB
constexpr int SYM_PLANE = 2 * SYM_BOX;  // one plane of a tile: 32 KB
constexpr int SYM_PREFETCH = 3;         // tiles prefetched into L2 ahead of their load

template <int N>
struct SymCfg {
  static constexpr int XBOX = N * BK * 2;      // one N x 64 bf16 box
  static constexpr int XSTAGE = 8 * XBOX;      // X_J, X_I x (hi, lo) x 2 boxes
  static constexpr int NA = N <= 16 ? 6 : 5;   // operator-plane stages
  static constexpr int SMEM = NA * SYM_PLANE + 2 * XSTAGE;
};

__host__ __device__ inline void sym_item(int q, int Tsb, int& S, int& C) {
  const int noff = Tsb * (Tsb - 1) / 2;
  if (q >= noff) {
    S = C = q - noff;
    return;
  }
  int s = 0, rem = q;
  while (rem >= Tsb - 1 - s) {
    rem -= Tsb - 1 - s;
    ++s;
  }
  S = s;
  C = s + 1 + rem;
}

// next tile of item (S, C) in issue order (row i, then column j); returns
// false past the last one
__host__ __device__ inline bool sym_next(int S, int C, int b, int T, int& i, int& j) {
  const bool diag = (S == C);
  for (;;) {
    ++j;
    if (j >= b) {
      ++i;
      if (i >= b) return false;
      j = diag ? i : 0;
    }
    if (S * b + i < T && C * b + j < T) return true;
  }
}

// Walks the tiles [t0, t1) of the global order (items in order, their tiles
// in issue order); every role of the kernel walks the same sequence.
struct SymCursor {
  int64_t t, t1;
  int q, S, C, i, j;
  const int* item_start;
  int Tsb, b, T;
  __device__ void start(int64_t t0_, int64_t t1_, const int* is, int items, int Tsb_, int b_,
                        int T_) {
    t = t0_;
    t1 = t1_;
    item_start = is;
    Tsb = Tsb_;
    b = b_;
    T = T_;
    if (t >= t1) return;
    int lo = 0, hi = items;  // item with item_start[q] <= t < item_start[q + 1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (is[mid] <= t) lo = mid;
      else hi = mid;
    }
    q = lo;
    sym_item(q, Tsb, S, C);
    i = 0;
    j = -1;
    sym_next(S, C, b, T, i, j);
    for (int64_t k = is[q]; k < t; ++k) sym_next(S, C, b, T, i, j);
  }
  __device__ bool valid() const { return t < t1; }
  // true when the tile just passed was the last of its segment
  __device__ bool next() {
    ++t;
    if (t >= t1) return true;
    if (t >= item_start[q + 1]) {
      ++q;
      sym_item(q, Tsb, S, C);
      i = 0;
      j = -1;
      sym_next(S, C, b, T, i, j);
      return true;
    }
    sym_next(S, C, b, T, i, j);
    return false;
  }
};

// The MMAs of one operator plane of a tile: the descriptors of the stage are
// formed once and advanced by constants (the 14-bit address field cannot
// carry: shared memory ends below 256 KB), so the issuing thread spends a
// few instructions per MMA.  HI: the hi plane (X hi and lo terms), else the
// lo plane (X hi term); TRANS: also the transposed product.
template <int N, bool HI, bool TRANS>
__device__ __forceinline__ void sym_mma(uint32_t dd, uint32_t dt, uint64_t da, uint64_t dm,
                                        uint64_t dxjh, uint64_t dxjl, uint64_t dxih,
                                        uint64_t dxil) {
  constexpr uint32_t idd = idesc_bf16(BM, N);               // A_IJ X_J
  constexpr uint32_t idt = idesc_bf16(BM, N) | (1u << 15);  // A_IJ^T X_I (A MN-major)
#pragma unroll
  for (int kk = 0; kk < SYM_TILE / 16; ++kk) {
    // direct: rows I, contraction over J (16 columns of one 64-wide box)
    const uint64_t ao = (uint64_t)(((kk >> 2) * SYM_BOX + (kk & 3) * 32) >> 4);
    const uint64_t xo = (uint64_t)(((kk >> 2) * SymCfg<N>::XBOX + (kk & 3) * 32) >> 4);
    mma_bf16_acc(dd, da + ao, dxjh + xo, idd);
    if (HI) mma_bf16_acc(dd, da + ao, dxjl + xo, idd);
    if (TRANS) {
      // transposed: rows J, contraction over I (16 tile rows per step)
      const uint64_t ro = (uint64_t)((kk * 16 * 128) >> 4);
      mma_bf16_acc(dt, dm + ro, dxih + xo, idt);
      if (HI) mma_bf16_acc(dt, dm + ro, dxil + xo, idt);
    }
  }
}

template <int N>
__global__ void __launch_bounds__(192, 1)
bf16x3_sym_kernel(const __grid_constant__ CUtensorMap mAhi,
                  const __grid_constant__ CUtensorMap mAlo,
                  const __grid_constant__ CUtensorMap mXhi,
                  const __grid_constant__ CUtensorMap mXlo, int c, int b, int T, int Tsb,
                  int items, int64_t tiles, const int* __restrict__ item_start,
                  const int* __restrict__ seg0, int tmem_cols, float* __restrict__ part,
                  int* __restrict__ err, const int* __restrict__ skip) {
  using G = SymCfg<N>;
  if (skip && *skip) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* xbase = base + G::NA * SYM_PLANE;
  uint64_t* bars = (uint64_t*)(xbase + 2 * G::XSTAGE);
  uint64_t* afull = bars;
  uint64_t* aempty = bars + G::NA;
  uint64_t* xfull = bars + 2 * G::NA;
  uint64_t* xempty = xfull + 2;
  uint64_t* accf = xempty + 2;  // a segment's accumulators are complete
  uint64_t* acce = accf + 1;    // a segment's accumulators are drained and zeroed
  volatile uint32_t* tmem_slot = (volatile uint32_t*)(acce + 1);
  // [0] plane stages issued [1] consumed [2] X stages issued [3] consumed
  // [4] segments committed to accf
  volatile int* counts = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t t0 = (int64_t)blockIdx.x * tiles / gridDim.x;
  const int64_t t1 = (int64_t)(blockIdx.x + 1) * tiles / gridDim.x;
  if (threadIdx.x == 0) {
    for (int s = 0; s < G::NA; ++s) {
      mbar_init(smem_u32(&afull[s]), 1);
      mbar_init(smem_u32(&aempty[s]), 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(smem_u32(&xfull[s]), 1);
      mbar_init(smem_u32(&xempty[s]), 1);
    }
    mbar_init(smem_u32(accf), 1);
    mbar_init(smem_u32(acce), 4);
    for (int k = 0; k < 5; ++k) counts[k] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32((const void*)tmem_slot), tmem_cols);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      int u = 0, x = 0;
      SymCursor cur, pre;
      cur.start(t0, t1, item_start, items, Tsb, b, T);
      pre = cur;
      auto prefetch = [&](const SymCursor& k) {
        const int I = (k.S * b + k.i) * SYM_TILE, J = (k.C * b + k.j) * SYM_TILE;
        tma_prefetch_2d(&mAhi, J, I);
        tma_prefetch_2d(&mAhi, J + BK, I);
        tma_prefetch_2d(&mAlo, J, I);
        tma_prefetch_2d(&mAlo, J + BK, I);
      };
      for (int k = 0; k < SYM_PREFETCH && pre.valid(); ++k) {
        prefetch(pre);
        pre.next();
      }
      bool stop = false;
      for (; cur.valid() && !stop; cur.next()) {
        if (pre.valid()) {
          prefetch(pre);
          pre.next();
        }
        const int I = (cur.S * b + cur.i) * SYM_TILE, J = (cur.C * b + cur.j) * SYM_TILE;
        // X_J, X_I (hi, lo)
        {
          const int s = x & 1;
          if (x >= 2 && !mbar_wait(smem_u32(&xempty[s]), ((x >> 1) - 1) & 1, err, 21)) break;
          if (*(volatile int*)err) break;
          uint8_t* xs = xbase + s * G::XSTAGE;
          const uint32_t fb = smem_u32(&xfull[s]);
          mbar_expect_tx(fb, (uint32_t)G::XSTAGE);
          tma_load_2d(smem_u32(xs), &mXhi, fb, J, 0);
          tma_load_2d(smem_u32(xs + G::XBOX), &mXhi, fb, J + BK, 0);
          tma_load_2d(smem_u32(xs + 2 * G::XBOX), &mXlo, fb, J, 0);
          tma_load_2d(smem_u32(xs + 3 * G::XBOX), &mXlo, fb, J + BK, 0);
          tma_load_2d(smem_u32(xs + 4 * G::XBOX), &mXhi, fb, I, 0);
          tma_load_2d(smem_u32(xs + 5 * G::XBOX), &mXhi, fb, I + BK, 0);
          tma_load_2d(smem_u32(xs + 6 * G::XBOX), &mXlo, fb, I, 0);
          tma_load_2d(smem_u32(xs + 7 * G::XBOX), &mXlo, fb, I + BK, 0);
          ++x;
        }
        // the tile's hi plane, then its lo plane
        for (int plane = 0; plane < 2; ++plane) {
          const int s = u % G::NA;
          if (u >= G::NA && !mbar_wait(smem_u32(&aempty[s]), ((u / G::NA) - 1) & 1, err, 22)) {
            stop = true;
            break;
          }
          uint8_t* as = base + s * SYM_PLANE;
          const uint32_t fb = smem_u32(&afull[s]);
          mbar_expect_tx(fb, (uint32_t)SYM_PLANE);
          const CUtensorMap* m = plane ? &mAlo : &mAhi;
          tma_load_2d(smem_u32(as), m, fb, J, I);
          tma_load_2d(smem_u32(as + SYM_BOX), m, fb, J + BK, I);
          ++u;
        }
      }
      counts[0] = u;
      counts[2] = x;
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      int u = 0, x = 0, seg = 0;
      bool need_acc = true, stop = false;
      SymCursor cur;
      cur.start(t0, t1, item_start, items, Tsb, b, T);
      while (cur.valid() && !stop) {
        if (need_acc) {  // this segment's accumulators are zeroed
          if (!mbar_wait(smem_u32(acce), seg & 1, err, 23)) break;
          fence_after();
          need_acc = false;
        }
        const bool diag = (cur.S == cur.C);
        const int ad = cur.i;
        const int at = diag ? cur.j : b + cur.j;
        const bool trans = !(diag && cur.i == cur.j);
        const int sx = x & 1;
        if (!mbar_wait(smem_u32(&xfull[sx]), (x >> 1) & 1, err, 24)) break;
        const uint32_t xs = smem_u32(xbase + sx * G::XSTAGE);
        const uint64_t dxjh = sdesc(xs), dxjl = sdesc(xs + 2 * G::XBOX),
                       dxih = sdesc(xs + 4 * G::XBOX), dxil = sdesc(xs + 6 * G::XBOX);
        const uint32_t dd = tmem + (uint32_t)(ad * N), dt = tmem + (uint32_t)(at * N);
        for (int plane = 0; plane < 2; ++plane) {
          const int s = u % G::NA;
          if (!mbar_wait(smem_u32(&afull[s]), (u / G::NA) & 1, err, 25)) {
            stop = true;
            break;
          }
          fence_after();
          const uint32_t a = smem_u32(base + s * SYM_PLANE);
          const uint64_t da = sdesc(a), dm = sdesc_mn(a, SYM_BOX);
          if (plane == 0) {
            if (trans) sym_mma<N, true, true>(dd, dt, da, dm, dxjh, dxjl, dxih, dxil);
            else sym_mma<N, true, false>(dd, dt, da, dm, dxjh, dxjl, dxih, dxil);
          } else {
            if (trans) sym_mma<N, false, true>(dd, dt, da, dm, dxjh, dxjl, dxih, dxil);
            else sym_mma<N, false, false>(dd, dt, da, dm, dxjh, dxjl, dxih, dxil);
          }
          mma_commit(smem_u32(&aempty[s]));
          ++u;
        }
        if (stop) break;
        mma_commit(smem_u32(&xempty[sx]));
        ++x;
        if (cur.next()) {  // end of a segment
          mma_commit(smem_u32(accf));
          ++seg;
          counts[4] = seg;
          need_acc = true;
        }
      }
      counts[1] = u;
      counts[3] = x;
    }
    __syncwarp();
  } else {  // warps 2..5: zero, then drain each segment's accumulators
    const int q4 = warp & 3;
    const uint32_t lanes = (uint32_t)(q4 * 32) << 16;
    const int ncols = 2 * b * N;
    auto zero = [&]() {
      for (int c0 = 0; c0 < ncols; c0 += 16) tmem_zero16(tmem + lanes + (uint32_t)c0);
      tmem_st_wait();
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(acce));
    };
    zero();
    SymCursor cur;
    cur.start(t0, t1, item_start, items, Tsb, b, T);
    int seg = 0;
    const int g0 = seg0[blockIdx.x];
    while (cur.valid()) {
      const int S = cur.S, C = cur.C;
      while (!cur.next()) {
      }
      if (!mbar_wait(smem_u32(accf), seg & 1, err, 26)) break;
      fence_after();
      const int nacc = (S == C) ? b : 2 * b;
      const int gs = g0 + seg;
      for (int a = 0; a < nacc; ++a) {
        const int blk = (a < b) ? S * b + a : C * b + (a - b);
        if (blk >= T) continue;  // rows past the matrix
        float* dst = part + ((int64_t)(gs * 2 * b + a) * c) * SYM_TILE + q4 * 32 + lane;
#pragma unroll
        for (int j0 = 0; j0 < N; j0 += 16) {
          uint32_t v[16];
          tmem_ld16(tmem + lanes + (uint32_t)(a * N + j0), v);
          tmem_ld_wait();
#pragma unroll
          for (int qq = 0; qq < 16; ++qq)
            if (j0 + qq < c) dst[(int64_t)(j0 + qq) * SYM_TILE] = __uint_as_float(v[qq]);
        }
      }
      ++seg;
      if (cur.valid()) zero();
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // this CTA's MMAs and TMA copies have landed before tensor memory is freed
    const int committed = counts[4];
    if (committed > 0) mbar_drain(smem_u32(accf), (committed - 1) & 1, err, 27);
    for (int u = counts[1]; u < counts[0]; ++u)
      if (!mbar_drain(smem_u32(&afull[u % G::NA]), (u / G::NA) & 1, err, 28)) break;
    for (int x = counts[3]; x < counts[2]; ++x)
      if (!mbar_drain(smem_u32(&xfull[x & 1]), (x >> 1) & 1, err, 29)) break;
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, tmem_cols);
}

// Y (float64) = sum of the slots listed for each super-row, in list order:
// entry e is segment e >> 1, half e & 1 (0: the item's rows, 1: its columns)
__global__ void sym_reduce_kernel(int64_t n, int c, int b, const int* __restrict__ red_ptr,
                                  const int* __restrict__ red_ent,
                                  const float* __restrict__ part, double* __restrict__ Y,
                                  int64_t ldy, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t tot = n * c;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / n, r = e % n;
    const int R = (int)(r / SYM_TILE), rr = (int)(r % SYM_TILE);
    const int s = R / b, blk = R % b;
    double sum = 0.0;
    for (int k = red_ptr[s]; k < red_ptr[s + 1]; ++k) {
      const int ent = red_ent[k];
      const int g = ent >> 1, a = (ent & 1) ? b + blk : blk;
      sum += (double)part[((int64_t)(g * 2 * b + a) * c + j) * SYM_TILE + rr];
    }
    Y[r + j * ldy] = sum;
  }
}

__global__ void split_bf16_kernel(int64_t rows, int64_t cols, const double* __restrict__ A,
                                  int64_t lda, __nv_bfloat16* __restrict__ hi,
                                  __nv_bfloat16* __restrict__ lo, int64_t ldb) {
  const int64_t tot = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % rows, j = e / rows;
    const double a = A[i + j * lda];
    const __nv_bfloat16 h = __double2bfloat16(a);
    hi[i + j * ldb] = h;
    lo[i + j * ldb] = __double2bfloat16(a - (double)__bfloat162float(h));
  }
}

__global__ void splitk_sum_kernel(int64_t n, int c, int splits, const float* __restrict__ part,
                                  double* __restrict__ Y, int64_t ldy,
                                  const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t tot = n * c;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / n, i = e % n;
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += (double)part[((int64_t)z * c + j) * n + i];
    Y[i + j * ldy] = s;
  }
}

// signature of cuTensorMapEncodeTiled (driver API, obtained at run time)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
  static const EncodeTiledFn fn = [] {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (EncodeTiledFn)p;
    return (EncodeTiledFn) nullptr;
  }();
  return fn;
}

// k-tiles per split: fewest waves of 2 x 152 resident CTAs x (tiles per CTA
// + pipeline fill)
int tc_per(int64_t n) {
  const int64_t tiles = (n + BM - 1) / BM;
  const int64_t kt = (n + BK - 1) / BK;
  const int64_t slots = 2 * (int64_t)kNumSMs;
  int64_t best = -1, best_cost = 0;
  for (int64_t per = 1; per <= kt; ++per) {
    const int64_t s = (kt + per - 1) / per;
    const int64_t cost = ((tiles * s + slots - 1) / slots) * (per + 2);
    if (best < 0 || cost <= best_cost) {
      best = per;
      best_cost = cost;
    }
  }
  return (int)best;
}

int tc_splits(int64_t n) {
  const int64_t kt = (n + BK - 1) / BK;
  const int per = tc_per(n);
  return (int)((kt + per - 1) / per);
}

}  // namespace

int64_t tc_ld(int64_t n) { return ((n + 63) / 64) * 64; }

cudaError_t tc_split_matrix(int64_t rows, int64_t cols, const double* A, int64_t lda, void* hi,
                            void* lo, int64_t ldb, cudaStream_t st) {
  const int64_t tot = rows * cols;
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((tot + 255) / 256, 16 * kNumSMs));
  split_bf16_kernel<<<g, 256, 0, st>>>(rows, cols, A, lda, (__nv_bfloat16*)hi,
                                       (__nv_bfloat16*)lo, ldb); LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

bool tc_make_map(CUtensorMap* map, const void* base, int64_t inner, int64_t outer,
                 int64_t ld_elems, int box_inner, int box_outer) {
  auto fn = encoder();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  const cuuint64_t strides[1] = {(cuuint64_t)ld_elems * 2};
  const cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                  strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

namespace {

// Schedule of the symmetric kernel for one (n, N) on one device: super-block
// edge b, the tile prefix of every item, the first segment of every CTA and,
// per super-row, the partial slots to sum.  Built on the host once and kept
// in device memory for the life of the process.
struct SymPlan {
  int b = 1, T = 0, Tsb = 0, items = 0, grid = 0, nseg = 0;
  int64_t tiles = 0;
  int* d_item_start = nullptr;
  int* d_seg0 = nullptr;
  int* d_red_ptr = nullptr;
  int* d_red_ent = nullptr;
};

// b: about half a CTA's share of tiles per item (fewer segment drains), at
// most the 2 b N <= 512 tensor-memory columns of its accumulators
void sym_shape(int64_t n, int N, SymPlan& p) {
  p.T = (int)((n + SYM_TILE - 1) / SYM_TILE);
  const double per_cta = (double)p.T * (p.T + 1) / 2.0 / kNumSMs;
  int b = (int)std::lround(std::sqrt(std::max(1.0, per_cta / 2.0)));
  b = std::max(1, std::min(b, 256 / N));
  b = std::min(b, std::max(1, p.T));
  p.b = b;
  p.Tsb = (p.T + b - 1) / b;
  p.items = p.Tsb * (p.Tsb + 1) / 2;
}

int64_t sym_item_tiles(int q, const SymPlan& p) {
  int S, C;
  sym_item(q, p.Tsb, S, C);
  const int64_t ri = std::min(p.b, p.T - S * p.b);
  if (S == C) return ri * (ri + 1) / 2;
  const int64_t cj = std::min(p.b, p.T - C * p.b);
  return ri * cj;
}

int sym_segments(int64_t n, int N) {
  SymPlan p;
  sym_shape(n, N, p);
  std::vector<int64_t> start(p.items + 1, 0);
  for (int q = 0; q < p.items; ++q) start[q + 1] = start[q] + sym_item_tiles(q, p);
  const int64_t tiles = start[p.items];
  const int grid = (int)std::min<int64_t>(kNumSMs, tiles);
  int nseg = 0;
  for (int k = 0; k < grid; ++k) {
    const int64_t t0 = (int64_t)k * tiles / grid, t1 = (int64_t)(k + 1) * tiles / grid;
    const int q0 = (int)(std::upper_bound(start.begin(), start.end(), t0) - start.begin()) - 1;
    const int q1 = (int)(std::upper_bound(start.begin(), start.end(), t1 - 1) - start.begin()) - 1;
    nseg += q1 - q0 + 1;
  }
  return nseg;
}

cudaError_t sym_plan_get(int64_t n, int N, const SymPlan** out) {
  static std::mutex mu;
  static std::map<std::tuple<int, int64_t, int>, SymPlan> cache;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_tuple(dev, n, N);
  auto it = cache.find(key);
  if (it != cache.end()) {
    *out = &it->second;
    return cudaSuccess;
  }
  SymPlan p;
  sym_shape(n, N, p);
  std::vector<int> start(p.items + 1, 0);
  for (int q = 0; q < p.items; ++q) start[q + 1] = start[q] + (int)sym_item_tiles(q, p);
  p.tiles = start[p.items];
  p.grid = (int)std::min<int64_t>(kNumSMs, p.tiles);
  std::vector<int> seg0(p.grid + 1, 0);
  std::vector<std::vector<int>> lists(p.Tsb);
  int g = 0;
  for (int k = 0; k < p.grid; ++k) {
    seg0[k] = g;
    const int64_t t0 = (int64_t)k * p.tiles / p.grid, t1 = (int64_t)(k + 1) * p.tiles / p.grid;
    const int q0 = (int)(std::upper_bound(start.begin(), start.end(), (int)t0) - start.begin()) - 1;
    const int q1 =
        (int)(std::upper_bound(start.begin(), start.end(), (int)(t1 - 1)) - start.begin()) - 1;
    for (int q = q0; q <= q1; ++q, ++g) {
      int S, C;
      sym_item(q, p.Tsb, S, C);
      lists[S].push_back(2 * g);
      if (S != C) lists[C].push_back(2 * g + 1);
    }
  }
  seg0[p.grid] = g;
  p.nseg = g;
  std::vector<int> red_ptr(p.Tsb + 1, 0), red_ent;
  for (int s = 0; s < p.Tsb; ++s) {
    red_ent.insert(red_ent.end(), lists[s].begin(), lists[s].end());
    red_ptr[s + 1] = (int)red_ent.size();
  }
  auto upload = [](const std::vector<int>& v, int** d) -> cudaError_t {
    cudaError_t e2 = cudaMalloc(d, std::max<size_t>(1, v.size()) * sizeof(int));
    if (e2 != cudaSuccess) return e2;
    return cudaMemcpy(*d, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice);
  };
  if ((e = upload(start, &p.d_item_start)) != cudaSuccess) return e;
  if ((e = upload(seg0, &p.d_seg0)) != cudaSuccess) return e;
  if ((e = upload(red_ptr, &p.d_red_ptr)) != cudaSuccess) return e;
  if ((e = upload(red_ent, &p.d_red_ent)) != cudaSuccess) return e;
  auto res = cache.emplace(key, p);
  *out = &res.first->second;
  return cudaSuccess;
}

bool use_sym(int c) { return c <= 32; }

size_t sym_part_bytes(int64_t n, int c) {
  const int N = c <= 16 ? 16 : 32;
  SymPlan p;
  sym_shape(n, N, p);
  return (size_t)sym_segments(n, N) * 2 * p.b * c * SYM_TILE * 4;
}

}  // namespace

// monotone in c: room for any product of up to c columns
size_t tc_ws_bytes(int64_t n, int c) {
  const int64_t ldb = tc_ld(n);
  size_t part = std::max(sym_part_bytes(n, std::min(c, 16)), sym_part_bytes(n, std::min(c, 32)));
  if (!use_sym(c)) part = std::max(part, (size_t)tc_splits(n) * c * n * 4);
  return (size_t)2 * ldb * c * 2 + part + 4096;
}

cudaError_t tc_apply(const TcOperand& A, int64_t n, int c, const double* X, int64_t ldx,
                     double* Y, int64_t ldy, void* ws, size_t ws_bytes, int* err,
                     const int* skip, cudaStream_t st) {
  if (c <= 0) return cudaSuccess;
  if (c > 128) return cudaErrorInvalidValue;
  if (ws_bytes < tc_ws_bytes(n, c)) return cudaErrorInvalidValue;
  const int64_t ldb = tc_ld(n);
  uint8_t* w = (uint8_t*)ws;
  __nv_bfloat16* xhi = (__nv_bfloat16*)w;
  __nv_bfloat16* xlo = xhi + (size_t)ldb * c;
  float* part = (float*)(((uintptr_t)(xlo + (size_t)ldb * c) + 255) & ~(uintptr_t)255);
  cudaError_t e = tc_split_matrix(n, c, X, ldx, xhi, xlo, ldb, st);
  if (e != cudaSuccess) return e;
  const int N = ((c + 15) / 16) * 16;
  CUtensorMap mxh, mxl;
  if (!tc_make_map(&mxh, xhi, n, c, ldb, BK, N) || !tc_make_map(&mxl, xlo, n, c, ldb, BK, N))
    return cudaErrorInvalidValue;
  if (use_sym(c)) {
    const SymPlan* pl = nullptr;
    e = sym_plan_get(n, N, &pl);
    if (e != cudaSuccess) return e;
    int tcols = 32;
    while (tcols < 2 * pl->b * N) tcols <<= 1;
    if (N == 16) {
      const size_t smem = (size_t)SymCfg<16>::SMEM + 1024 + 256;
      static const cudaError_t a16 = cudaFuncSetAttribute(
          bf16x3_sym_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (a16 != cudaSuccess) return a16;
      bf16x3_sym_kernel<16><<<pl->grid, 192, smem, st>>>(
          A.hi_map, A.lo_map, mxh, mxl, c, pl->b, pl->T, pl->Tsb, pl->items, pl->tiles,
          pl->d_item_start, pl->d_seg0, tcols, part, err, skip); LREP_COUNT_LAUNCH();
    } else {
      const size_t smem = (size_t)SymCfg<32>::SMEM + 1024 + 256;
      static const cudaError_t a32 = cudaFuncSetAttribute(
          bf16x3_sym_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (a32 != cudaSuccess) return a32;
      bf16x3_sym_kernel<32><<<pl->grid, 192, smem, st>>>(
          A.hi_map, A.lo_map, mxh, mxl, c, pl->b, pl->T, pl->Tsb, pl->items, pl->tiles,
          pl->d_item_start, pl->d_seg0, tcols, part, err, skip); LREP_COUNT_LAUNCH();
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t tot = n * c;
    const unsigned g =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>((tot + 255) / 256, 8 * kNumSMs));
    sym_reduce_kernel<<<g, 256, 0, st>>>(n, c, pl->b, pl->d_red_ptr, pl->d_red_ent, part, Y,
                                         ldy, skip);
    LREP_COUNT_LAUNCH();
    return cudaGetLastError();
  }
  const int kt = (int)((n + BK - 1) / BK);
  const int per = tc_per(n);
  const int s = (kt + per - 1) / per;
  int tcols = 32;
  while (tcols < N) tcols <<= 1;
  const int tile_x = N * BK * 2;
  const int stage_bytes = ((2 * TILE_A + 2 * tile_x) + 1023) & ~1023;
  const size_t smem = (size_t)STAGES * stage_bytes + 1024 + 256;
  static const cudaError_t attr = cudaFuncSetAttribute(
      bf16x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (attr != cudaSuccess) return attr;
  dim3 grid((unsigned)((n + BM - 1) / BM), (unsigned)s);
  bf16x3_kernel<<<grid, 128, smem, st>>>(A.hi_map, A.lo_map, mxh, mxl, (int)n, c, N, per, kt,
                                         tcols, part, err, skip); LREP_COUNT_LAUNCH();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t tot = n * c;
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((tot + 255) / 256, 8 * kNumSMs));
  splitk_sum_kernel<<<g, 256, 0, st>>>(n, c, s, part, Y, ldy, skip); LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

}  // namespace lrep
