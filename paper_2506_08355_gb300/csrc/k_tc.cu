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

// hi = bf16(a), lo = bf16(a - hi); columns over grid y, rows over grid x
__global__ void split_bf16_kernel(int64_t rows, int64_t cols, const double* __restrict__ A,
                                  int64_t lda, __nv_bfloat16* __restrict__ hi,
                                  __nv_bfloat16* __restrict__ lo, int64_t ldb) {
  for (int64_t j = blockIdx.y; j < cols; j += gridDim.y)
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows;
         i += (int64_t)gridDim.x * blockDim.x) {
      const double a = A[i + j * lda];
      const __nv_bfloat16 h = __double2bfloat16(a);
      hi[i + j * ldb] = h;
      lo[i + j * ldb] = __double2bfloat16(a - (double)__bfloat162float(h));
    }
}

// Y = sum over the splits of the fp32 partials, in split order, in fp64;
// column j = blockIdx.y
__global__ void splitk_sum_kernel(int64_t n, int c, int splits, const float* __restrict__ part,
                                  double* __restrict__ Y, int64_t ldy,
                                  const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int j = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += (double)part[((int64_t)z * c + j) * n + i];
    Y[i + j * ldy] = s;
  }
}

// 2-D launch shape of the column-wise kernels above: ~4 CTAs per SM in all
dim3 colwise_grid(int64_t rows, int64_t cols) {
  const int64_t gy = std::min<int64_t>(std::max<int64_t>(cols, 1), 65535);
  const int64_t want = std::max<int64_t>(1, (4 * kNumSMs + gy - 1) / gy);
  const int64_t gx = std::max<int64_t>(1, std::min<int64_t>((rows + 255) / 256, want));
  return dim3((unsigned)gx, (unsigned)gy);
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
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  split_bf16_kernel<<<colwise_grid(rows, cols), 256, 0, st>>>(
      rows, cols, A, lda, (__nv_bfloat16*)hi, (__nv_bfloat16*)lo, ldb); LREP_COUNT_LAUNCH();
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

size_t tc_ws_bytes(int64_t n, int c) {
  const int64_t ldb = tc_ld(n);
  return (size_t)2 * ldb * c * 2 + (size_t)tc_splits(n) * c * n * 4 + 4096;
}

TcBuffers tc_buffers(void* ws, int64_t n, int c) {
  TcBuffers b;
  b.ldb = tc_ld(n);
  b.xhi = ws;
  b.xlo = (uint8_t*)ws + (size_t)b.ldb * c * 2;
  b.part = (float*)(((uintptr_t)b.xlo + (size_t)b.ldb * c * 2 + 255) & ~(uintptr_t)255);
  b.splits = tc_splits(n);
  return b;
}

cudaError_t tc_product_partials(const TcOperand& A, int64_t n, int c, const double* X,
                                int64_t ldx, bool x_split, void* ws, size_t ws_bytes, int* err,
                                const int* skip, cudaStream_t st) {
  if (c <= 0) return cudaSuccess;
  if (c > 128) return cudaErrorInvalidValue;
  if (ws_bytes < tc_ws_bytes(n, c)) return cudaErrorInvalidValue;
  const TcBuffers b = tc_buffers(ws, n, c);
  if (!x_split) {
    const cudaError_t e = tc_split_matrix(n, c, X, ldx, b.xhi, b.xlo, b.ldb, st);
    if (e != cudaSuccess) return e;
  }
  const int N = ((c + 15) / 16) * 16;
  CUtensorMap mxh, mxl;
  if (!tc_make_map(&mxh, b.xhi, n, c, b.ldb, BK, N) ||
      !tc_make_map(&mxl, b.xlo, n, c, b.ldb, BK, N))
    return cudaErrorInvalidValue;
  const int kt = (int)((n + BK - 1) / BK);
  const int per = tc_per(n);
  int tcols = 32;
  while (tcols < N) tcols <<= 1;
  const int tile_x = N * BK * 2;
  const int stage_bytes = ((2 * TILE_A + 2 * tile_x) + 1023) & ~1023;
  const size_t smem = (size_t)STAGES * stage_bytes + 1024 + 256;
  static const cudaError_t attr = cudaFuncSetAttribute(
      bf16x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (attr != cudaSuccess) return attr;
  dim3 grid((unsigned)((n + BM - 1) / BM), (unsigned)b.splits);
  bf16x3_kernel<<<grid, 128, smem, st>>>(A.hi_map, A.lo_map, mxh, mxl, (int)n, c, N, per, kt,
                                         tcols, b.part, err, skip); LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t tc_apply(const TcOperand& A, int64_t n, int c, const double* X, int64_t ldx,
                     double* Y, int64_t ldy, void* ws, size_t ws_bytes, int* err,
                     const int* skip, cudaStream_t st) {
  if (c <= 0) return cudaSuccess;
  cudaError_t e = tc_product_partials(A, n, c, X, ldx, false, ws, ws_bytes, err, skip, st);
  if (e != cudaSuccess) return e;
  const TcBuffers b = tc_buffers(ws, n, c);
  splitk_sum_kernel<<<colwise_grid(n, c), 256, 0, st>>>(n, c, b.splits, b.part, Y, ldy, skip);
  LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

}  // namespace lrep
