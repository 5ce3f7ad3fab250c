// Internal helpers shared by the CUDA translation units of the solver.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstdio>

namespace lrep {

// kernels launched by this library since load (lrep_launch_count)
extern std::atomic<long long> g_launches;
#define LREP_COUNT_LAUNCH() (::lrep::g_launches.fetch_add(1, std::memory_order_relaxed))

constexpr int kNumSMs = 152;          // GB300: 2 dies x 76 SMs
constexpr int kMaxSegs = 3;           // column segments of one logical block

// A logical n x (sum cols) block made of up to kMaxSegs column-major
// pieces (e.g. [X0 | X_locked] next to [X~ | P~]).
struct Segs {
  const double* ptr[kMaxSegs];
  int64_t ld[kMaxSegs];
  int cols[kMaxSegs];
  int nseg;
  __host__ __device__ int total() const {
    int t = 0;
    for (int s = 0; s < nseg; ++s) t += cols[s];
    return t;
  }
  __host__ __device__ const double* col(int j) const {
    for (int s = 0; s < nseg; ++s) {
      if (j < cols[s]) return ptr[s] + (int64_t)j * ld[s];
      j -= cols[s];
    }
    return nullptr;
  }
};

inline Segs seg1(const double* p, int64_t ld, int cols) {
  Segs s{};
  s.ptr[0] = p; s.ld[0] = ld; s.cols[0] = cols; s.nseg = 1;
  return s;
}
inline Segs seg_push(Segs s, const double* p, int64_t ld, int cols) {
  if (cols <= 0) return s;
  s.ptr[s.nseg] = p; s.ld[s.nseg] = ld; s.cols[s.nseg] = cols; s.nseg++;
  return s;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum for blockDim.x a multiple of 32 (<= 1024); every thread
// receives the result.  `red` must hold 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  double t = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  t = red[0];
  __syncthreads();
  return t;
}

// "Last block done" handshake for two-stage reductions with a fixed
// summation order: every block writes its partials, then the last block to
// arrive reduces them in index order and resets the counter for the next
// launch.  Returns true in the last block.
__device__ __forceinline__ bool arrive_last(unsigned int* counter) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int nblk = gridDim.x * gridDim.y * gridDim.z;
    last = (atomicAdd(counter, 1u) == nblk - 1);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) *counter = 0u;
  return last;
}

// float64 <-> float32 conversions on the integer units.  GB300 executes
// every float64 instruction, conversions included, on its FP64 units (about
// 2 per clock per SM), so a float32 kernel that loads and stores float64
// data is bound by its conversions.  These rebuild the other format's bit
// pattern with integer instructions and selects (no branch, no call).
// f64_to_f32: round to nearest even; results below the float32 normal
// range flush to a signed zero, overflow gives a signed infinity, NaN stays
// NaN.
__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sign = hi & 0x80000000u;
  const unsigned e = (hi >> 20) & 0x7FFu;
  const unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);  // top 23 mantissa bits
  const unsigned rest = lo & 0x1FFFFFFFu;                  // the 29 dropped bits
  unsigned f = sign | ((e - 896u) << 23) | m;
  // a carry out of the mantissa steps the exponent (to infinity past the
  // largest float), as rounding to nearest does
  f += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
  const bool nan = e == 0x7FFu && ((hi & 0xFFFFFu) | lo) != 0u;
  f = e < 897u ? sign : f;
  f = e > 1150u ? (sign | 0x7F800000u | (nan ? 0x400000u : 0u)) : f;
  return __uint_as_float(f);
}

// f64_to_f32_rz: rounded toward zero (error below 2^-23 relative, the float
// kernels' own rounding), half the instructions of f64_to_f32: the float
// pattern is the double's top bits with the exponent rebased, computed
// modulo 2^9 in the exponent field (exact for biased exponents 897..1150);
// smaller magnitudes flush to a signed zero, larger ones and NaN give a
// signed infinity.
__device__ __forceinline__ float f64_to_f32_rz(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned mag = hi & 0x7FFFFFFFu;
  unsigned f = ((mag << 3) | (lo >> 29)) - (896u << 23);
  f = mag < (897u << 20) ? 0u : f;
  f = mag >= (1151u << 20) ? 0x7F800000u : f;
  return __uint_as_float(f | (hi & 0x80000000u));
}

// f32_to_f64: exact for normal numbers, zero, infinities (NaN stays NaN);
// float32 subnormals flush to a signed zero.
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u, fe = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  unsigned hi = sign | ((fe + 896u) << 20) | (m >> 3);
  unsigned lo = u << 29;
  hi = fe == 0u ? sign : hi;
  lo = fe == 0u ? 0u : lo;
  hi = fe == 0xFFu ? (sign | 0x7FF00000u | (m >> 3) | (m ? 0x80000u : 0u)) : hi;
  return __hiloint2double((int)hi, (int)lo);
}

// Read through L2 (partials written by other blocks of the same launch).
__device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }

// Number of row slabs used by the fixed-order reductions over n rows.
inline int reduction_slabs(int64_t n, int rows_per_slab_min = 512, int max_slabs = 2 * kNumSMs) {
  int64_t s = (n + rows_per_slab_min - 1) / rows_per_slab_min;
  if (s < 1) s = 1;
  if (s > max_slabs) s = max_slabs;
  return (int)s;
}

}  // namespace lrep
