// Matrix-free Fourier spectral operator of the BdG example (Section 4,
// Example "large-scale dense matrix"): on a periodic nx*ny*nz grid of a
// box with side lengths L_d,
//   Y = coef * Lap_F X + d .* X,
//   Lap_F = sum_d F_d^-1 diag(-kappa_d^2) F_d,  kappa_d(m) = 2 pi m / L_d,
// m the signed frequency in [-N_d/2, N_d/2) (the Nyquist mode m = -N_d/2
// keeps kappa^2 = (pi N_d / L_d)^2).  The 3-D Fourier Laplacian is the sum
// of three 1-D ones, since the 3-D DFT is the tensor product of 1-D DFTs and
// |kappa|^2 is a sum over the axes; the product is therefore three passes,
// one per axis, each a batch of 1-D transforms along grid lines.
//
// One pass: a CTA stages a tile of grid lines of the axis in shared memory
// (coalesced: the tile is the lines of consecutive positions in the faster
// axes), packs two real lines into one complex line (the multiplier is real
// and even in m, so F^-1 diag(mu) F maps real lines to real lines and acts
// on the two halves separately), runs a radix-2 decimation-in-frequency FFT
// (natural order in, bit-reversed out), multiplies by the multiplier (with
// the 1/N of the inverse folded in), and a decimation-in-time inverse
// (bit-reversed in, natural out), so no permutation is ever done.  The last
// forward stage, the multiplier and the first inverse stage touch the same
// pair of points and run fused in registers.  The first pass writes
// Y = pass + d .* X, the others add to Y.
//
// The arithmetic type T is double for the float64 products and float for
// the inexact products of the block CG (eq. block_GS) in mixed precision;
// loads, stores and the diagonal term stay float64 in both.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace lrep {
namespace {

constexpr int kSpecThreads = 256;

__device__ __forceinline__ void sincospi_t(double x, double* s, double* c) { sincospi(x, s, c); }
__device__ __forceinline__ void sincospi_t(float x, float* s, float* c) { sincospif(x, s, c); }

// Tile geometry of one pass for line length N = 2^LOGN: E real values per
// tile (E / N lines, E / 2N complex lines), padded rows of N + 1 values.
template <int LOGN>
struct SpecTile {
  static constexpr int N = 1 << LOGN;
  static constexpr int E = N >= 8 ? 4096 : 2048;
  static constexpr int TL = E / N;      // real lines per tile
  static constexpr int LTL = (N >= 8 ? 12 : 11) - LOGN;
  static constexpr int P = TL / 2;      // complex lines per tile
  static constexpr int ROW = N + 1;     // padded complex row
  static constexpr int EPT = E / kSpecThreads;
  static constexpr int BPT = E / 4 / kSpecThreads;  // butterflies per thread per stage
};

// Lines of the axis: line (col, o, w), o < O, w < s, element a at
// col * ld + o * N * s + w + a * s.  A tile is TO consecutive (col, o)
// blocks (flattened g = col * O + o) times TW consecutive w; tiles are
// numbered block-major with s / TW w-blocks per block.  All of O, s, TW, TO
// are powers of two and passed as their base-2 logarithms.
struct AxisGeom {
  int64_t nblocks;  // c * O
  int lO, ls, lTW, lnwb;
};

template <int LOGN>
__device__ __forceinline__ bool spec_element(const AxisGeom& ag, int64_t g0, int64_t w0, int e,
                                             int64_t* col, int64_t* off, int* lt, int* a) {
  const int wl = e & ((1 << ag.lTW) - 1);
  *a = (e >> ag.lTW) & ((1 << LOGN) - 1);
  const int lo = e >> (ag.lTW + LOGN);
  *lt = (lo << ag.lTW) + wl;
  const int64_t g = g0 + lo;
  *col = g >> ag.lO;
  const int64_t o = g & ((int64_t(1) << ag.lO) - 1);
  *off = (o << (LOGN + ag.ls)) + w0 + wl + ((int64_t)*a << ag.ls);
  return g < ag.nblocks;
}

template <typename T, int LOGN, bool DIAG>
__global__ void __launch_bounds__(kSpecThreads, 2)
spectral_axis_kernel(AxisGeom ag, const double* __restrict__ X, int64_t ldx,
                     double* __restrict__ Y, int64_t ldy, const double* __restrict__ d,
                     double scale, const int* __restrict__ skip) {
  using G = SpecTile<LOGN>;
  constexpr int N = G::N;
  constexpr int HALF = N / 2;
  if (skip && *skip) return;
  __shared__ T re[G::P * G::ROW];
  __shared__ T im[G::P * G::ROW];
  __shared__ T twr[HALF], twi[HALF];
  for (int t = threadIdx.x; t < HALF; t += kSpecThreads) {
    T sv, cv;
    sincospi_t(T(-2 * t) / T(N), &sv, &cv);  // exp(-2 pi i t / N)
    twr[t] = cv;
    twi[t] = sv;
  }
  const int64_t tile = blockIdx.x;
  const int64_t g0 = (tile >> ag.lnwb) << (G::LTL - ag.lTW);
  const int64_t w0 = (tile & ((int64_t(1) << ag.lnwb) - 1)) << ag.lTW;

  // load: element e -> (lo, a, wl), wl fastest, so that each (col, o)
  // block is read as runs of TW consecutive values
#pragma unroll 4
  for (int k = 0; k < G::EPT; ++k) {
    int64_t col, off;
    int lt, a;
    const bool ok = spec_element<LOGN>(ag, g0, w0, threadIdx.x + k * kSpecThreads, &col, &off,
                                       &lt, &a);
    const double v = ok ? X[col * ldx + off] : 0.0;
    T* dst = (lt & 1) ? im : re;
    dst[(lt >> 1) * G::ROW + a] = (T)v;
  }
  __syncthreads();

  // forward, decimation in frequency: span m = N >> st, half h = m / 2,
  // pair (i0, i0 + h) with i0 = 2j - k, k = j mod h; twiddle w_m^k
#pragma unroll 1
  for (int st = 0; st < LOGN - 1; ++st) {
    const int h = HALF >> st;
#pragma unroll 2
    for (int r = 0; r < G::BPT; ++r) {
      const int b = threadIdx.x + r * kSpecThreads;
      const int q = b / HALF, j = b % HALF;
      const int k = j & (h - 1);
      const int i0 = q * G::ROW + 2 * j - k, i1 = i0 + h;
      const T ar = re[i0], ai = im[i0], br = re[i1], bi = im[i1];
      const T dr = ar - br, di = ai - bi;
      const T wr = twr[k << st], wi = twi[k << st];
      re[i0] = ar + br;
      im[i0] = ai + bi;
      re[i1] = dr * wr - di * wi;
      im[i1] = dr * wi + di * wr;
    }
    __syncthreads();
  }
  // last forward stage (span 2), multiplier, first inverse stage (span 2):
  // position p holds frequency bitrev(p)
  const T sc = (T)scale;
#pragma unroll
  for (int r = 0; r < G::BPT; ++r) {
    const int b = threadIdx.x + r * kSpecThreads;
    const int q = b / HALF, j = b % HALF;
    const int i0 = q * G::ROW + 2 * j, i1 = i0 + 1;
    const T ar = re[i0], ai = im[i0], br = re[i1], bi = im[i1];
    const int f0 = (int)(__brev((unsigned)(2 * j)) >> (32 - LOGN));
    const int f1 = f0 + HALF;  // bitrev(2j + 1) = bitrev(2j) + N / 2
    const int m0 = f0 < HALF ? f0 : f0 - N, m1 = f1 < HALF ? f1 : f1 - N;
    const T mu0 = sc * (T)(m0 * m0), mu1 = sc * (T)(m1 * m1);
    const T xr = (ar + br) * mu0, xi = (ai + bi) * mu0;
    const T yr = (ar - br) * mu1, yi = (ai - bi) * mu1;
    re[i0] = xr + yr;
    im[i0] = xi + yi;
    re[i1] = xr - yr;
    im[i1] = xi - yi;
  }
  __syncthreads();
  // inverse, decimation in time: span m = 2h, h = 2^st, twiddle conj(w_m^k)
#pragma unroll 1
  for (int st = 1; st < LOGN; ++st) {
    const int h = 1 << st;
    const int sh = LOGN - 1 - st;  // log2(N / m)
#pragma unroll 2
    for (int r = 0; r < G::BPT; ++r) {
      const int b = threadIdx.x + r * kSpecThreads;
      const int q = b / HALF, j = b % HALF;
      const int k = j & (h - 1);
      const int i0 = q * G::ROW + 2 * j - k, i1 = i0 + h;
      const T wr = twr[k << sh], wi = -twi[k << sh];
      const T br = re[i1], bi = im[i1];
      const T tr = br * wr - bi * wi, ti = br * wi + bi * wr;
      const T ar = re[i0], ai = im[i0];
      re[i0] = ar + tr;
      im[i0] = ai + ti;
      re[i1] = ar - tr;
      im[i1] = ai - ti;
    }
    __syncthreads();
  }

  // store (the diagonal term re-reads X, which the load left in L2)
#pragma unroll 4
  for (int k = 0; k < G::EPT; ++k) {
    int64_t col, off;
    int lt, a;
    if (!spec_element<LOGN>(ag, g0, w0, threadIdx.x + k * kSpecThreads, &col, &off, &lt, &a))
      continue;
    const T* src = (lt & 1) ? im : re;
    const double v = (double)src[(lt >> 1) * G::ROW + a];
    double* y = Y + col * ldy + off;
    if (DIAG)
      *y = fma(d[off], X[col * ldx + off], v);
    else
      *y += v;
  }
}

__global__ void spectral_diag_kernel(int64_t n, int c, const double* __restrict__ d,
                                     const double* __restrict__ X, int64_t ldx,
                                     double* __restrict__ Y, int64_t ldy,
                                     const int* __restrict__ skip) {
  if (skip && *skip) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * c;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = i / n, r = i - (i / n) * n;
    Y[col * ldy + r] = d[r] * X[col * ldx + r];
  }
}

int ilog2(int64_t v) {
  int l = 0;
  while ((int64_t(1) << l) < v) ++l;
  return l;
}

template <typename T, int LOGN>
cudaError_t launch_axis(bool diag, int64_t n, int c, int64_t s, double scale,
                        const double* d, const double* X, int64_t ldx, double* Y,
                        int64_t ldy, const int* skip, cudaStream_t st) {
  using G = SpecTile<LOGN>;
  const int64_t O = n / ((int64_t)G::N * s);
  const int64_t TW = std::min<int64_t>(s, G::TL);
  const int64_t TO = G::TL / TW;
  AxisGeom ag;
  ag.nblocks = (int64_t)c * O;
  ag.lO = ilog2(O);
  ag.ls = ilog2(s);
  ag.lTW = ilog2(TW);
  ag.lnwb = ilog2(s / TW);
  const int64_t tiles = (ag.nblocks + TO - 1) / TO * (s / TW);
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  if (diag)
    spectral_axis_kernel<T, LOGN, true><<<(unsigned)tiles, kSpecThreads, 0, st>>>(
        ag, X, ldx, Y, ldy, d, scale, skip);
  else
    spectral_axis_kernel<T, LOGN, false><<<(unsigned)tiles, kSpecThreads, 0, st>>>(
        ag, X, ldx, Y, ldy, d, scale, skip);
  LREP_COUNT_LAUNCH();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_axis_n(int logn, bool diag, int64_t n, int c, int64_t s, double scale,
                          const double* d, const double* X, int64_t ldx, double* Y,
                          int64_t ldy, const int* skip, cudaStream_t st) {
  switch (logn) {
#define SPEC_CASE(L) \
  case L:            \
    return launch_axis<T, L>(diag, n, c, s, scale, d, X, ldx, Y, ldy, skip, st);
    SPEC_CASE(1) SPEC_CASE(2) SPEC_CASE(3) SPEC_CASE(4)
    SPEC_CASE(5) SPEC_CASE(6) SPEC_CASE(7) SPEC_CASE(8)
#undef SPEC_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t spectral_apply_t(const int dims[3], const double scale[3], const double* d, int c,
                             const double* X, int64_t ldx, double* Y, int64_t ldy,
                             const int* skip, cudaStream_t st) {
  if (c <= 0) return cudaSuccess;
  const int64_t n = (int64_t)dims[0] * dims[1] * dims[2];
  int64_t s = 1;
  bool first = true;
  for (int ax = 0; ax < 3; ++ax) {
    const int N = dims[ax];
    if (N > 1) {
      const int logn = spectral_log2(N);
      if (logn < 1) return cudaErrorInvalidValue;
      const cudaError_t e =
          launch_axis_n<T>(logn, first, n, c, s, scale[ax], d, X, ldx, Y, ldy, skip, st);
      if (e != cudaSuccess) return e;
      first = false;
    }
    s *= N;
  }
  if (first) {  // a single grid point: only the diagonal term
    spectral_diag_kernel<<<kNumSMs, 256, 0, st>>>(n, c, d, X, ldx, Y, ldy, skip);
    LREP_COUNT_LAUNCH();
    return cudaGetLastError();
  }
  return cudaSuccess;
}

}  // namespace

int spectral_log2(int N) {
  for (int l = 1; l <= kSpectralMaxLog; ++l)
    if (N == (1 << l)) return l;
  return -1;
}

cudaError_t spectral_apply(bool fp32, const int dims[3], const double scale[3],
                           const double* d, int c, const double* X, int64_t ldx, double* Y,
                           int64_t ldy, const int* skip, cudaStream_t st) {
  return fp32 ? spectral_apply_t<float>(dims, scale, d, c, X, ldx, Y, ldy, skip, st)
              : spectral_apply_t<double>(dims, scale, d, c, X, ldx, Y, ldy, skip, st);
}

}  // namespace lrep
