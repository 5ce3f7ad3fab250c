// Tensor-core (tcgen05) operator products: internal interface.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lrep {

// One symmetric operator split as bf16 hi + lo (row i = column i, leading
// dimension ldb elements) with its TMA descriptors (box 64 x 128,
// 128-byte swizzle).
struct TcOperand {
  CUtensorMap hi_map;
  CUtensorMap lo_map;
  void* hi = nullptr;
  void* lo = nullptr;
  int64_t ldb = 0;
};

int64_t tc_ld(int64_t n);
// hi = bf16(A), lo = bf16(A - hi) for a rows x cols column-major block
cudaError_t tc_split_matrix(int64_t rows, int64_t cols, const double* A, int64_t lda, void* hi,
                            void* lo, int64_t ldb, cudaStream_t st);
bool tc_make_map(CUtensorMap* map, const void* base, int64_t inner, int64_t outer,
                 int64_t ld_elems, int box_inner, int box_outer);
size_t tc_ws_bytes(int64_t n, int c);
// Where tc_apply keeps X's split and the split-K partials in its workspace:
// xhi, xlo (bf16, leading dimension ldb), part (fp32, splits x c x n,
// part[(z * c + j) * n + i]).
struct TcBuffers {
  void* xhi;
  void* xlo;
  int64_t ldb;
  float* part;
  int splits;
};
TcBuffers tc_buffers(void* ws, int64_t n, int c);
// The product without its split-K sum: the partials stay in the workspace
// for the caller to reduce (the fused CG step).  x_split: X's bf16 split is
// already in the workspace (X is then not read).
cudaError_t tc_product_partials(const TcOperand& A, int64_t n, int c, const double* X,
                                int64_t ldx, bool x_split, void* ws, size_t ws_bytes, int* err,
                                const int* skip, cudaStream_t st);
// Y = A X for up to 128 columns; *err receives a non-zero code if a
// pipeline wait expired (the result is then invalid).
cudaError_t tc_apply(const TcOperand& A, int64_t n, int c, const double* X, int64_t ldx,
                     double* Y, int64_t ldy, void* ws, size_t ws_bytes, int* err,
                     const int* skip, cudaStream_t st);

}  // namespace lrep
