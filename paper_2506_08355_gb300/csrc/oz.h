// FP64-accurate dense operator products on the bf16 tensor cores by
// error-free slicing (k_oz.cu): internal interface.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace lrep {

constexpr int kOzSlices = 7;  // base-2^8 digits per float64 value

// A symmetric n x n operator held as 7 bfloat16 digit planes: plane s,
// row i, column k at slices[(s * rows_pad + i) * ldk + k] (rows_pad a
// multiple of 128, ldk a multiple of 64, padding zero), with the row
// exponents sig[i] (A_ik = 2^sig[i] * sum_s digit_s * 2^(-8 (s + 1)), up to
// 2^(sig[i] - 57)) and the TMA descriptor of the planes (box 64 x 128).
struct OzOperand {
  CUtensorMap map;
  void* slices = nullptr;
  int* sig = nullptr;
  int64_t n = 0, ldk = 0, rows_pad = 0;
};

int64_t oz_ldk(int64_t n);
int64_t oz_rows_pad(int64_t n);
// device bytes of one OzOperand's digit planes and exponents
size_t oz_operand_bytes(int64_t n);
// o->slices (oz_operand_bytes) must be allocated by the caller; fills the
// digit planes, the exponents (placed after the planes) and the descriptor.
cudaError_t oz_slice_operator(int64_t n, const double* A, int64_t lda, OzOperand* o,
                              cudaStream_t st);
size_t oz_ws_bytes(int64_t n, int c);
// Y = A X (n x c, float64); *err receives a non-zero code if a pipeline wait
// expired (the result is then invalid).  skip: optional device flag; when it
// is non-zero the call leaves Y untouched.
cudaError_t oz_apply(const OzOperand& A, int c, const double* X, int64_t ldx, double* Y,
                     int64_t ldy, void* ws, size_t ws_bytes, int* err, const int* skip,
                     cudaStream_t st);

// Tall-skinny products with float64 accuracy on the same machinery (same
// error bound form, with e_i bounding row i of the left factor and f_j
// column j of the right factor):
//   G (a x b, ldg) = A^T B for segmented n x a and n x b blocks;
//   C (n x c, ldc) = alpha C + beta A B for a segmented n x k block A and a
//   k x c matrix B (ldb); beta != 0.
size_t oz_gram_ws_bytes(int64_t n, int a, int b);
cudaError_t oz_gram(int64_t n, const Segs& A, const Segs& B, double* G, int64_t ldg, void* ws,
                    size_t ws_bytes, int* err, cudaStream_t st);
size_t oz_update_ws_bytes(int64_t n, int k, int c);
cudaError_t oz_update(int64_t n, int k, int c, double alpha, const Segs& A, const double* B,
                      int64_t ldb, double beta, double* C, int64_t ldc, void* ws,
                      size_t ws_bytes, int* err, cudaStream_t st);

}  // namespace lrep
