// Tensor-core operators of the dense K and M, built once per problem from
// the float64 matrices according to opts.precision:
//  * bit 0 (MIXED_BF16X3): hi + lo bfloat16 split for the inexact CG
//    products of eq. block_GS (k_tc.cu); spectral and stencil operators need
//    no split and run those products with float32 arithmetic (k_spectral.cu,
//    k_ops.cu);
//  * bit 1 (FP64_SLICED): seven bf16 digit planes for float64-accurate
//    products by error-free slicing (k_oz.cu): every product that enters H^
//    (eq. hat_H) and every residual (eq. tol), and the CG products when bit 0
//    is clear; for any operator kind, the large tall-skinny Grams and block
//    updates of the solver take the same route (bosp.cu).
// Without bit 1, float64 products use the FP64 kernels.
#include <cuda_runtime.h>

#include "oz.h"
#include "problem.h"
#include "tc.h"

namespace lrep {

namespace {
bool want_tc(const lrep_problem p) { return (p->opts.precision & LREP_PREC_MIXED_BF16X3) != 0; }
bool want_oz(const lrep_problem p) { return (p->opts.precision & LREP_PREC_FP64_SLICED) != 0; }
}  // namespace

bool split_ready(lrep_problem p) {
  const Operator& o = p->op;
  const bool dense = o.kind == OP_DENSE;
  return (p->opts.precision == LREP_PREC_FP64 || o.tc_err) &&
         (!want_tc(p) || o.tcK || o.kind == OP_SPECTRAL || o.kind == OP_STENCIL) &&
         (!want_oz(p) || !dense || (o.ozK && (!o.hasB || o.ozB)));
}

size_t split_bytes(lrep_problem p) {
  const int64_t n = p->op.n;
  size_t b = 0;
  if (want_tc(p) && p->op.kind == OP_DENSE)
    b += (size_t)2 * 2 * 2 * tc_ld(n) * n;  // K, M x (hi, lo) bf16
  if (want_oz(p) && p->op.kind == OP_DENSE)               // K, M (B) x 7 digit planes
    b += (size_t)(p->op.hasB ? 3 : 2) * oz_operand_bytes(n);
  return b;
}

lrep_status build_split(lrep_problem p) {
  Operator& o = p->op;
  free_split(p);
  if (p->opts.precision == LREP_PREC_FP64) return LREP_OK;
  if (want_tc(p) && o.kind != OP_DENSE && o.kind != OP_SPECTRAL && o.kind != OP_STENCIL)
    return p->fail(LREP_ERR_ARG,
                   "mixed-precision CG products need a dense, stencil or spectral operator");
  const int64_t n = o.n;
  const double* src[2] = {o.K, o.M};
  if (want_tc(p) && o.kind == OP_DENSE) {
    const int64_t ldb = tc_ld(n);
    const size_t bytes = (size_t)ldb * n * 2;
    TcOperand* t[2] = {new TcOperand(), new TcOperand()};
    o.tcK = t[0];
    o.tcM = t[1];
    for (int i = 0; i < 2; ++i) {
      cudaError_t e = cudaMalloc(&t[i]->hi, bytes);
      if (e == cudaSuccess) e = cudaMalloc(&t[i]->lo, bytes);
      if (e != cudaSuccess) {
        free_split(p);
        return p->fail(LREP_ERR_NOMEM, "bf16 split of the operator: out of device memory");
      }
      t[i]->ldb = ldb;
      e = tc_split_matrix(n, n, src[i], o.ld, t[i]->hi, t[i]->lo, ldb, p->stream);
      if (e != cudaSuccess) {
        free_split(p);
        return p->fail(LREP_ERR_CUDA, std::string("bf16 split: ") + cudaGetErrorString(e));
      }
      if (!tc_make_map(&t[i]->hi_map, t[i]->hi, n, n, ldb, 64, 128) ||
          !tc_make_map(&t[i]->lo_map, t[i]->lo, n, n, ldb, 64, 128)) {
        free_split(p);
        return p->fail(LREP_ERR_CUDA, "cuTensorMapEncodeTiled failed for the operator split");
      }
    }
  }
  if (want_oz(p) && o.kind == OP_DENSE) {
    OzOperand* z[3] = {new OzOperand(), new OzOperand(), o.hasB ? new OzOperand() : nullptr};
    o.ozK = z[0];
    o.ozM = z[1];
    o.ozB = z[2];
    const double* src3[3] = {o.K, o.M, o.B};
    for (int i = 0; i < (o.hasB ? 3 : 2); ++i) {
      if (cudaMalloc(&z[i]->slices, oz_operand_bytes(n)) != cudaSuccess) {
        free_split(p);
        return p->fail(LREP_ERR_NOMEM, "digit planes of the operator: out of device memory");
      }
      const cudaError_t e = oz_slice_operator(n, src3[i], o.ld, z[i], p->stream);
      if (e != cudaSuccess) {
        free_split(p);
        return p->fail(LREP_ERR_CUDA, std::string("digit planes: ") + cudaGetErrorString(e));
      }
    }
  }
  if (cudaMalloc(&o.tc_err, sizeof(int)) != cudaSuccess ||
      cudaMemsetAsync(o.tc_err, 0, sizeof(int), p->stream) != cudaSuccess ||
      cudaStreamSynchronize(p->stream) != cudaSuccess) {
    free_split(p);
    return p->fail(LREP_ERR_CUDA, "tensor-core operator: device error");
  }
  return LREP_OK;
}

void free_split(lrep_problem p) {
  Operator& o = p->op;
  for (TcOperand** t : {&o.tcK, &o.tcM}) {
    if (*t) {
      if ((*t)->hi) cudaFree((*t)->hi);
      if ((*t)->lo) cudaFree((*t)->lo);
      delete *t;
      *t = nullptr;
    }
  }
  for (OzOperand** z : {&o.ozK, &o.ozM, &o.ozB}) {
    if (*z) {
      if ((*z)->slices) cudaFree((*z)->slices);
      delete *z;
      *z = nullptr;
    }
  }
  if (o.tc_err) cudaFree(o.tc_err);
  o.tc_err = nullptr;
}

size_t apply_cg_ws_elems(lrep_problem p, int c) {
  size_t b = 0;
  if (p->op.tcK) b = std::max(b, tc_ws_bytes(p->op.n, c));
  if (p->op.ozK) b = std::max(b, oz_ws_bytes(p->op.n, c));
  return b ? b / sizeof(double) + 1 : 0;
}

lrep_status apply_sliced(lrep_problem p, int which, int c, const double* X, int64_t ldx,
                         double* Y, int64_t ldy, const int* skip, double* ws, size_t ws_elems) {
  const Operator& o = p->op;
  const OzOperand& A = which == LREP_OP_K ? *o.ozK : which == LREP_OP_M ? *o.ozM : *o.ozB;
  cudaError_t e = oz_apply(A, c, X, ldx, Y, ldy, ws,
                           ws_elems * sizeof(double), o.tc_err, skip, p->stream);
  if (e != cudaSuccess)
    return p->fail(LREP_ERR_CUDA, std::string("sliced product: ") + cudaGetErrorString(e));
  return LREP_OK;
}

bool cg_fused(lrep_problem p) {
  return want_tc(p) && p->op.kind == OP_DENSE && p->op.tcK && p->op.tcM;
}

lrep_status apply_cg_partials(lrep_problem p, int which, int c, const double* X, int64_t ldx,
                              bool x_split, const int* skip, double* ws, size_t ws_elems,
                              CgFused* out) {
  const Operator& o = p->op;
  if (!cg_fused(p)) return p->fail(LREP_ERR_STATE, "mixed precision operator split missing");
  const cudaError_t e = tc_product_partials(which == LREP_OP_K ? *o.tcK : *o.tcM, o.n, c, X,
                                            ldx, x_split, ws, ws_elems * sizeof(double),
                                            o.tc_err, skip, p->stream);
  if (e != cudaSuccess)
    return p->fail(LREP_ERR_CUDA, std::string("tensor-core product: ") + cudaGetErrorString(e));
  const TcBuffers b = tc_buffers(ws, o.n, c);
  *out = CgFused{b.part, b.splits, b.xhi, b.xlo, b.ldb};
  return LREP_OK;
}

lrep_status apply_op_cg(lrep_problem p, int which, int c, const double* X,
                        int64_t ldx, double* Y, int64_t ldy, const int* skip,
                        double* ws, size_t ws_elems) {
  if (!want_tc(p)) return apply_op(p, which, c, X, ldx, Y, ldy, skip, ws, ws_elems);
  const Operator& o = p->op;
  if (o.kind == OP_STENCIL) {  // float32 arithmetic, float64 loads and stores
    const cudaError_t e = stencil_apply(true, o.nx, o.ny, o.nz, o.coef_h2,
                                        which == LREP_OP_K ? o.dK : o.dM, c, X, ldx, Y, ldy,
                                        skip, p->stream);
    if (e != cudaSuccess)
      return p->fail(LREP_ERR_CUDA, std::string("stencil product: ") + cudaGetErrorString(e));
    return LREP_OK;
  }
  if (o.kind == OP_SPECTRAL) {  // float32 transforms
    const int dims[3] = {o.nx, o.ny, o.nz};
    const cudaError_t e = spectral_apply(true, dims, o.spec_scale,
                                         which == LREP_OP_K ? o.dK : o.dM, c, X, ldx, Y, ldy,
                                         skip, p->stream);
    if (e != cudaSuccess)
      return p->fail(LREP_ERR_CUDA, std::string("spectral product: ") + cudaGetErrorString(e));
    return LREP_OK;
  }
  if (!o.tcK) return p->fail(LREP_ERR_STATE, "mixed precision operator split missing");
  cudaError_t e = tc_apply(which == LREP_OP_K ? *o.tcK : *o.tcM, o.n, c, X, ldx, Y, ldy, ws,
                           ws_elems * sizeof(double), o.tc_err, skip, p->stream);
  if (e != cudaSuccess)
    return p->fail(LREP_ERR_CUDA, std::string("tensor-core product: ") + cudaGetErrorString(e));
  return LREP_OK;
}

}  // namespace lrep
