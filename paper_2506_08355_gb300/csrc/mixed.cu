// Mixed-precision CG operator (LREP_PREC_MIXED_BF16X3): K and M split once
// into bfloat16 hi + lo parts; the CG products of eq. block_GS run on the
// tensor cores (k_tc.cu).  Every product that enters H^ (eq. hat_H) and
// every residual (eq. tol) stays float64.
#include <cuda_runtime.h>

#include "problem.h"
#include "tc.h"

namespace lrep {

lrep_status build_split(lrep_problem p) {
  Operator& o = p->op;
  if (o.kind != OP_DENSE) return p->fail(LREP_ERR_ARG, "mixed precision needs a dense operator");
  free_split(p);
  const int64_t n = o.n, ldb = tc_ld(n);
  const size_t bytes = (size_t)ldb * n * 2;
  TcOperand* t[2] = {new TcOperand(), new TcOperand()};
  o.tcK = t[0];
  o.tcM = t[1];
  const double* src[2] = {o.K, o.M};
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
  if (cudaMalloc(&o.tc_err, sizeof(int)) != cudaSuccess ||
      cudaMemsetAsync(o.tc_err, 0, sizeof(int), p->stream) != cudaSuccess ||
      cudaStreamSynchronize(p->stream) != cudaSuccess) {
    free_split(p);
    return p->fail(LREP_ERR_CUDA, "bf16 split: device error");
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
  if (o.tc_err) cudaFree(o.tc_err);
  o.tc_err = nullptr;
}

size_t apply_cg_ws_elems(lrep_problem p, int c) {
  if (p->opts.precision == LREP_PREC_MIXED_BF16X3 && p->op.tcK)
    return tc_ws_bytes(p->op.n, c) / sizeof(double) + 1;
  return 0;
}

lrep_status apply_op_cg(lrep_problem p, int which, int c, const double* X,
                        int64_t ldx, double* Y, int64_t ldy, const int* skip,
                        double* ws, size_t ws_elems) {
  if (p->opts.precision == LREP_PREC_FP64)
    return apply_op(p, which, c, X, ldx, Y, ldy, skip, ws, ws_elems);
  const Operator& o = p->op;
  if (!o.tcK) return p->fail(LREP_ERR_STATE, "mixed precision operator split missing");
  cudaError_t e = tc_apply(which == LREP_OP_K ? *o.tcK : *o.tcM, o.n, c, X, ldx, Y, ldy, ws,
                           ws_elems * sizeof(double), o.tc_err, skip, p->stream);
  if (e != cudaSuccess)
    return p->fail(LREP_ERR_CUDA, std::string("tensor-core product: ") + cudaGetErrorString(e));
  return LREP_OK;
}

}  // namespace lrep
