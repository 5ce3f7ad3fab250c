// Mixed-precision CG operator: K, M split into bf16 hi + lo parts whose
// three cross products run on the tensor cores with fp32 accumulation
// (eq. block_GS only needs a relative residual of cg_tol).
#include <cuda_runtime.h>

#include "problem.h"

namespace lrep {

lrep_status build_split(lrep_problem p) {
  return p->fail(LREP_ERR_ARG, "mixed precision (bf16x3 tensor-core CG products) is not built in this library");
}

void free_split(lrep_problem p) {
  for (void** q : {&p->op.Khi, &p->op.Klo, &p->op.Mhi, &p->op.Mlo}) {
    if (*q) cudaFree(*q);
    *q = nullptr;
  }
}

lrep_status apply_op_cg(lrep_problem p, int which, int c, const double* X,
                        int64_t ldx, double* Y, int64_t ldy, const int* skip,
                        double* ws, size_t ws_elems) {
  if (p->opts.precision == LREP_PREC_FP64)
    return apply_op(p, which, c, X, ldx, Y, ldy, skip, ws, ws_elems);
  return p->fail(LREP_ERR_STATE, "mixed precision operator missing");
}

}  // namespace lrep
