// extern "C" entry points of lrep.h and lrep_ops.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/lrep.h"
#include "../../include/lrep_ops.h"
#include "oz.h"
#include "problem.h"

using namespace lrep;

std::atomic<long long> lrep::g_launches{0};

namespace {

thread_local std::string g_err;  // errors of calls without a problem

int64_t pad_ld(int64_t n) { return ((n + 31) / 32) * 32; }

bool valid_mem(int32_t mem) {
  return mem == LREP_MEM_HOST || mem == LREP_MEM_DEVICE_COPY || mem == LREP_MEM_DEVICE_BORROW;
}

lrep_status cuda_fail(lrep_problem p, const char* what, cudaError_t e) {
  const std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  if (p) return p->fail(LREP_ERR_CUDA, m);
  g_err = m;
  return LREP_ERR_CUDA;
}

#define PCK(p, expr)                                       \
  do {                                                     \
    cudaError_t _e = (expr);                               \
    if (_e != cudaSuccess) return cuda_fail(p, #expr, _e); \
  } while (0)

lrep_problem new_problem(int64_t n, void* stream) {
  lrep_problem p = new lrep_problem_s();
  p->stream = (cudaStream_t)stream;
  p->op.n = n;
  lrep_default_options(&p->opts);
  return p;
}

// device copy of a column-major n x c block (source host or device) with
// the library's padded leading dimension
lrep_status copy_block(lrep_problem p, const double* src, int64_t ld_src, int64_t n,
                       int64_t c, double** dst_out) {
  const int64_t ld = pad_ld(n);
  double* dst = nullptr;
  PCK(p, cudaMalloc(&dst, sizeof(double) * ld * std::max<int64_t>(c, 1)));
  p->op.owned.push_back(dst);
  PCK(p, cudaMemcpy2DAsync(dst, ld * sizeof(double), src, ld_src * sizeof(double),
                           n * sizeof(double), c, cudaMemcpyDefault, p->stream));
  *dst_out = dst;
  return LREP_OK;
}

template <class T>
lrep_status copy_array(lrep_problem p, const T* src, int64_t count, T** dst_out) {
  T* dst = nullptr;
  PCK(p, cudaMalloc(&dst, sizeof(T) * std::max<int64_t>(count, 1)));
  p->op.owned.push_back(dst);
  if (count > 0)
    PCK(p, cudaMemcpyAsync(dst, src, sizeof(T) * count, cudaMemcpyDefault, p->stream));
  *dst_out = dst;
  return LREP_OK;
}

__global__ void ab_to_km_kernel(int64_t cnt, double* a, double* b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double x = a[i], y = b[i];
    a[i] = x - y;
    b[i] = x + y;
  }
}

// per-device scratch pool of the op-level entry points
struct Pool {
  std::mutex mu;
  Arena arena[16];
};
Pool g_pool;

lrep_status pool_take(size_t elems, double** out, void* stream) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 16) return cuda_fail(nullptr, "cudaGetDevice", e);
  std::lock_guard<std::mutex> g(g_pool.mu);
  Arena& A = g_pool.arena[dev];
  const size_t bytes = (elems + 64) * sizeof(double);
  if (A.cap < bytes) {
    e = A.reserve(std::max(bytes, (size_t)1 << 20), (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, "scratch pool", e);
  }
  *out = reinterpret_cast<double*>(A.base);
  return LREP_OK;
}

}  // namespace

namespace lrep {
void set_global_error(const char* msg) { g_err = msg; }
lrep_status apply_op_cg(lrep_problem p, int which, int c, const double* X,
                        int64_t ldx, double* Y, int64_t ldy, const int* skip,
                        double* ws, size_t ws_elems);
}

extern "C" {

void lrep_default_options(lrep_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->struct_size = (int32_t)sizeof(lrep_options);
  o->precision = LREP_PREC_FP64;
  o->s = 3;
  o->ngs = 1;
  o->cg_maxit = 20;
  o->cg_tol = 1e-2;
  o->maxit = 500;
  o->discard_tol = 1e-10;
  o->seed = 0;
  o->refresh_every = 8;
  o->rebiorth_tol = 1e-12;
  o->verbose = 0;
  o->profile = 0;
}

lrep_status lrep_create_dense(lrep_problem* out, int64_t n, const double* P1,
                              const double* P2, int64_t ld, int32_t form,
                              int32_t mem, void* stream) {
  if (!out || n <= 0 || !P1 || !P2 || ld < n || !valid_mem(mem) ||
      (form != LREP_FORM_AB && form != LREP_FORM_KM)) {
    g_err = "lrep_create_dense: invalid argument";
    return LREP_ERR_ARG;
  }
  if (mem == LREP_MEM_DEVICE_BORROW && form != LREP_FORM_KM) {
    g_err = "lrep_create_dense: borrowed matrices must be given as K, M";
    return LREP_ERR_ARG;
  }
  lrep_problem p = new_problem(n, stream);
  p->op.kind = OP_DENSE;
  if (mem == LREP_MEM_DEVICE_BORROW) {
    p->op.K = const_cast<double*>(P1);
    p->op.M = const_cast<double*>(P2);
    p->op.ld = ld;
  } else {
    lrep_status s = copy_block(p, P1, ld, n, n, &p->op.K);
    if (s == LREP_OK) s = copy_block(p, P2, ld, n, n, &p->op.M);
    if (s != LREP_OK) {
      g_err = p->err;
      lrep_destroy(p);
      return s;
    }
    p->op.ld = pad_ld(n);
    if (form == LREP_FORM_AB) km_from_ab(n, p->op.K, p->op.M, p->op.ld, p->stream);
  }
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) {
    g_err = std::string("lrep_create_dense: ") + cudaGetErrorString(e);
    lrep_destroy(p);
    return LREP_ERR_CUDA;
  }
  *out = p;
  return LREP_OK;
}

lrep_status lrep_create_csr(lrep_problem* out, int64_t n, int32_t form,
                            const int64_t* rp1, const int32_t* ci1, const double* v1,
                            const int64_t* rp2, const int32_t* ci2, const double* v2,
                            int32_t mem, void* stream) {
  if (!out || n <= 0 || !rp1 || !ci1 || !v1 || !rp2 || !ci2 || !v2 || !valid_mem(mem) ||
      (form != LREP_FORM_AB && form != LREP_FORM_KM)) {
    g_err = "lrep_create_csr: invalid argument";
    return LREP_ERR_ARG;
  }
  lrep_problem p = new_problem(n, stream);
  p->op.kind = OP_CSR;
  int64_t nnz1 = 0, nnz2 = 0;
  if (mem == LREP_MEM_HOST) {
    nnz1 = rp1[n];
    nnz2 = rp2[n];
  } else {
    cudaMemcpy(&nnz1, rp1 + n, sizeof(int64_t), cudaMemcpyDeviceToHost);
    cudaMemcpy(&nnz2, rp2 + n, sizeof(int64_t), cudaMemcpyDeviceToHost);
  }
  if (form == LREP_FORM_AB && (nnz1 != nnz2 || mem == LREP_MEM_DEVICE_BORROW)) {
    g_err = "lrep_create_csr: form AB needs equal patterns and copied inputs";
    lrep_destroy(p);
    return LREP_ERR_ARG;
  }
  if (mem == LREP_MEM_DEVICE_BORROW) {
    p->op.rpK = const_cast<int64_t*>(rp1); p->op.ciK = const_cast<int32_t*>(ci1);
    p->op.vK = const_cast<double*>(v1);
    p->op.rpM = const_cast<int64_t*>(rp2); p->op.ciM = const_cast<int32_t*>(ci2);
    p->op.vM = const_cast<double*>(v2);
  } else {
    lrep_status s = copy_array(p, rp1, n + 1, &p->op.rpK);
    if (s == LREP_OK) s = copy_array(p, ci1, nnz1, &p->op.ciK);
    if (s == LREP_OK) s = copy_array(p, v1, nnz1, &p->op.vK);
    if (s == LREP_OK) s = copy_array(p, rp2, n + 1, &p->op.rpM);
    if (s == LREP_OK) s = copy_array(p, ci2, nnz2, &p->op.ciM);
    if (s == LREP_OK) s = copy_array(p, v2, nnz2, &p->op.vM);
    if (s != LREP_OK) {
      g_err = p->err;
      lrep_destroy(p);
      return s;
    }
    if (form == LREP_FORM_AB)
      ab_to_km_kernel<<<256, 256, 0, p->stream>>>(nnz1, p->op.vK, p->op.vM); LREP_COUNT_LAUNCH();
  }
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) {
    g_err = std::string("lrep_create_csr: ") + cudaGetErrorString(e);
    lrep_destroy(p);
    return LREP_ERR_CUDA;
  }
  *out = p;
  return LREP_OK;
}

lrep_status lrep_create_spectral(lrep_problem* out, int32_t nx, int32_t ny, int32_t nz,
                                 const double* L, double lap_coef, const double* dK,
                                 const double* dM, int32_t mem, void* stream) {
  const int dims[3] = {nx, ny, nz};
  bool ok = out && L && dK && dM && valid_mem(mem) && std::isfinite(lap_coef);
  for (int a = 0; ok && a < 3; ++a)
    ok = (dims[a] == 1 || spectral_log2(dims[a]) > 0) && L[a] > 0.0 && std::isfinite(L[a]);
  if (!ok) {
    g_err = "lrep_create_spectral: invalid argument (grid sizes must be powers of two "
            "from 1 to 256, box lengths positive)";
    return LREP_ERR_ARG;
  }
  const int64_t n = (int64_t)nx * ny * nz;
  lrep_problem p = new_problem(n, stream);
  p->op.kind = OP_SPECTRAL;
  p->op.nx = nx; p->op.ny = ny; p->op.nz = nz;
  for (int a = 0; a < 3; ++a) {
    const double k1 = 2.0 * 3.14159265358979323846 / L[a];  // 2 pi / L
    p->op.spec_scale[a] = -lap_coef * k1 * k1 / (double)dims[a];
  }
  if (mem == LREP_MEM_DEVICE_BORROW) {
    p->op.dK = const_cast<double*>(dK);
    p->op.dM = const_cast<double*>(dM);
  } else {
    lrep_status s = copy_array(p, dK, n, &p->op.dK);
    if (s == LREP_OK) s = copy_array(p, dM, n, &p->op.dM);
    if (s != LREP_OK) {
      g_err = p->err;
      lrep_destroy(p);
      return s;
    }
  }
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) {
    g_err = std::string("lrep_create_spectral: ") + cudaGetErrorString(e);
    lrep_destroy(p);
    return LREP_ERR_CUDA;
  }
  *out = p;
  return LREP_OK;
}

lrep_status lrep_create_stencil(lrep_problem* out, int32_t nx, int32_t ny, int32_t nz,
                                double h, double lap_coef, const double* dK,
                                const double* dM, int32_t mem, void* stream) {
  if (!out || nx <= 0 || ny <= 0 || nz <= 0 || !(h > 0.0) || !dK || !dM || !valid_mem(mem)) {
    g_err = "lrep_create_stencil: invalid argument";
    return LREP_ERR_ARG;
  }
  const int64_t n = (int64_t)nx * ny * nz;
  lrep_problem p = new_problem(n, stream);
  p->op.kind = OP_STENCIL;
  p->op.nx = nx; p->op.ny = ny; p->op.nz = nz;
  p->op.coef_h2 = lap_coef / (h * h);
  if (mem == LREP_MEM_DEVICE_BORROW) {
    p->op.dK = const_cast<double*>(dK);
    p->op.dM = const_cast<double*>(dM);
  } else {
    lrep_status s = copy_array(p, dK, n, &p->op.dK);
    if (s == LREP_OK) s = copy_array(p, dM, n, &p->op.dM);
    if (s != LREP_OK) {
      g_err = p->err;
      lrep_destroy(p);
      return s;
    }
  }
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) {
    g_err = std::string("lrep_create_stencil: ") + cudaGetErrorString(e);
    lrep_destroy(p);
    return LREP_ERR_CUDA;
  }
  *out = p;
  return LREP_OK;
}

lrep_status lrep_create_operator(lrep_problem* out, int64_t n, lrep_apply_fn fn,
                                 void* user, void* stream) {
  if (!out || n <= 0 || !fn) {
    g_err = "lrep_create_operator: invalid argument";
    return LREP_ERR_ARG;
  }
  lrep_problem p = new_problem(n, stream);
  p->op.kind = OP_CALLBACK;
  p->op.fn = fn;
  p->op.user = user;
  *out = p;
  return LREP_OK;
}

lrep_status lrep_set_mass_dense(lrep_problem p, const double* B, int64_t ld, int32_t mem) {
  if (!p) return LREP_ERR_ARG;
  bosp_abort(p);  // a solve in progress ends with any change to the problem
  if (p->op.kind != OP_DENSE || !valid_mem(mem) || (B && ld < p->op.n))
    return p->fail(LREP_ERR_ARG, "lrep_set_mass_dense: dense problem and ld >= n required");
  const int64_t n = p->op.n;
  if (!B) {
    p->op.hasB = false;
    p->op.B = nullptr;
  } else if (mem == LREP_MEM_DEVICE_BORROW) {
    if (ld != p->op.ld)
      return p->fail(LREP_ERR_ARG, "lrep_set_mass_dense: a borrowed B needs the K, M leading "
                                   "dimension");
    p->op.B = const_cast<double*>(B);
    p->op.hasB = true;
  } else {
    double* dst = nullptr;
    PCK(p, cudaMalloc(&dst, sizeof(double) * p->op.ld * n));
    p->op.owned.push_back(dst);
    PCK(p, cudaMemcpy2DAsync(dst, p->op.ld * sizeof(double), B, ld * sizeof(double),
                             n * sizeof(double), n, cudaMemcpyDefault, p->stream));
    p->op.B = dst;
    p->op.hasB = true;
  }
  PCK(p, cudaStreamSynchronize(p->stream));
  // tensor-core forms of the operator now include (or drop) B
  if (p->opts.precision != LREP_PREC_FP64) return build_split(p);
  return LREP_OK;
}

lrep_status lrep_set_mass_csr(lrep_problem p, const int64_t* rowptr, const int32_t* colind,
                              const double* values, int32_t mem) {
  if (!p) return LREP_ERR_ARG;
  bosp_abort(p);  // a solve in progress ends with any change to the problem
  if (p->op.kind != OP_CSR || !valid_mem(mem) || (rowptr && (!colind || !values)))
    return p->fail(LREP_ERR_ARG, "lrep_set_mass_csr: CSR problem and all three arrays required");
  const int64_t n = p->op.n;
  if (!rowptr) {
    p->op.hasB = false;
    p->op.rpB = nullptr; p->op.ciB = nullptr; p->op.vB = nullptr;
    return LREP_OK;
  }
  if (mem == LREP_MEM_DEVICE_BORROW) {
    p->op.rpB = const_cast<int64_t*>(rowptr);
    p->op.ciB = const_cast<int32_t*>(colind);
    p->op.vB = const_cast<double*>(values);
  } else {
    int64_t nnz = 0;
    if (mem == LREP_MEM_HOST) {
      nnz = rowptr[n];
    } else {
      PCK(p, cudaMemcpyAsync(&nnz, rowptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost,
                             p->stream));
      PCK(p, cudaStreamSynchronize(p->stream));
    }
    lrep_status s = copy_array(p, rowptr, n + 1, &p->op.rpB);
    if (s == LREP_OK) s = copy_array(p, colind, nnz, &p->op.ciB);
    if (s == LREP_OK) s = copy_array(p, values, nnz, &p->op.vB);
    if (s != LREP_OK) return s;
  }
  p->op.hasB = true;
  PCK(p, cudaStreamSynchronize(p->stream));
  return LREP_OK;
}

lrep_status lrep_set_mass_callback(lrep_problem p, int32_t enable) {
  if (!p) return LREP_ERR_ARG;
  bosp_abort(p);  // a solve in progress ends with any change to the problem
  if (p->op.kind != OP_CALLBACK)
    return p->fail(LREP_ERR_ARG, "lrep_set_mass_callback: callback problem required");
  p->op.hasB = enable != 0;
  return LREP_OK;
}

lrep_status lrep_set_nullspace(lrep_problem p, int32_t r, const double* X0,
                               const double* Y0, int64_t ld, int32_t mem) {
  if (!p) return LREP_ERR_ARG;
  bosp_abort(p);  // a solve in progress ends with any change to the problem
  if (r < 0 || r > 64 || (r > 0 && (!X0 || ld < p->op.n)) || !valid_mem(mem))
    return p->fail(LREP_ERR_ARG, "lrep_set_nullspace: invalid argument (0 <= r <= 64)");
  p->r = r;
  p->X0in = p->Y0in = nullptr;
  if (r == 0) return LREP_OK;
  lrep_status s = copy_block(p, X0, ld, p->op.n, r, &p->X0in);
  if (s == LREP_OK && Y0) s = copy_block(p, Y0, ld, p->op.n, r, &p->Y0in);
  if (s != LREP_OK) return s;
  PCK(p, cudaStreamSynchronize(p->stream));
  return LREP_OK;
}

lrep_status lrep_find_nullspace(lrep_problem p, int32_t r_max, double tol, int32_t maxit,
                                double* X0_out, int64_t ld_out, int32_t mem_out,
                                int32_t* r_host, int32_t* iters_host) {
  if (!p) return LREP_ERR_ARG;
  bosp_abort(p);  // a solve in progress ends with any change to the problem
  if (r_max < 0 || r_max > 60 || !(tol > 0.0) || !(tol < 1.0) || maxit < 1 || !r_host ||
      (X0_out && (ld_out < p->op.n ||
                  (mem_out != LREP_MEM_HOST && mem_out != LREP_MEM_DEVICE_COPY))))
    return p->fail(LREP_ERR_ARG, "lrep_find_nullspace: invalid argument (0 <= r_max <= 60)");
  int r = 0, its = 0;
  const lrep_status s = find_nullspace(p, r_max, tol, maxit, &r, &its);
  if (s != LREP_OK) return s;
  if (X0_out && r > 0) {
    PCK(p, cudaMemcpy2DAsync(X0_out, ld_out * sizeof(double), p->X0in,
                             pad_ld(p->op.n) * sizeof(double), p->op.n * sizeof(double), r,
                             mem_out == LREP_MEM_HOST ? cudaMemcpyDeviceToHost
                                                      : cudaMemcpyDeviceToDevice,
                             p->stream));
    PCK(p, cudaStreamSynchronize(p->stream));
  }
  *r_host = r;
  if (iters_host) *iters_host = its;
  return LREP_OK;
}

lrep_status lrep_set_options(lrep_problem p, const lrep_options* o) {
  if (!p || !o) return LREP_ERR_ARG;
  bosp_abort(p);  // a solve in progress ends with any change to the problem
  if (o->struct_size != (int32_t)sizeof(lrep_options))
    return p->fail(LREP_ERR_ARG, "lrep_set_options: struct_size mismatch");
  if (o->s < 2 || o->ngs < 1 || o->cg_maxit < 0 || !(o->cg_tol > 0.0) || o->maxit < 1 ||
      !(o->discard_tol >= 0.0) || o->refresh_every < 1 || !(o->rebiorth_tol > 0.0) ||
      o->precision < LREP_PREC_FP64 || o->precision > LREP_PREC_MIXED_SLICED)
    return p->fail(LREP_ERR_ARG, "lrep_set_options: invalid value");
  if ((o->precision & LREP_PREC_MIXED_BF16X3) && p->op.kind != OP_DENSE &&
      p->op.kind != OP_SPECTRAL && p->op.kind != OP_STENCIL)
    return p->fail(LREP_ERR_ARG,
                   "mixed-precision CG products need a dense, stencil or spectral operator");
  const bool rebuild = (o->precision != p->opts.precision);
  p->opts = *o;
  if (rebuild) {
    free_split(p);
    if (o->precision != LREP_PREC_FP64) return build_split(p);
  }
  return LREP_OK;
}

lrep_status lrep_set_start(lrep_problem p, int32_t ncols, const double* U0,
                           const double* V0, int64_t ld, int32_t mem) {
  if (!p) return LREP_ERR_ARG;
  bosp_abort(p);  // a solve in progress ends with any change to the problem
  if (ncols < 0 || (ncols > 0 && (!U0 || !V0 || ld < p->op.n)) || !valid_mem(mem))
    return p->fail(LREP_ERR_ARG, "lrep_set_start: invalid argument");
  p->start_cols = ncols;
  p->U0 = p->V0 = nullptr;
  if (ncols == 0) return LREP_OK;
  lrep_status s = copy_block(p, U0, ld, p->op.n, ncols, &p->U0);
  if (s == LREP_OK) s = copy_block(p, V0, ld, p->op.n, ncols, &p->V0);
  if (s != LREP_OK) return s;
  PCK(p, cudaStreamSynchronize(p->stream));
  return LREP_OK;
}

lrep_status lrep_solve(lrep_problem p, int32_t nev, int32_t block, double tol) {
  if (!p) return LREP_ERR_ARG;
  if (nev < 1 || block < 1 || !(tol > 0.0))
    return p->fail(LREP_ERR_ARG, "lrep_solve: nev, block >= 1 and tol > 0 required");
  p->err.clear();
  return bosp_solve(p, nev, block, tol);
}

lrep_status lrep_solve_begin(lrep_problem p, int32_t nev, int32_t block, double tol) {
  if (!p) return LREP_ERR_ARG;
  if (nev < 1 || block < 1 || !(tol > 0.0))
    return p->fail(LREP_ERR_ARG, "lrep_solve_begin: nev, block >= 1 and tol > 0 required");
  p->err.clear();
  return bosp_begin(p, nev, block, tol);
}

lrep_status lrep_solve_advance(lrep_problem p, int32_t locks, int32_t* locked,
                               int32_t* done) {
  if (!p) return LREP_ERR_ARG;
  if (locks < 1) return p->fail(LREP_ERR_ARG, "lrep_solve_advance: locks >= 1 required");
  bool ended = false;
  int nlocked = 0;
  const lrep_status s = bosp_advance(p, locks, &ended, &nlocked);
  if (locked) *locked = nlocked;
  if (done) *done = ended ? 1 : 0;
  return s;
}

lrep_status lrep_query(lrep_problem p, int32_t what, void* dst, int64_t dst_bytes,
                       int32_t mem) {
  if (!p || !dst || dst_bytes < 0) return LREP_ERR_ARG;
  if (mem != LREP_MEM_HOST && mem != LREP_MEM_DEVICE_COPY)
    return p->fail(LREP_ERR_ARG, "lrep_query: mem must be HOST or DEVICE_COPY");
  // the profiles describe the work so far, also while a solve is in progress
  const bool profile_query =
      what == LREP_Q_PROFILE || what == LREP_Q_PROFILE_CG || what == LREP_Q_PROFILE_CLASSES;
  if (!p->solved && !(profile_query && p->active))
    return p->fail(LREP_ERR_STATE, "lrep_query before a solve");
  const int64_t n = p->op.n;
  const int nc = p->nconv;
  auto put = [&](const void* src, int64_t bytes, bool src_dev) -> lrep_status {
    if (bytes > dst_bytes) return p->fail(LREP_ERR_ARG, "lrep_query: destination too small");
    cudaMemcpyKind k = src_dev ? (mem == LREP_MEM_HOST ? cudaMemcpyDeviceToHost
                                                       : cudaMemcpyDeviceToDevice)
                               : (mem == LREP_MEM_HOST ? cudaMemcpyHostToHost
                                                       : cudaMemcpyHostToDevice);
    PCK(p, cudaMemcpy(dst, src, bytes, k));
    return LREP_OK;
  };
  auto put_block = [&](const double* src) -> lrep_status {
    const int64_t bytes = (int64_t)sizeof(double) * n * nc;
    if (bytes > dst_bytes) return p->fail(LREP_ERR_ARG, "lrep_query: destination too small");
    if (nc == 0) return LREP_OK;
    PCK(p, cudaStreamSynchronize(p->stream));
    PCK(p, cudaMemcpy2D(dst, n * sizeof(double), src, p->res_ld * sizeof(double),
                        n * sizeof(double), nc,
                        mem == LREP_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice));
    return LREP_OK;
  };
  switch (what) {
    case LREP_Q_NCONV: { int32_t v = nc; return put(&v, sizeof(v), false); }
    case LREP_Q_EIGVALS: return put(p->lam.data(), sizeof(double) * nc, false);
    case LREP_Q_X: return put_block(p->Xres);
    case LREP_Q_Y: return put_block(p->Yres);
    case LREP_Q_U:
    case LREP_Q_V: {
      const int64_t bytes = (int64_t)sizeof(double) * n * nc;
      if (bytes > dst_bytes) return p->fail(LREP_ERR_ARG, "lrep_query: destination too small");
      if (nc == 0) return LREP_OK;
      double *U = nullptr, *V = nullptr;
      PCK(p, cudaMalloc(&U, bytes));
      PCK(p, cudaMalloc(&V, bytes));
      cudaError_t e = uv_from_xy(n, nc, p->Xres, p->Yres, p->res_ld, U, V, n, p->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
      if (e == cudaSuccess)
        e = cudaMemcpy(dst, what == LREP_Q_U ? U : V, bytes,
                       mem == LREP_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice);
      cudaFree(U);
      cudaFree(V);
      if (e != cudaSuccess) return cuda_fail(p, "lrep_query U/V", e);
      return LREP_OK;
    }
    case LREP_Q_RESID: return put(p->resid.data(), sizeof(double) * nc, false);
    case LREP_Q_ITERS: { int32_t v = p->iters; return put(&v, sizeof(v), false); }
    case LREP_Q_MATVECS: { int64_t v = p->matvecs; return put(&v, sizeof(v), false); }
    case LREP_Q_TIMINGS: return put(p->timings, sizeof(p->timings), false);
    case LREP_Q_BIORTH_ERR: return put(&p->biorth_err, sizeof(double), false);
    case LREP_Q_HISTORY:
      return put(p->history.data(), sizeof(double) * (int64_t)p->history.size(), false);
    case LREP_Q_REBIORTHS: { int32_t v = p->rebiorths; return put(&v, sizeof(v), false); }
    case LREP_Q_PROFILE: return put(p->prof, sizeof(p->prof), false);
    case LREP_Q_PROFILE_CG: return put(p->prof_cg, sizeof(p->prof_cg), false);
    case LREP_Q_PROFILE_CLASSES: return put(p->prof_class, sizeof(p->prof_class), false);
    default: return p->fail(LREP_ERR_ARG, "lrep_query: unknown item");
  }
}

const char* lrep_last_error(lrep_problem p) {
  if (!p) return g_err.c_str();
  return p->err.c_str();
}

lrep_status lrep_destroy(lrep_problem p) {
  if (!p) return LREP_ERR_ARG;
  if (p->stream) cudaStreamSynchronize(p->stream);
  else cudaDeviceSynchronize();
  bosp_abort(p);
  free_split(p);
  for (void* q : p->op.owned) cudaFree(q);
  p->op.owned.clear();
  p->ws.release();
  p->op_arena.release();
  delete p;
  return LREP_OK;
}

// ------------------------------------------------------------- op level

lrep_status lrep_op_apply(lrep_problem p, int32_t op, int32_t ncols, const double* X,
                          int64_t ldx, double* Y, int64_t ldy) {
  if (!p || !X || !Y || ncols < 0 || ldx < p->op.n || ldy < p->op.n ||
      (op != LREP_OP_K && op != LREP_OP_M && !(op == LREP_OP_B && p->op.hasB)))
    return p ? p->fail(LREP_ERR_ARG, "lrep_op_apply: invalid argument") : LREP_ERR_ARG;
  const size_t ws = apply_ws_elems(p, ncols);
  if (p->op_arena.cap < (ws + 64) * sizeof(double))
    PCK(p, p->op_arena.reserve((ws + 64) * sizeof(double), p->stream));
  return apply_op(p, op, ncols, X, ldx, Y, ldy, nullptr,
                  reinterpret_cast<double*>(p->op_arena.base), ws);
}

lrep_status lrep_op_apply_cg(lrep_problem p, int32_t op, int32_t ncols, const double* X,
                             int64_t ldx, double* Y, int64_t ldy) {
  if (!p || !X || !Y || ncols < 0 || ldx < p->op.n || ldy < p->op.n ||
      (op != LREP_OP_K && op != LREP_OP_M))
    return p ? p->fail(LREP_ERR_ARG, "lrep_op_apply_cg: invalid argument") : LREP_ERR_ARG;
  const size_t ws = apply_ws_elems(p, ncols);
  if (p->op_arena.cap < (ws + 64) * sizeof(double))
    PCK(p, p->op_arena.reserve((ws + 64) * sizeof(double), p->stream));
  lrep_status s = apply_op_cg(p, op, ncols, X, ldx, Y, ldy, nullptr,
                              reinterpret_cast<double*>(p->op_arena.base), ws);
  if (s == LREP_OK && p->op.tc_err) {
    int h = 0;
    PCK(p, cudaMemcpyAsync(&h, p->op.tc_err, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    PCK(p, cudaStreamSynchronize(p->stream));
    if (h) return p->fail(LREP_ERR_CUDA, "tensor-core pipeline wait expired");
  }
  return s;
}

lrep_status lrep_op_cg(lrep_problem p, int32_t op, int32_t ncols, const double* B,
                       int64_t ldb, double* X, int64_t ldx, double tol, int32_t maxit,
                       int32_t* iters) {
  if (!p) return LREP_ERR_ARG;
  const int64_t n = p->op.n;
  if (!B || !X || ncols < 1 || ncols > 64 || ldb < n || ldx < n || maxit < 0 ||
      !(tol >= 0.0) || (op != LREP_OP_K && op != LREP_OP_M))
    return p->fail(LREP_ERR_ARG, "lrep_op_cg: invalid argument");
  bosp_abort(p);
  const size_t blk = (size_t)ldx * ncols;
  const size_t aws = apply_ws_elems(p, ncols);
  const size_t need = 3 * blk + cg_part_elems(n, ncols) + aws + 8 * (size_t)ncols + 4096;
  if (p->op_arena.cap < need * sizeof(double))
    PCK(p, p->op_arena.reserve(need * sizeof(double), p->stream));
  Arena& A = p->op_arena;
  A.off = 0;
  double* R = A.take<double>(blk);
  double* P = A.take<double>(blk);
  double* Q = A.take<double>(blk);
  CgState cg{};
  cg.rho = A.take<double>(ncols);
  cg.stop = A.take<double>(ncols);
  cg.alpha = A.take<double>(ncols);
  cg.beta = A.take<double>(ncols);
  cg.active = A.take<int>(ncols);
  cg.done = A.take<int>(8);
  cg.iters = A.take<int>(8);
  cg.counter = A.take<unsigned int>(128);
  cg.part = A.take<double>(cg_part_elems(n, ncols));
  double* ws = A.take<double>(aws + 1);
  if (!ws) return p->fail(LREP_ERR_NOMEM, "lrep_op_cg: workspace layout overflow");
  PCK(p, cudaMemsetAsync(cg.done, 0, 8 * sizeof(int), p->stream));
  PCK(p, cudaMemsetAsync(cg.iters, 0, 8 * sizeof(int), p->stream));
  PCK(p, cudaMemsetAsync(cg.counter, 0, 128 * sizeof(unsigned int), p->stream));
  PCK(p, cg_init(n, ncols, B, ldb, X, R, P, ldx, tol, cg, p->stream));
  const bool fused = cg_fused(p);  // as in the solver's CG
  const bool coop = fused && cg_step_coop_fits(n, ncols, cg);
  for (int it = 0; it < maxit; ++it) {
    if (fused) {
      CgFused fb{};
      const lrep_status s =
          apply_cg_partials(p, op, ncols, P, ldx, it > 0, cg.done, ws, aws, &fb);
      if (s != LREP_OK) return s;
      if (coop) {
        PCK(p, cg_step_coop(n, ncols, fb.part, fb.splits, X, R, P, ldx, cg, fb.xhi, fb.xlo,
                            fb.ldb, it, p->op.tc_err, p->stream));
        continue;
      }
      PCK(p, cg_sum_alpha(n, ncols, fb.part, fb.splits, P, Q, ldx, cg, p->stream));
      PCK(p, cg_update(n, ncols, X, R, P, Q, ldx, cg, p->stream));
      PCK(p, cg_pdir_split(n, ncols, R, P, ldx, cg, fb.xhi, fb.xlo, fb.ldb, p->stream));
      continue;
    }
    const lrep_status s = apply_op_cg(p, op, ncols, P, ldx, Q, ldx, cg.done, ws, aws);
    if (s != LREP_OK) return s;
    PCK(p, cg_alpha(n, ncols, P, Q, ldx, cg, p->stream));
    PCK(p, cg_update(n, ncols, X, R, P, Q, ldx, cg, p->stream));
    PCK(p, cg_pdir(n, ncols, R, P, ldx, cg, p->stream));
  }
  int h[2] = {0, 0};
  PCK(p, cudaMemcpyAsync(h, cg.iters, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  if (p->op.tc_err)
    PCK(p, cudaMemcpyAsync(h + 1, p->op.tc_err, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  PCK(p, cudaStreamSynchronize(p->stream));
  if (h[1]) return p->fail(LREP_ERR_CUDA, "tensor-core pipeline wait expired");
  if (iters) *iters = h[0];
  return LREP_OK;
}

lrep_status lrep_op_gram(int64_t n, int32_t a, int32_t b, const double* A, int64_t lda,
                         const double* B, int64_t ldb, double* G, int64_t ldg,
                         void* stream) {
  if (n < 0 || a < 0 || b < 0 || (a > 0 && (!A || lda < n)) || (b > 0 && (!B || ldb < n)) ||
      !G || ldg < a) {
    g_err = "lrep_op_gram: invalid argument";
    return LREP_ERR_ARG;
  }
  if (a == 0 || b == 0) return LREP_OK;
  const size_t need = gram_ws_elems(n, a, b);
  double* ws = nullptr;
  lrep_status s = pool_take(need, &ws, stream);
  if (s != LREP_OK) return s;
  if (n == 0) {
    cudaError_t e = cudaMemset2DAsync(G, ldg * sizeof(double), 0, a * sizeof(double), b,
                                      (cudaStream_t)stream);
    return e == cudaSuccess ? LREP_OK : cuda_fail(nullptr, "lrep_op_gram", e);
  }
  cudaError_t e = gram_f64(n, seg1(A, lda, a), seg1(B, ldb, b), G, ldg, ws, need,
                           (cudaStream_t)stream);
  return e == cudaSuccess ? LREP_OK : cuda_fail(nullptr, "lrep_op_gram", e);
}

// device word for the timeout flag of the sliced kernels (one per device)
int* sliced_err_flag(void* stream) {
  static int* flags[16] = {nullptr};
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 16) return nullptr;
  std::lock_guard<std::mutex> g(mu);
  if (!flags[dev]) {
    if (cudaMalloc(&flags[dev], sizeof(int)) != cudaSuccess) return flags[dev] = nullptr;
    if (cudaMemsetAsync(flags[dev], 0, sizeof(int), (cudaStream_t)stream) != cudaSuccess)
      return nullptr;
  }
  return flags[dev];
}

lrep_status sliced_status(const char* what, cudaError_t e, void* stream) {
  if (e != cudaSuccess) return cuda_fail(nullptr, what, e);
  int h = 0;
  int* f = sliced_err_flag(stream);
  e = cudaMemcpyAsync(&h, f, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(nullptr, what, e);
  if (h) {
    g_err = std::string(what) + ": tensor-core pipeline wait expired";
    return LREP_ERR_CUDA;
  }
  return LREP_OK;
}

lrep_status lrep_op_gram_sliced(int64_t n, int32_t a, int32_t b, const double* A, int64_t lda,
                                const double* B, int64_t ldb, double* G, int64_t ldg,
                                void* stream) {
  if (n < 1 || a < 0 || b < 0 || (a > 0 && (!A || lda < n)) || (b > 0 && (!B || ldb < n)) ||
      !G || ldg < a) {
    g_err = "lrep_op_gram_sliced: invalid argument";
    return LREP_ERR_ARG;
  }
  if (a == 0 || b == 0) return LREP_OK;
  const size_t need = oz_gram_ws_bytes(n, a, b) / sizeof(double) + 64;
  double* ws = nullptr;
  lrep_status s = pool_take(need, &ws, stream);
  if (s != LREP_OK) return s;
  int* err = sliced_err_flag(stream);
  if (!err) return cuda_fail(nullptr, "lrep_op_gram_sliced", cudaErrorMemoryAllocation);
  cudaError_t e = oz_gram(n, seg1(A, lda, a), seg1(B, ldb, b), G, ldg, ws,
                          need * sizeof(double), err, (cudaStream_t)stream);
  return sliced_status("lrep_op_gram_sliced", e, stream);
}

lrep_status lrep_op_update_sliced(int64_t n, int32_t k, int32_t c, double alpha,
                                  const double* A, int64_t lda, const double* B, int64_t ldb,
                                  double beta, double* C, int64_t ldc, void* stream) {
  if (n < 1 || k < 1 || k > 768 || c < 0 || !A || lda < n || !B || ldb < k || !C ||
      ldc < n || beta == 0.0) {
    g_err = "lrep_op_update_sliced: invalid argument (1 <= k <= 768, beta != 0)";
    return LREP_ERR_ARG;
  }
  if (c == 0) return LREP_OK;
  const size_t need = oz_update_ws_bytes(n, k, c) / sizeof(double) + 64;
  double* ws = nullptr;
  lrep_status s = pool_take(need, &ws, stream);
  if (s != LREP_OK) return s;
  int* err = sliced_err_flag(stream);
  if (!err) return cuda_fail(nullptr, "lrep_op_update_sliced", cudaErrorMemoryAllocation);
  cudaError_t e = oz_update(n, k, c, alpha, seg1(A, lda, k), B, ldb, beta, C, ldc, ws,
                            need * sizeof(double), err, (cudaStream_t)stream);
  return sliced_status("lrep_op_update_sliced", e, stream);
}

lrep_status lrep_op_update(int64_t n, int32_t k, int32_t c, double alpha, const double* A,
                           int64_t lda, const double* B, int64_t ldb, double beta,
                           double* C, int64_t ldc, void* stream) {
  if (n < 0 || k < 0 || c < 0 || (k > 0 && (!A || lda < n || !B || ldb < k)) || !C || ldc < n) {
    g_err = "lrep_op_update: invalid argument";
    return LREP_ERR_ARG;
  }
  cudaError_t e = update_f64(n, c, alpha, seg1(A, lda, k), B, ldb, beta, C, ldc,
                             (cudaStream_t)stream);
  return e == cudaSuccess ? LREP_OK : cuda_fail(nullptr, "lrep_op_update", e);
}

lrep_status lrep_op_small_lrep(int32_t d, const double* Khat, const double* Mhat, int32_t ld,
                               double* lam, double* Xh, double* Yh, int32_t ldo,
                               int32_t* info_host, void* stream) {
  if (d < 1 || d > 256 || !Khat || !Mhat || ld < d || !lam || !Xh || !Yh || ldo < d ||
      !info_host) {
    g_err = "lrep_op_small_lrep: invalid argument (1 <= d <= 256)";
    return LREP_ERR_ARG;
  }
  double* ws = nullptr;
  lrep_status s = pool_take(small_work_elems(d) + 8, &ws, stream);
  if (s != LREP_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  SmallJob J{};
  J.Khat = Khat; J.Mhat = Mhat; J.ld_in = ld; J.S = nullptr;
  J.lam = lam; J.Xh = Xh; J.Yh = Yh; J.ldo = ldo;
  J.work = ws + 8; J.info = reinterpret_cast<int*>(ws); J.biorth_err = ws + 1;
  J.d = d; J.w_prev = 0;
  cudaError_t e = small_lrep_one(J, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(info_host, ws, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? LREP_OK : cuda_fail(nullptr, "lrep_op_small_lrep", e);
}

lrep_status lrep_op_biorth(int64_t n, int32_t m, const double* W, const double* Z, int64_t ld,
                           double tau, double* P, double* Q, int64_t ldo,
                           int32_t* kept_host, void* stream) {
  if (n < 1 || m < 0 || m > 256 || !W || !Z || ld < n || !P || !Q || ldo < n || !kept_host ||
      !(tau >= 0.0)) {
    g_err = "lrep_op_biorth: invalid argument (m <= 256)";
    return LREP_ERR_ARG;
  }
  *kept_host = 0;
  if (m == 0) return LREP_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t g = (size_t)4 * m * m;
  const size_t need = gram_ws_elems(n, 2 * m, 2 * m) + g + 4 * (size_t)m * m +
                      biorth_coef_work_elems(m) + 2 * (size_t)ld * m + 64;
  double* ws = nullptr;
  lrep_status s = pool_take(need, &ws, stream);
  if (s != LREP_OK) return s;
  double* G2 = ws;
  double* cA = G2 + g;
  double* cB = cA + (size_t)m * m;
  double* cA2 = cB + (size_t)m * m;
  double* cB2 = cA2 + (size_t)m * m;
  double* cw = cB2 + (size_t)m * m;
  double* tA = cw + biorth_coef_work_elems(m);
  double* tB = tA + (size_t)ld * m;
  int* cnt = reinterpret_cast<int*>(tB + (size_t)ld * m);
  double* gws = reinterpret_cast<double*>(cnt + 16);
  gws = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(gws) + 255) & ~(uintptr_t)255);
  const size_t gws_elems = gram_ws_elems(n, 2 * m, 2 * m);
  int h = 0;
  Segs s1 = seg_push(seg1(W, ld, m), Z, ld, m);
  cudaError_t e = gram_f64(n, s1, s1, G2, 2 * m, gws, gws_elems, st);
  if (e == cudaSuccess) e = biorth_coef(m, G2, 2 * m, nullptr, nullptr, tau, cA, cB, m, cw, cnt, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, cnt, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(nullptr, "lrep_op_biorth", e);
  const int k1 = h;
  if (k1 == 0) return LREP_OK;
  e = update_f64(n, k1, 0.0, seg1(W, ld, m), cA, m, 1.0, tA, ld, st);
  if (e == cudaSuccess) e = update_f64(n, k1, 0.0, seg1(Z, ld, m), cB, m, 1.0, tB, ld, st);
  Segs s2 = seg_push(seg1(tA, ld, k1), tB, ld, k1);
  if (e == cudaSuccess) e = gram_f64(n, s2, s2, G2, 2 * k1, gws, gws_elems, st);
  if (e == cudaSuccess)
    e = biorth_coef(k1, G2, 2 * k1, nullptr, nullptr, tau, cA2, cB2, k1, cw, cnt, st, true);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, cnt, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(nullptr, "lrep_op_biorth", e);
  const int k2 = h;
  e = update_f64(n, k2, 0.0, seg1(tA, ld, k1), cA2, k1, 1.0, P, ldo, st);
  if (e == cudaSuccess) e = update_f64(n, k2, 0.0, seg1(tB, ld, k1), cB2, k1, 1.0, Q, ldo, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(nullptr, "lrep_op_biorth", e);
  *kept_host = k2;
  return LREP_OK;
}

lrep_status lrep_op_residuals(int64_t n, int32_t w, const double* X, const double* Y,
                              const double* KX, const double* MY, int64_t ld,
                              const double* lam, double* eps, void* stream) {
  if (n < 1 || w < 0 || !X || !Y || !KX || !MY || ld < n || !lam || !eps) {
    g_err = "lrep_op_residuals: invalid argument";
    return LREP_ERR_ARG;
  }
  if (w == 0) return LREP_OK;
  const size_t need = residual_ws_elems(n, w) + 64;
  double* ws = nullptr;
  lrep_status s = pool_take(need, &ws, stream);
  if (s != LREP_OK) return s;
  unsigned int* counter = reinterpret_cast<unsigned int*>(ws);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(counter, 0, 256, st);
  if (e == cudaSuccess)
    e = residuals_f64(n, w, X, Y, KX, MY, ld, lam, eps, ws + 32, counter, st);
  return e == cudaSuccess ? LREP_OK : cuda_fail(nullptr, "lrep_op_residuals", e);
}

lrep_status lrep_op_philox_normal(int64_t n, int32_t ncols, uint64_t seed, int32_t stream_id,
                                  double* out, int64_t ld, void* stream) {
  if (n < 0 || ncols < 0 || !out || ld < n) {
    g_err = "lrep_op_philox_normal: invalid argument";
    return LREP_ERR_ARG;
  }
  cudaError_t e = philox_normal(n, ncols, seed, stream_id, out, ld, (cudaStream_t)stream);
  return e == cudaSuccess ? LREP_OK : cuda_fail(nullptr, "lrep_op_philox_normal", e);
}

int64_t lrep_launch_count(void) { return (int64_t)g_launches.load(); }

}  // extern "C"
