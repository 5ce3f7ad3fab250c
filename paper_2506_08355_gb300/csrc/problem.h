// Problem object behind the C ABI (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lrep.h"
#include "kernels.h"

namespace lrep {
struct TcOperand;
struct OzOperand;

enum OpKind { OP_DENSE = 0, OP_CSR = 1, OP_STENCIL = 2, OP_CALLBACK = 3, OP_SPECTRAL = 4 };

// Device arena: one cudaMalloc, bump allocation, zero-filled on the stream
// that uses it.
struct Arena {
  char* base = nullptr;
  size_t cap = 0, off = 0;
  cudaError_t reserve(size_t bytes, cudaStream_t st);
  template <class T>
  T* take(size_t count) {
    const size_t a = 256;
    off = (off + a - 1) / a * a;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return off <= cap ? p : nullptr;
  }
  void release();
};

struct Operator {
  int kind = OP_DENSE;
  int64_t n = 0;
  // dense (column-major, ld)
  double* K = nullptr;
  double* M = nullptr;
  int64_t ld = 0;
  // csr
  int64_t* rpK = nullptr;
  int32_t* ciK = nullptr;
  double* vK = nullptr;
  int64_t* rpM = nullptr;
  int32_t* ciM = nullptr;
  double* vM = nullptr;
  // stencil and spectral (grid nx*ny*nz, diagonals dK, dM)
  int nx = 0, ny = 0, nz = 0;
  double coef_h2 = 0.0;
  double spec_scale[3] = {0.0, 0.0, 0.0};  // spectral: -coef (2 pi / L)^2 / N per axis
  double* dK = nullptr;
  double* dM = nullptr;
  // callback
  lrep_apply_fn fn = nullptr;
  void* user = nullptr;
  // mass matrix B of the generalized LREP (none: B = I)
  bool hasB = false;
  double* B = nullptr;  // dense (ld)
  int64_t* rpB = nullptr;  // csr
  int32_t* ciB = nullptr;
  double* vB = nullptr;
  struct OzOperand* ozB = nullptr;  // digit planes of dense B (FP64_SLICED)
  // mixed precision: bf16 hi/lo split of dense K and M (tc.h)
  struct TcOperand* tcK = nullptr;
  struct TcOperand* tcM = nullptr;
  // sliced float64 emulation: 7 bf16 digit planes of dense K and M (oz.h)
  struct OzOperand* ozK = nullptr;
  struct OzOperand* ozM = nullptr;
  int* tc_err = nullptr;  // pipeline timeout flag of the tensor-core kernels
  std::vector<void*> owned;  // device allocations freed at destroy
};

struct lrep_solver;  // forward

}  // namespace lrep

struct lrep_problem_s {
  lrep::Operator op;
  cudaStream_t stream = nullptr;
  lrep_options opts{};
  std::string err;
  // nullspace (caller input, device copies)
  int r = 0;
  double* X0in = nullptr;
  double* Y0in = nullptr;
  // optional start
  int start_cols = 0;
  double* U0 = nullptr;
  double* V0 = nullptr;
  // results (device, n x nconv, ld = res_ld)
  int nconv = 0;
  int nev_solved = 0;
  std::vector<double> lam;
  std::vector<double> resid;
  std::vector<double> history;
  double* Xres = nullptr;
  double* Yres = nullptr;
  int64_t res_ld = 0;
  int iters = 0;
  int64_t matvecs = 0;
  int rebiorths = 0;
  double timings[5] = {0, 0, 0, 0, 0};
  double biorth_err = 0.0;
  bool solved = false;
  // operator-product profile (options.profile)
  double prof[4] = {0, 0, 0, 0};
  double prof_cg[4] = {0, 0, 0, 0};  // CG-operator products alone
  double prof_class[2 * LREP_PC_COUNT] = {};  // (seconds, spans) per LREP_PC_* class
  // scratch for op-level calls on this problem
  lrep::Arena op_arena;
  // solver workspace (kept between solves of the same shape)
  lrep::Arena ws;
  // a solve in progress between lrep_solve_begin and its last
  // lrep_solve_advance (bosp.cu), else null
  void* active = nullptr;
  size_t ws_key[4] = {0, 0, 0, 0};

  lrep_status fail(lrep_status st, const std::string& msg) {
    err = msg;
    return st;
  }
};

namespace lrep {
// y = op(X) with the problem's float64 operator; skip: device flag (CG).
lrep_status apply_op(lrep_problem p, int which, int c, const double* X,
                     int64_t ldx, double* Y, int64_t ldy, const int* skip,
                     double* ws, size_t ws_elems);
// y = op(X) with the CG (possibly low-precision) operator.
lrep_status apply_op_cg(lrep_problem p, int which, int c, const double* X,
                        int64_t ldx, double* Y, int64_t ldy, const int* skip,
                        double* ws, size_t ws_elems);
// The CG product on the dense operator under the mixed precision in fused
// form (cg_fused): the tensor-core product leaves its split-K partials for
// cg_sum_alpha, and X's bf16 split may already be in place (written by
// cg_pdir_split); out receives where both live in ws.
struct CgFused {
  const float* part;
  int splits;
  void* xhi;
  void* xlo;
  int64_t ldb;
};
bool cg_fused(lrep_problem p);
lrep_status apply_cg_partials(lrep_problem p, int which, int c, const double* X, int64_t ldx,
                              bool x_split, const int* skip, double* ws, size_t ws_elems,
                              CgFused* out);
// y = op(X) by the sliced float64 emulation (dense, digit planes built)
lrep_status apply_sliced(lrep_problem p, int which, int c, const double* X,
                         int64_t ldx, double* Y, int64_t ldy, const int* skip,
                         double* ws, size_t ws_elems);
size_t apply_ws_elems(lrep_problem p, int c);
size_t apply_cg_ws_elems(lrep_problem p, int c);
// Cross-solve batching of the small projected problems (serving): when
// given, the solver hands each small LREP to the batcher instead of
// launching it; the batcher orders the caller's stream after the launch.
struct SmallBatcher {
  virtual ~SmallBatcher() {}
  virtual cudaError_t run(const SmallJob& job, cudaStream_t st) = 0;
};
lrep_status bosp_solve(lrep_problem p, int nev, int nb, double tol,
                       SmallBatcher* batcher = nullptr);
// the same solve in steps: begin (Steps 1-2), then advance by lock events
// until *ended; abort drops a solve in progress
lrep_status bosp_begin(lrep_problem p, int nev, int nb, double tol,
                       SmallBatcher* batcher = nullptr);
lrep_status bosp_advance(lrep_problem p, int max_locks, bool* ended, int* locked);
void bosp_abort(lrep_problem p);
// device bytes the solver's workspace needs for (nev, nb) on p
size_t bosp_footprint(lrep_problem p, int nev, int nb);
// orthonormal basis of N(K) by LOBPCG (nullspace.cu); sets p->r, p->X0in
lrep_status find_nullspace(lrep_problem p, int r_max, double tol, int maxit, int* r_out,
                           int* iters_out);
// tensor-core precisions: build what opts.precision needs of the bf16 hi/lo
// split and the digit planes of the dense operator
lrep_status build_split(lrep_problem p);
void free_split(lrep_problem p);
bool split_ready(lrep_problem p);
// device bytes build_split allocates for opts.precision
size_t split_bytes(lrep_problem p);
}  // namespace lrep
