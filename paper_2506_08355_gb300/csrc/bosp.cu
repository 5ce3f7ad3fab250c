// Host driver of the BOSP iteration (Alg. 2 with the moving window of
// Section 3.3).  Every arithmetic step runs in the library's kernels on the
// problem's stream; the host keeps only the control state (window position,
// locked count, active set) and reads back a few scalars per iteration.
//
// Block layout: all n-row blocks are column-major with ld = n rounded up to
// 32.  U = [X | P | W] and V = [Y | Q | Z] live in two double-buffered
// arrays together with K U and M V; the next basis is assembled in the
// other buffer: Ritz vectors of the projected problem (pullback) at their
// Ritz index, followed by P~ and W~ after the window.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "oz.h"
#include "problem.h"

namespace lrep {

cudaError_t Arena::reserve(size_t bytes, cudaStream_t st) {
  release();
  if (bytes == 0) bytes = 256;
  cudaError_t e = cudaMalloc(&base, bytes);
  if (e != cudaSuccess) {
    base = nullptr;
    return e;
  }
  cap = bytes;
  off = 0;
  // zero-filled in the order of the stream that will use it (a legacy-stream
  // memset would not be ordered before work on a non-blocking stream)
  return cudaMemsetAsync(base, 0, bytes, st);
}

void Arena::release() {
  if (base) cudaFree(base);
  base = nullptr;
  cap = off = 0;
}

size_t apply_ws_elems(lrep_problem p, int c) {
  size_t w = 0;
  if (p->op.kind == OP_DENSE) w = dense_apply_ws_elems(p->op.n, c);
  return std::max(w, apply_cg_ws_elems(p, c));
}

lrep_status apply_op(lrep_problem p, int which, int c, const double* X,
                     int64_t ldx, double* Y, int64_t ldy, const int* skip,
                     double* ws, size_t ws_elems) {
  Operator& o = p->op;
  cudaError_t e = cudaSuccess;
  const bool isK = (which == LREP_OP_K);
  const bool isB = (which == LREP_OP_B);
  if (isB && !o.hasB) return p->fail(LREP_ERR_STATE, "no mass matrix B set");
  switch (o.kind) {
    case OP_DENSE:
      if (p->opts.precision & LREP_PREC_FP64_SLICED) {
        if (!o.ozK || (isB && !o.ozB))
          return p->fail(LREP_ERR_STATE, "digit planes of the operator missing");
        return apply_sliced(p, which, c, X, ldx, Y, ldy, skip, ws, ws_elems);
      }
      e = dense_apply_f64(o.n, c, isB ? o.B : isK ? o.K : o.M, o.ld, X, ldx, Y, ldy, ws,
                          ws_elems, skip, p->stream);
      break;
    case OP_CSR:
      e = csr_apply_f64(o.n, isB ? o.rpB : isK ? o.rpK : o.rpM,
                        isB ? o.ciB : isK ? o.ciK : o.ciM, isB ? o.vB : isK ? o.vK : o.vM,
                        c, X, ldx, Y, ldy, skip, p->stream);
      break;
    case OP_STENCIL:
      if (isB) return p->fail(LREP_ERR_STATE, "stencil problems have no mass matrix");
      e = stencil_apply_f64(o.nx, o.ny, o.nz, o.coef_h2, isK ? o.dK : o.dM, c,
                            X, ldx, Y, ldy, skip, p->stream);
      break;
    case OP_SPECTRAL: {
      if (isB) return p->fail(LREP_ERR_STATE, "spectral problems have no mass matrix");
      const int dims[3] = {o.nx, o.ny, o.nz};
      e = spectral_apply(false, dims, o.spec_scale, isK ? o.dK : o.dM, c, X, ldx, Y, ldy, skip,
                         p->stream);
      break;
    }
    case OP_CALLBACK: {
      if (skip) {
        int h = 0;
        e = cudaMemcpyAsync(&h, skip, sizeof(int), cudaMemcpyDeviceToHost, p->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
        if (e != cudaSuccess) break;
        if (h) return LREP_OK;
      }
      const int rc = o.fn(o.user, which, o.n, c, X, ldx, Y, ldy, (void*)p->stream);
      if (rc != 0)
        return p->fail(LREP_ERR_CALLBACK, "operator callback returned " + std::to_string(rc));
      e = cudaGetLastError();
      break;
    }
    default:
      return p->fail(LREP_ERR_STATE, "unknown operator kind");
  }
  if (e != cudaSuccess)
    return p->fail(LREP_ERR_CUDA, std::string("operator product: ") + cudaGetErrorString(e));
  return LREP_OK;
}

namespace {

__global__ void diag_copy_kernel(int m, const double* __restrict__ G, int ldg,
                                 double* __restrict__ out) {
  for (int i = threadIdx.x; i < m; i += blockDim.x) out[i] = G[i + (size_t)i * ldg];
}

#define LCK(expr)                                                                   \
  do {                                                                              \
    cudaError_t _e = (expr);                                                        \
    if (_e != cudaSuccess)                                                          \
      return p->fail(LREP_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
  } while (0)
#define LST(expr)                      \
  do {                                 \
    lrep_status _s = (expr);           \
    if (_s != LREP_OK) return _s;      \
  } while (0)

struct Solver {
  lrep_problem p;
  cudaStream_t st;
  int64_t n, ld;
  int nev, nb, w, r, dmax, C, Lmax, cgcols;
  bool moving;
  double tol;
  // double-buffered bases
  double* UX[2];
  double* UY[2];
  double* KX[2];
  double* MY[2];
  int cur = 0;
  int64_t off = 0;
  int d = 0;
  // deflation basis [X0 | locked], [Y0 | locked]; orthonormal basis of X0
  double *Dx, *Dy, *Q0;
  // generalized LREP (mass matrix B): B-companions of the bases, carried by
  // the same combinations (B U, B V, B Dx, B Dy) and fresh B W, B Z
  bool gen = false;
  double* BU[2];
  double* BV[2];
  double *BDx, *BDy, *BWr, *BZr, *BT, *BTW, *BTZ;
  // CG and W/Z blocks
  double *Rhs, *Zr, *Wr, *Rr, *Pr, *Qr, *TW, *TZ;
  // small matrices
  double *Kh, *Mh, *Sh, *Xh, *Yh, *swork, *Ph, *Qh, *pqwork, *G2, *cA, *cB, *cA2,
      *cB2, *cwork, *Cproj;
  double *lam_d, *eps_d, *berr_d, *refw2, *refz2, *lam_act, *lam_lock;
  int *info_d, *cnt_d, *act_d;
  // scratch for reductions and split-K
  double* ws;
  size_t ws_elems = 0, part_elems = 0;
  // sliced (tensor-core, float64-accurate) Grams and updates
  bool oz = false;
  uint8_t* ozws = nullptr;
  size_t ozws_bytes = 0;
  double* part;
  double *Rg, *Rinv, *Rwork;  // r x r scratch of the V0 normalisation
  unsigned int* counters;  // [0] residual [1] colnorm [2..] cg (128)
  CgState cg;
  // pinned host mirror
  struct Host {
    double lam[512];
    double eps[512];
    double berr;
    int info;
    int cnt[4];
    int cg_iters;
    int tc_err;
    int act[64];
    double lam_act[64];
    int pflag[520];  // profile: skip flag seen by each pending CG product
  }* h = nullptr;
  // host control state
  int ell = 0, w_prev = 0;
  bool stale = false;
  std::vector<double> locked;
  cudaEvent_t ev[6];
  bool events = false;
  SmallBatcher* batcher = nullptr;
  struct Pending {
    cudaEvent_t a, b;
    int c;     // product columns, or -1 for a span that is not a product
    bool cgop;
    int flag;  // index into h->pflag, or -1 (product always runs)
    int cls;   // LREP_PC_* class of the span
  };
  std::vector<cudaEvent_t> prof_free, prof_all;
  std::vector<Pending> prof_pending;

  lrep_status take_event(cudaEvent_t* e) {
    if (prof_free.empty()) {
      cudaEvent_t x;
      LCK(cudaEventCreate(&x));
      prof_all.push_back(x);
      prof_free.push_back(x);
    }
    *e = prof_free.back();
    prof_free.pop_back();
    return LREP_OK;
  }

  // after a stream synchronisation: account the timed products
  void resolve_profile() {
    for (const Pending& q : prof_pending) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, q.a, q.b);
      if (q.flag < 0 || h->pflag[q.flag] == 0) {
        if (q.c >= 0) account_product(q.c, ms, q.cgop);
        p->prof_class[2 * q.cls] += ms * 1e-3;
        p->prof_class[2 * q.cls + 1] += 1.0;
      }
      prof_free.push_back(q.a);
      prof_free.push_back(q.b);
    }
    prof_pending.clear();
  }

  double* Ucur() { return UX[cur] + off * ld; }
  double* Vcur() { return UY[cur] + off * ld; }
  double* KUcur() { return KX[cur] + off * ld; }
  double* MVcur() { return MY[cur] + off * ld; }
  int nx() const { return 1 - cur; }
  // B-companion of a basis block (the block itself when B = I)
  double* BUcur() { return gen ? BU[cur] + off * ld : Ucur(); }
  double* BVcur() { return gen ? BV[cur] + off * ld : Vcur(); }
  double* bux(int t) { return gen ? BU[t] : UX[t]; }
  double* bvy(int t) { return gen ? BV[t] : UY[t]; }
  double* bdx() { return gen ? BDx : Dx; }
  double* bdy() { return gen ? BDy : Dy; }

  lrep_status sync() {
    LCK(cudaStreamSynchronize(st));
    if (!prof_pending.empty()) resolve_profile();
    return LREP_OK;
  }

  // With options.profile set, f's device work is timed by CUDA events on
  // the solver's stream and accounted to class cls (LREP_Q_PROFILE_CLASSES).
  template <class F>
  lrep_status timed(int cls, F&& f) {
    if (!p->opts.profile) return f();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    LST(take_event(&e0));
    LST(take_event(&e1));
    LCK(cudaEventRecord(e0, st));
    const lrep_status s = f();
    if (s != LREP_OK) return s;
    LCK(cudaEventRecord(e1, st));
    prof_pending.push_back(Pending{e0, e1, -1, false, -1, cls});
    if (prof_pending.size() >= 512) LST(sync());
    return LREP_OK;
  }

  // Lays out every device buffer in the arena (dry run when A.base is
  // null: only the size is computed).
  void layout(Arena& A) {
    const int dd = 2 * dmax;
    const size_t sm = (size_t)dmax * dmax;
    const int rr = std::max(r, 1);
    auto blk = [&](int cols) { return A.take<double>((size_t)ld * cols); };
    for (int b = 0; b < 2; ++b) {
      UX[b] = blk(C); UY[b] = blk(C); KX[b] = blk(C); MY[b] = blk(C);
    }
    Dx = blk(r + nev); Dy = blk(r + nev); Q0 = blk(rr);
    if (gen) {
      for (int b = 0; b < 2; ++b) { BU[b] = blk(C); BV[b] = blk(C); }
      BDx = blk(r + nev); BDy = blk(r + nev);
      BWr = blk(cgcols); BZr = blk(cgcols); BT = blk(cgcols); BTW = blk(cgcols);
      BTZ = blk(cgcols);
    }
    Rhs = blk(cgcols); Zr = blk(cgcols); Wr = blk(cgcols); Rr = blk(cgcols);
    Pr = blk(cgcols); Qr = blk(cgcols); TW = blk(cgcols); TZ = blk(cgcols);
    Kh = A.take<double>(sm); Mh = A.take<double>(sm); Sh = A.take<double>(sm);
    Xh = A.take<double>(sm); Yh = A.take<double>(sm);
    swork = A.take<double>(small_work_elems(dmax));
    Ph = A.take<double>((size_t)dmax * cgcols); Qh = A.take<double>((size_t)dmax * cgcols);
    pqwork = A.take<double>(pq_work_elems(dmax, cgcols));
    G2 = A.take<double>((size_t)dd * dd);
    cA = A.take<double>(sm); cB = A.take<double>(sm);
    cA2 = A.take<double>(sm); cB2 = A.take<double>(sm);
    cwork = A.take<double>(biorth_coef_work_elems(dmax));
    Cproj = A.take<double>((size_t)Lmax * cgcols + (size_t)rr * dmax);
    Rg = A.take<double>((size_t)rr * rr);
    Rinv = A.take<double>((size_t)rr * rr);
    Rwork = A.take<double>((size_t)rr * rr);
    lam_d = A.take<double>(512); eps_d = A.take<double>(512);
    berr_d = A.take<double>(64); refw2 = A.take<double>(64); refz2 = A.take<double>(64);
    lam_act = A.take<double>(64); lam_lock = A.take<double>(std::max(nev, 64));
    info_d = A.take<int>(64); cnt_d = A.take<int>(64); act_d = A.take<int>(64);
    ws = A.take<double>(std::max<size_t>(ws_elems, 1));
    part = A.take<double>(std::max<size_t>(part_elems, 1));
    ozws = oz ? A.take<uint8_t>(ozws_bytes) : nullptr;
    counters = A.take<unsigned int>(256);
    cg.rho = A.take<double>(cgcols); cg.stop = A.take<double>(cgcols);
    cg.alpha = A.take<double>(cgcols); cg.beta = A.take<double>(cgcols);
    cg.active = A.take<int>(cgcols); cg.done = A.take<int>(8);
    cg.iters = A.take<int>(8);
    cg.part = part;
    cg.counter = counters + 2;
  }

  // sizes of every workspace piece (alloc and bosp_footprint)
  void plan() {
    gen = p->op.hasB;
    ld = ((n + 31) / 32) * 32;
    cgcols = std::max(nb, std::max(r, 1));
    const int dd = 2 * dmax;
    const int rr = std::max(r, 1);
    size_t wsz = 0;
    wsz = std::max(wsz, gram_ws_elems(n, dmax, dmax));
    wsz = std::max(wsz, gram_ws_elems(n, dd, dd));
    wsz = std::max(wsz, gram_ws_elems(n, Lmax, cgcols));
    wsz = std::max(wsz, gram_ws_elems(n, rr, std::max(rr, dmax)));
    wsz = std::max(wsz, gram_ws_elems(n, nev, nev));
    wsz = std::max(wsz, apply_ws_elems(p, std::max(C, cgcols)));
    ws_elems = wsz;
    oz = (p->opts.precision & LREP_PREC_FP64_SLICED) != 0;
    if (oz) {
      size_t b = 0;
      const int shapes[5][2] = {{dmax, dmax}, {dd, dd}, {Lmax, cgcols},
                                {rr, std::max(rr, dmax)}, {nev, nev}};
      for (const auto& sh : shapes) b = std::max(b, oz_gram_ws_bytes(n, sh[0], sh[1]));
      const int kmax = std::max(std::max(dmax, dd), std::max(Lmax, rr));
      b = std::max(b, oz_update_ws_bytes(n, kmax, std::max(dmax, std::max(cgcols, nev))));
      ozws_bytes = b + 512;
    }
    part_elems = std::max(residual_ws_elems(n, std::max(C, nev)),
                          std::max(colnorm_ws_elems(n, cgcols), cg_part_elems(n, cgcols)));
  }

  size_t bytes_needed() {
    plan();
    Arena dry;
    dry.base = nullptr;
    dry.cap = ~(size_t)0;
    layout(dry);
    return dry.off + 4096;
  }

  lrep_status alloc() {
    const size_t key[4] = {(size_t)n, (size_t)nev, (size_t)nb,
                           (size_t)(w * 1000 + r * 7 + p->opts.precision +
                                    (p->op.hasB ? 100000000 : 0))};
    const size_t bytes = bytes_needed();
    Arena& A = p->ws;
    bool reuse = (A.base != nullptr) && A.cap >= bytes;
    for (int i = 0; i < 4; ++i) reuse = reuse && p->ws_key[i] == key[i];
    if (!reuse) {
      LCK(A.reserve(bytes, st));
      for (int i = 0; i < 4; ++i) p->ws_key[i] = key[i];
    } else {
      LCK(cudaMemsetAsync(A.base, 0, A.cap, st));
    }
    A.off = 0;
    layout(A);
    if (A.off > A.cap) return p->fail(LREP_ERR_NOMEM, "workspace layout overflow");
    LCK(cudaMallocHost(&h, sizeof(Host)));
    return LREP_OK;
  }

  void release_host() {
    if (h) cudaFreeHost(h);
    h = nullptr;
    if (!prof_pending.empty() && cudaStreamSynchronize(st) == cudaSuccess) resolve_profile();
    for (auto& e : prof_all) cudaEventDestroy(e);
    prof_all.clear();
    prof_free.clear();
    if (events)
      for (auto& e : ev) cudaEventDestroy(e);
    events = false;
  }

  // ---------------------------------------------------------- primitives
  // float64-accurate products below this many flops stay on the FP64 units
  // (the sliced form costs ~5 launches)
  static constexpr double kSlicedMinFlops = 1.6e7;
  // The sliced route moves a fixed number of passes over its inputs and
  // digit planes (contraction padded to 64 for updates); the FP64 kernels
  // cost 2 flops per multiply-add at ~0.9 TF/s.  Grams take the sliced route
  // unless one side has fewer than 8 columns (a rank-few projection: the
  // digit passes over the long side then cost more than the FP64 product);
  // updates only where
  // the modelled sliced time (at ~5 TB/s) is below half the FP64 time, so
  // thin ones (k = 24, c = 8, say) stay FP64.
  static bool sliced_gram_pays(int a, int b) { return a >= 8 && b >= 8; }
  static bool sliced_update_pays(int k, int c) {
    const double ldk = (k + 63) / 64 * 64;
    const double t_sl = (8.0 * k + 28.0 * ldk + 24.0 * c) / 5e12;
    const double t_fp = 2.0 * k * c / 0.9e12;
    return t_sl < 0.5 * t_fp;
  }
  lrep_status gram(const Segs& A, const Segs& B, double* G, int64_t ldg) {
    return timed(LREP_PC_GRAM, [&] { return gram_(A, B, G, ldg); });
  }
  lrep_status gram_(const Segs& A, const Segs& B, double* G, int64_t ldg) {
    if (oz && 2.0 * n * A.total() * B.total() >= kSlicedMinFlops &&
        sliced_gram_pays(A.total(), B.total())) {
      LCK(oz_gram(n, A, B, G, ldg, ozws, ozws_bytes, p->op.tc_err, st));
      return LREP_OK;
    }
    // row slabs capped to the planned workspace (shapes outside the plan,
    // e.g. the 2 nb x 2 nb Gram of [W Z] on a long grid, use fewer slabs)
    LCK(gram_f64_capped(n, A, B, G, ldg, ws, ws_elems, st));
    return LREP_OK;
  }
  lrep_status update(int c, double alpha, const Segs& A, const double* B,
                     int64_t ldb, double beta, double* Cm) {
    return timed(LREP_PC_UPDATE, [&] { return update_(c, alpha, A, B, ldb, beta, Cm); });
  }
  lrep_status update_(int c, double alpha, const Segs& A, const double* B,
                      int64_t ldb, double beta, double* Cm) {
    if (oz && beta != 0.0 && 2.0 * n * A.total() * c >= kSlicedMinFlops &&
        sliced_update_pays(A.total(), c)) {
      LCK(oz_update(n, A.total(), c, alpha, A, B, ldb, beta, Cm, ld, ozws, ozws_bytes,
                    p->op.tc_err, st));
      return LREP_OK;
    }
    LCK(update_f64(n, c, alpha, A, B, ldb, beta, Cm, ld, st));
    return LREP_OK;
  }
  lrep_status apply(int which, int c, const double* X, double* Y,
                    const int* skip = nullptr, bool cgop = false) {
    if (c <= 0) return LREP_OK;
    return product(c, skip, cgop, [&] {
      return cgop ? apply_op_cg(p, which, c, X, ld, Y, ld, skip, ws, ws_elems)
                  : apply_op(p, which, c, X, ld, Y, ld, skip, ws, ws_elems);
    });
  }
  // one operator product `run` of c columns, counted and (when profiling)
  // timed as its class
  template <class F>
  lrep_status product(int c, const int* skip, bool cgop, F&& run) {
    p->matvecs += skip ? 0 : c;
    const bool prof = p->opts.profile != 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (prof) {
      LST(take_event(&e0));
      LST(take_event(&e1));
      LCK(cudaEventRecord(e0, st));
    }
    lrep_status s = run();
    if (prof && s == LREP_OK) {
      LCK(cudaEventRecord(e1, st));
      int flag = -1;
      if (skip) {  // products skipped on the device (converged CG) are not counted
        flag = (int)prof_pending.size();
        LCK(cudaMemcpyAsync(&h->pflag[flag], skip, sizeof(int), cudaMemcpyDeviceToHost, st));
      }
      prof_pending.push_back(Pending{e0, e1, c, cgop, flag, cgop ? LREP_PC_PROD_CG : LREP_PC_PROD});
      if (prof_pending.size() >= 512) LST(sync());
    }
    return s;
  }

  // algorithmic work of one product of c columns
  void account_product(int c, float ms, bool cgop) {
    const Operator& o = p->op;
    double nnz = 0.0, opbytes = 0.0;
    if (o.kind == OP_DENSE) {
      nnz = (double)n * n;
      const int prec = p->opts.precision;
      if (cgop && (prec & LREP_PREC_MIXED_BF16X3))
        opbytes = 4.0 * nnz;   // hi + lo bf16
      else if (prec & LREP_PREC_FP64_SLICED)
        opbytes = 14.0 * nnz;  // 7 bf16 digit planes
      else
        opbytes = 8.0 * nnz;
    } else if (o.kind == OP_STENCIL) {
      nnz = 7.0 * n;
      opbytes = 8.0 * n;  // the diagonal
    } else if (o.kind == OP_SPECTRAL) {
      // conventional FFT count: 5 N log2 N flops per complex line of N per
      // transform, two real lines per complex line, forward + inverse, and
      // the multiplier; as "nnz" per point (2 nnz c flops per product)
      double per = 1.0;  // the diagonal
      for (int a : {o.nx, o.ny, o.nz})
        if (a > 1) per += 0.5 * (5.0 * spectral_log2(a) + 1.0);
      nnz = per * n;
      opbytes = 8.0 * n;
    } else if (o.kind == OP_CSR) {
      nnz = 7.0 * n;
      opbytes = 12.0 * nnz + 8.0 * (n + 1);
    }
    const double add[4] = {ms * 1e-3, 1.0, 2.0 * nnz * c, opbytes + 16.0 * n * c};
    for (int i = 0; i < 4; ++i) {
      p->prof[i] += add[i];
      if (cgop) p->prof_cg[i] += add[i];
    }
  }

  // Block CG (one CG per column) for op * X = B; check_every > 0 reads the
  // done flag every that many iterations (long solves).
  lrep_status cg_solve(int which, int c, const double* B, double* X, double ctol,
                       int maxit, int check_every, bool cgop) {
    LCK(cudaMemsetAsync(cg.iters, 0, sizeof(int), st));
    LST(timed(LREP_PC_CGVEC, [&] {
      LCK(cg_init(n, c, B, ld, X, Rr, Pr, ld, ctol, cg, st));
      return LREP_OK;
    }));
    // dense operator under the mixed precision: the product's split-K sum
    // runs inside cg_sum_alpha and the directions' bf16 split inside
    // cg_pdir_split (two launches and passes fewer; the partial sum and
    // the split taken in fp32)
    // (in one cooperative launch when the block fits it)
    const bool fused = cgop && c > 0 && cg_fused(p);
    const bool coop = fused && cg_step_coop_fits(n, c, cg);
    if (coop) LCK(cudaMemsetAsync(cg.counter + 8, 0, (size_t)c * sizeof(unsigned int), st));
    for (int it = 0; it < maxit; ++it) {
      if (fused) {
        CgFused fb{};
        LST(product(c, cg.done, true, [&] {
          return apply_cg_partials(p, which, c, Pr, ld, it > 0, cg.done, ws, ws_elems, &fb);
        }));
        LST(timed(LREP_PC_CGVEC, [&] {
          if (coop) {
            LCK(cg_step_coop(n, c, fb.part, fb.splits, X, Rr, Pr, ld, cg, fb.xhi, fb.xlo, fb.ldb,
                             it, p->op.tc_err, st));
            return LREP_OK;
          }
          LCK(cg_sum_alpha(n, c, fb.part, fb.splits, Pr, Qr, ld, cg, st));
          LCK(cg_update(n, c, X, Rr, Pr, Qr, ld, cg, st));
          LCK(cg_pdir_split(n, c, Rr, Pr, ld, cg, fb.xhi, fb.xlo, fb.ldb, st));
          return LREP_OK;
        }));
      } else {
        LST(apply(which, c, Pr, Qr, cg.done, cgop));
        LST(timed(LREP_PC_CGVEC, [&] {
          LCK(cg_alpha(n, c, Pr, Qr, ld, cg, st));
          LCK(cg_update(n, c, X, Rr, Pr, Qr, ld, cg, st));
          LCK(cg_pdir(n, c, Rr, Pr, ld, cg, st));
          return LREP_OK;
        }));
      }
      if (check_every > 0 && (it + 1) % check_every == 0) {
        int done = 0;
        LCK(cudaMemcpyAsync(&h->cnt[3], cg.done, sizeof(int), cudaMemcpyDeviceToHost, st));
        LST(sync());
        done = h->cnt[3];
        if (done) break;
      }
    }
    LCK(cudaMemcpyAsync(&h->cg_iters, cg.iters, sizeof(int), cudaMemcpyDeviceToHost, st));
    LST(sync());
    p->matvecs += (int64_t)h->cg_iters * c;
    return LREP_OK;
  }

  // Alg. 1 for the n x m pair (A, B) in coefficient form, two passes; the
  // result (kept columns) is written to (outA, outB) and the same
  // combinations are applied to (KA, MB) when given.  ref2 (device,
  // squared entering norms) may be null.  Returns the kept count in *kept.
  lrep_status biorth_block(const double* Ain, const double* Bin, int m,
                           const double* KA, const double* MB, double* tA,
                           double* tB, double* tKA, double* tMB, double* outA,
                           double* outB, double* outKA, double* outMB,
                           const double* refa2, const double* refb2, int* kept,
                           const double* BAin = nullptr, const double* BBin = nullptr,
                           double* tBA = nullptr, double* tBB = nullptr,
                           double* outBA = nullptr, double* outBB = nullptr,
                           bool near_identity = false) {
    const double tau = p->opts.discard_tol;
    *kept = 0;
    if (m <= 0) return LREP_OK;
    const int ldg = 2 * dmax;
    // Gram [A B]^T [BA BB]: the B-inner products when companions are given
    const bool bc = BAin != nullptr;
    Segs s = seg_push(seg1(Ain, ld, m), Bin, ld, m);
    Segs sb = bc ? seg_push(seg1(BAin, ld, m), BBin, ld, m) : s;
    LST(gram(s, sb, G2, ldg));
    LST(timed(LREP_PC_ALG1, [&] {
      LCK(biorth_coef(m, G2, ldg, refa2, refb2, tau, cA, cB, dmax, cwork, cnt_d, st,
                      near_identity));
      return LREP_OK;
    }));
    LCK(cudaMemcpyAsync(&h->cnt[0], cnt_d, sizeof(int), cudaMemcpyDeviceToHost, st));
    LST(sync());
    const int k1 = h->cnt[0];
    if (k1 == 0) return LREP_OK;
    LST(update(k1, 0.0, seg1(Ain, ld, m), cA, dmax, 1.0, tA));
    LST(update(k1, 0.0, seg1(Bin, ld, m), cB, dmax, 1.0, tB));
    if (KA) {
      LST(update(k1, 0.0, seg1(KA, ld, m), cA, dmax, 1.0, tKA));
      LST(update(k1, 0.0, seg1(MB, ld, m), cB, dmax, 1.0, tMB));
    }
    if (bc) {
      LST(update(k1, 0.0, seg1(BAin, ld, m), cA, dmax, 1.0, tBA));
      LST(update(k1, 0.0, seg1(BBin, ld, m), cB, dmax, 1.0, tBB));
    }
    Segs s2 = seg_push(seg1(tA, ld, k1), tB, ld, k1);
    Segs s2b = bc ? seg_push(seg1(tBA, ld, k1), tBB, ld, k1) : s2;
    LST(gram(s2, s2b, G2, ldg));
    LST(timed(LREP_PC_ALG1, [&] {
      LCK(biorth_coef(k1, G2, ldg, nullptr, nullptr, tau, cA2, cB2, dmax, cwork, cnt_d, st,
                      true));
      return LREP_OK;
    }));
    LCK(cudaMemcpyAsync(&h->cnt[0], cnt_d, sizeof(int), cudaMemcpyDeviceToHost, st));
    LST(sync());
    const int k2 = h->cnt[0];
    LST(update(k2, 0.0, seg1(tA, ld, k1), cA2, dmax, 1.0, outA));
    LST(update(k2, 0.0, seg1(tB, ld, k1), cB2, dmax, 1.0, outB));
    if (KA) {
      LST(update(k2, 0.0, seg1(tKA, ld, k1), cA2, dmax, 1.0, outKA));
      LST(update(k2, 0.0, seg1(tMB, ld, k1), cB2, dmax, 1.0, outMB));
    }
    if (bc) {
      LST(update(k2, 0.0, seg1(tBA, ld, k1), cA2, dmax, 1.0, outBA));
      LST(update(k2, 0.0, seg1(tBB, ld, k1), cB2, dmax, 1.0, outBB));
    }
    *kept = k2;
    return LREP_OK;
  }

  // ------------------------------------------------------------- setup
  lrep_status setup() {
    // generalized nullspace (eq. V0_basis)
    if (r > 0) {
      LCK(copy_cols(n, r, p->X0in, ld, Dx, ld, st));
      // generalized LREP: M Y0 = B X0, X0^T B Y0 = I
      if (gen) LST(apply(LREP_OP_B, r, Dx, BDx));
      if (p->Y0in) {
        LCK(copy_cols(n, r, p->Y0in, ld, Dy, ld, st));
      } else {
        LST(cg_solve(LREP_OP_M, r, bdx(), Dy, 1e-14, 20000, 50, false));
      }
      double* T = UX[1];
      LST(gram(seg1(bdx(), ld, r), seg1(Dy, ld, r), Rg, r));
      LCK(chol_upper_inverse(r, Rg, r, Rinv, r, Rwork, info_d, st));
      LST(update(r, 0.0, seg1(Dx, ld, r), Rinv, r, 1.0, T));
      LCK(copy_cols(n, r, T, ld, Dx, ld, st));
      LST(update(r, 0.0, seg1(Dy, ld, r), Rinv, r, 1.0, T));
      LCK(copy_cols(n, r, T, ld, Dy, ld, st));
      if (gen) {
        LST(apply(LREP_OP_B, r, Dx, BDx));
        LST(apply(LREP_OP_B, r, Dy, BDy));
      }
      // orthonormal basis of span(X0) for the right-hand sides of K W = ...
      LCK(copy_cols(n, r, Dx, ld, Q0, ld, st));
      for (int pass = 0; pass < 2; ++pass) {
        LST(gram(seg1(Q0, ld, r), seg1(Q0, ld, r), Rg, r));
        LCK(chol_upper_inverse(r, Rg, r, Rinv, r, Rwork, info_d + 1, st));
        LST(update(r, 0.0, seg1(Q0, ld, r), Rinv, r, 1.0, T));
        LCK(copy_cols(n, r, T, ld, Q0, ld, st));
      }
      LCK(cudaMemcpyAsync(h->cnt, info_d, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
      LST(sync());
      if (h->cnt[0] || h->cnt[1])
        return p->fail(LREP_ERR_ARG, "nullspace basis X0 is rank deficient or X0^T M^-1 X0 not SPD");
    }
    // Step 1: random U, V
    const int d0 = (int)std::min<int64_t>(w + 2 * nb, n - r);
    if (p->U0 && p->start_cols >= d0) {
      LCK(copy_cols(n, d0, p->U0, ld, UX[0], ld, st));
      LCK(copy_cols(n, d0, p->V0, ld, UY[0], ld, st));
    } else {
      LCK(philox_normal(n, d0, p->opts.seed, 0, UX[0], ld, st));
      LCK(philox_normal(n, d0, p->opts.seed, 1, UY[0], ld, st));
    }
    // Step 2: project off V0 (twice) and biorthogonalise
    if (r > 0) {
      for (int pass = 0; pass < 2; ++pass) {
        LST(gram(seg1(bdy(), ld, r), seg1(UX[0], ld, d0), Cproj, r));
        LST(update(d0, 1.0, seg1(Dx, ld, r), Cproj, r, -1.0, UX[0]));
        LST(gram(seg1(bdx(), ld, r), seg1(UY[0], ld, d0), Cproj, r));
        LST(update(d0, 1.0, seg1(Dy, ld, r), Cproj, r, -1.0, UY[0]));
      }
    }
    int kept = 0;
    if (gen) {
      LST(apply(LREP_OP_B, d0, UX[0], BU[0]));
      LST(apply(LREP_OP_B, d0, UY[0], BV[0]));
      LST(biorth_block(UX[0], UY[0], d0, nullptr, nullptr, UX[1], UY[1], nullptr, nullptr,
                       UX[0], UY[0], nullptr, nullptr, nullptr, nullptr, &kept, BU[0], BV[0],
                       BU[1], BV[1], BU[0], BV[0]));
    } else {
      LST(biorth_block(UX[0], UY[0], d0, nullptr, nullptr, UX[1], UY[1], nullptr,
                       nullptr, UX[0], UY[0], nullptr, nullptr, nullptr, nullptr, &kept));
    }
    if (kept == 0) return p->fail(LREP_ERR_BREAKDOWN, "start block lost every column");
    cur = 0; off = 0; d = kept;
    LST(refresh());
    w_prev = std::min(w, d);
    return LREP_OK;
  }

  lrep_status refresh() {
    LST(apply(LREP_OP_K, d, Ucur(), KUcur()));
    LST(apply(LREP_OP_M, d, Vcur(), MVcur()));
    if (gen) {
      LST(apply(LREP_OP_B, d, Ucur(), BUcur()));
      LST(apply(LREP_OP_B, d, Vcur(), BVcur()));
    }
    stale = false;
    return LREP_OK;
  }

  // ----------------------------------------- Step 3 + Step 4 (one pass)
  // Grams, small LREP, pullback of Ritz pairs [0, e) into the next buffer
  // and their residuals; reads back lam, eps, info and the biorth error.
  lrep_status rayleigh_ritz(int e) {
    const Segs sU = seg1(Ucur(), ld, d), sV = seg1(Vcur(), ld, d);
    const Segs sKU = seg1(KUcur(), ld, d), sMV = seg1(MVcur(), ld, d);
    if (events) LCK(cudaEventRecord(ev[0], st));
    LST(gram(sU, sKU, Kh, dmax));
    LST(gram(sV, sMV, Mh, dmax));
    LST(gram(sU, seg1(BVcur(), ld, d), Sh, dmax));  // U^T B V (safeguard)
    SmallJob job{};
    job.Khat = Kh; job.Mhat = Mh; job.ld_in = dmax; job.S = Sh;
    job.lam = lam_d; job.Xh = Xh; job.Yh = Yh; job.ldo = dmax;
    job.work = swork; job.info = info_d; job.biorth_err = berr_d;
    job.d = d; job.w_prev = w_prev;
    LST(timed(LREP_PC_SMALL, [&] {
      if (batcher)
        LCK(batcher->run(job, st));
      else
        LCK(small_lrep_one(job, st));
      return LREP_OK;
    }));
    const int t = nx();
    LST(update(e, 0.0, sU, Xh, dmax, 1.0, UX[t]));
    LST(update(e, 0.0, sV, Yh, dmax, 1.0, UY[t]));
    LST(update(e, 0.0, sKU, Xh, dmax, 1.0, KX[t]));
    LST(update(e, 0.0, sMV, Yh, dmax, 1.0, MY[t]));
    if (gen) {
      LST(update(e, 0.0, seg1(BUcur(), ld, d), Xh, dmax, 1.0, BU[t]));
      LST(update(e, 0.0, seg1(BVcur(), ld, d), Yh, dmax, 1.0, BV[t]));
    }
    if (events) LCK(cudaEventRecord(ev[1], st));
    LST(timed(LREP_PC_OTHER, [&] {
      LCK(residuals_f64(n, e, UX[t], UY[t], KX[t], MY[t], ld, lam_d, eps_d, part,
                        counters, st, gen ? BU[t] : nullptr, gen ? BV[t] : nullptr));
      return LREP_OK;
    }));
    LCK(cudaMemcpyAsync(h->lam, lam_d, sizeof(double) * d, cudaMemcpyDeviceToHost, st));
    LCK(cudaMemcpyAsync(h->eps, eps_d, sizeof(double) * e, cudaMemcpyDeviceToHost, st));
    LCK(cudaMemcpyAsync(&h->berr, berr_d, sizeof(double), cudaMemcpyDeviceToHost, st));
    LCK(cudaMemcpyAsync(&h->info, info_d, sizeof(int), cudaMemcpyDeviceToHost, st));
    h->tc_err = 0;
    if (p->op.tc_err)
      LCK(cudaMemcpyAsync(&h->tc_err, p->op.tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (events) LCK(cudaEventRecord(ev[2], st));
    LST(sync());
    if (h->tc_err)
      return p->fail(LREP_ERR_CUDA, "tensor-core pipeline wait expired (code " +
                                        std::to_string(h->tc_err) + ")");
    if (h->info == 1 || h->info == 2)
      return p->fail(LREP_ERR_NOT_SPD,
                     h->info == 1 ? "projected K^ = U^T K U is not positive definite "
                                    "(is K singular without a nullspace basis?)"
                                  : "projected M^ = V^T M V is not positive definite");
    for (int i = 0; i < e; ++i)
      if (!std::isfinite(h->eps[i]) || !std::isfinite(h->lam[i]))
        return p->fail(LREP_ERR_BREAKDOWN, "non-finite Ritz value or residual");
    return LREP_OK;
  }

  // Rayleigh-Ritz with one recovery: K^ or M^ that fails to be positive
  // definite (products carried by recurrence drifted, or U, V lost
  // biorthogonality) is retried once from fresh products of a
  // re-biorthogonalised basis.
  lrep_status rayleigh_ritz_safe(int* e) {
    lrep_status s = rayleigh_ritz(*e);
    if (s != LREP_ERR_NOT_SPD) return s;
    p->err.clear();
    LST(refresh());
    LST(rebiorth());
    LST(refresh());
    *e = std::min(d, std::min(w, d) + (moving ? 2 * nb : 0));
    return rayleigh_ritz(*e);
  }

  // safeguard: Step 2's biorthogonalisation applied to the current U, V;
  // K U and M V follow by the same combinations.
  lrep_status rebiorth() {
    const int t = nx();
    int kept = 0;
    if (gen)
      LST(biorth_block(Ucur(), Vcur(), d, KUcur(), MVcur(), UX[t], UY[t], KX[t], MY[t],
                       UX[cur], UY[cur], KX[cur], MY[cur], nullptr, nullptr, &kept, BUcur(),
                       BVcur(), BU[t], BV[t], BU[cur], BV[cur], true));
    else
      LST(biorth_block(Ucur(), Vcur(), d, KUcur(), MVcur(), UX[t], UY[t], KX[t], MY[t],
                       UX[cur], UY[cur], KX[cur], MY[cur], nullptr, nullptr, &kept, nullptr,
                       nullptr, nullptr, nullptr, nullptr, nullptr, true));
    if (kept == 0) return p->fail(LREP_ERR_BREAKDOWN, "re-biorthogonalisation lost every column");
    off = 0;
    d = kept;
    p->rebiorths++;
    return LREP_OK;
  }

  lrep_status lock(int first, int count) {
    const int t = nx();
    LCK(copy_cols(n, count, UX[t] + (int64_t)first * ld, ld, Dx + (int64_t)(r + ell) * ld, ld, st));
    LCK(copy_cols(n, count, UY[t] + (int64_t)first * ld, ld, Dy + (int64_t)(r + ell) * ld, ld, st));
    if (gen) {
      LCK(copy_cols(n, count, BU[t] + (int64_t)first * ld, ld, BDx + (int64_t)(r + ell) * ld, ld,
                    st));
      LCK(copy_cols(n, count, BV[t] + (int64_t)first * ld, ld, BDy + (int64_t)(r + ell) * ld, ld,
                    st));
    }
    // the new pairs are made biorthogonal to the earlier ones (X0 and the
    // pairs locked before), twice: over the ~100 iterations between two
    // locks the window drifts from the locked pairs by rounding (1.5e-9 in
    // X^T Y at n = 32768 without this), since only W, Z are projected each
    // iteration (eq. update_W/Z); the change is of that size and leaves the
    // residuals below tol (they are recomputed with fresh products at the end)
    const int prev = r + ell;
    if (prev > 0) {
      double* Xn = Dx + (int64_t)prev * ld;
      double* Yn = Dy + (int64_t)prev * ld;
      for (int c0 = 0; c0 < count; c0 += cgcols) {
        const int cc = std::min(cgcols, count - c0);
        const int64_t o = (int64_t)c0 * ld;
        for (int pass = 0; pass < 2; ++pass) {
          LST(gram(seg1(bdy(), ld, prev), seg1(Xn + o, ld, cc), Cproj, prev));
          LST(update(cc, 1.0, seg1(Dx, ld, prev), Cproj, prev, -1.0, Xn + o));
          if (gen) LST(update(cc, 1.0, seg1(BDx, ld, prev), Cproj, prev, -1.0, BDx + prev * ld + o));
          LST(gram(seg1(bdx(), ld, prev), seg1(Yn + o, ld, cc), Cproj, prev));
          LST(update(cc, 1.0, seg1(Dy, ld, prev), Cproj, prev, -1.0, Yn + o));
          if (gen) LST(update(cc, 1.0, seg1(BDy, ld, prev), Cproj, prev, -1.0, BDy + prev * ld + o));
        }
      }
    }
    for (int i = 0; i < count; ++i) locked.push_back(h->lam[first + i]);
    ell += count;
    return LREP_OK;
  }

  // ------------------------------------------------------------- solve
  // outer-iteration state kept between calls of iterate()
  int it_ = 0;
  bool converged_ = false;

  lrep_status begin() {
    auto t0 = std::chrono::steady_clock::now();
    LST(setup());
    LST(sync());
    p->timings[0] += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    it_ = 0;
    converged_ = false;
    return LREP_OK;
  }

  // Outer iterations of Alg. 2 until `max_locks` lock events (Section 3.3:
  // each locks 2 nb converged pairs, or the last nev - locked) have happened
  // in this call, or the solve has ended (*ended = true: converged or maxit;
  // the results are then final and the return value is the solve's status).
  // Stops only at iteration boundaries, so the next call continues exactly
  // where this one left off.
  lrep_status iterate(int max_locks, bool* ended) {
    *ended = false;
    const int maxit = p->opts.maxit;
    const int every = std::max(1, p->opts.refresh_every);
    int locks = 0;
    while (it_ < maxit) {
      const int it = ++it_;
      if (it > 1 && it % every == 0) LST(refresh());
      const int want_max = std::min(w, d);
      int e = std::min(d, want_max + (moving ? 2 * nb : 0));
      LST(rayleigh_ritz_safe(&e));
      if (h->berr > p->opts.rebiorth_tol) {
        // the safeguard fires on a basis that is biorthogonal to ~1e-12, so
        // Alg. 1's coefficients are near the identity and K U, M V (B U,
        // B V) follow them accurately: no fresh products here (the refresh
        // schedule and the pre-decision refresh still apply)
        LST(rebiorth());
        stale = true;
        e = std::min(d, std::min(w, d) + (moving ? 2 * nb : 0));
        LST(rayleigh_ritz_safe(&e));
      }
      int wv = std::min(w, d);
      int want = std::min(wv, nev - ell);
      int c = 0;
      while (c < wv && h->eps[c] < tol) ++c;
      const bool decide = (c >= want) || (moving && c >= 2 * nb);
      if (decide && stale) {
        // decisions are taken on freshly computed products
        LST(refresh());
        e = std::min(d, std::min(w, d) + (moving ? 2 * nb : 0));
        LST(rayleigh_ritz_safe(&e));
        wv = std::min(w, d);
        want = std::min(wv, nev - ell);
        c = 0;
        while (c < wv && h->eps[c] < tol) ++c;
      }
      double emax = 0.0;
      for (int i = 0; i < std::min(wv, want); ++i) emax = std::max(emax, h->eps[i]);
      p->history.push_back(emax);
      if (p->opts.verbose)
        fprintf(stderr, "[lrep] it %d d %d locked %d conv %d/%d maxres %.3e lam0 %.12e\n",
                it, d, ell, c, want, emax, h->lam[0]);
      if (c >= want) {
        LST(lock(0, want));
        converged_ = true;
        break;
      }
      int win0 = 0;
      if (moving && c >= 2 * nb) {
        LST(lock(0, 2 * nb));
        ++locks;
        win0 = 2 * nb;
        wv = std::min(w, d - win0);
      }
      const int end = win0 + wv;
      // active set: the first nb unconverged pairs of the window
      int na = 0;
      for (int j = win0; j < end && na < nb; ++j)
        if (!(h->eps[j] < tol)) {
          h->act[na] = j;
          h->lam_act[na] = h->lam[j];
          ++na;
        }
      if (na == 0) {  // everything in the window converged but not locked
        LST(lock(win0, std::min(wv, nev - ell)));
        ++locks;
        converged_ = ell >= nev;
        if (converged_) break;
        if (locks >= max_locks) return LREP_OK;
        continue;
      }
      LCK(cudaMemcpyAsync(act_d, h->act, sizeof(int) * na, cudaMemcpyHostToDevice, st));
      LCK(cudaMemcpyAsync(lam_act, h->lam_act, sizeof(double) * na, cudaMemcpyHostToDevice, st));
      LST(step5_6_7(win0, wv, end, na));
      if (d == 0) return p->fail(LREP_ERR_BREAKDOWN, "search space collapsed");
      if (locks >= max_locks) return LREP_OK;
    }
    *ended = true;
    p->iters = std::min(it_, maxit);
    LST(finalize());
    return converged_ ? LREP_OK : LREP_NOT_CONVERGED;
  }

  lrep_status step5_6_7(int win0, int wv, int end, int na) {
    const int t = nx();
    double* TX = UX[t];
    double* TY = UY[t];
    double* TK = KX[t];
    double* TM = MY[t];
    // Step 5: eq. hat_pq in R^d and Alg. 1 there (P is empty after a move)
    const bool with_p = (win0 == 0);
    if (with_p) {
      PqJob pj{};
      pj.Xh = Xh; pj.Yh = Yh; pj.ld = dmax; pj.d = d; pj.end = end;
      pj.w_prev = w_prev; pj.na = na; pj.act = act_d; pj.Ph = Ph; pj.Qh = Qh;
      pj.ldo = dmax; pj.work = pqwork; pj.count = cnt_d + 1; pj.tau = p->opts.discard_tol;
      LST(timed(LREP_PC_SMALL, [&] {
        LCK(small_pq(pj, st));
        return LREP_OK;
      }));
      LCK(cudaMemcpyAsync(&h->cnt[1], cnt_d + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    } else {
      h->cnt[1] = 0;
    }
    cudaEvent_t evp = ev[5];
    if (events) LCK(cudaEventRecord(ev[3], st));
    LCK(cudaEventRecord(evp, st));
    // Step 6: eq. block_GS, one CG per column, W^(0) = 0
    const bool cgop = true;
    double* Wsol = Wr;
    double* Zsol = Zr;
    for (int sweep = 0; sweep < std::max(1, p->opts.ngs); ++sweep) {
      // M Z = W Lambda + (X~ Lambda - M Y~); generalized: B W, B X~
      if (gen && sweep) LST(apply(LREP_OP_B, na, Wsol, BT));
      LST(timed(LREP_PC_OTHER, [&] {
        LCK(gather_combine(n, na, act_d, lam_act, bux(t), -1.0, TM, sweep ? lam_act : nullptr,
                           sweep ? (gen ? BT : Wsol) : nullptr, ld, Rhs, ld, st));
        return LREP_OK;
      }));
      LST(cg_solve(LREP_OP_M, na, Rhs, Zsol, p->opts.cg_tol, p->opts.cg_maxit, 0, cgop));
      // K W = Z Lambda + (Y~ Lambda - K X~), projected onto range(K);
      // generalized: B Z, B Y~
      if (gen) LST(apply(LREP_OP_B, na, Zsol, BT));
      LST(timed(LREP_PC_OTHER, [&] {
        LCK(gather_combine(n, na, act_d, lam_act, bvy(t), -1.0, TK, lam_act, gen ? BT : Zsol,
                           ld, Rhs, ld, st));
        return LREP_OK;
      }));
      if (r > 0) {
        LST(gram(seg1(Q0, ld, r), seg1(Rhs, ld, na), Cproj, r));
        LST(update(na, 1.0, seg1(Q0, ld, r), Cproj, r, -1.0, Rhs));
      }
      LST(cg_solve(LREP_OP_K, na, Rhs, Wsol, p->opts.cg_tol, p->opts.cg_maxit, 0, cgop));
    }
    // entering norms for the discard rule (B-norms when generalized: B W, B Z
    // are formed here and follow W, Z through the projections below)
    if (gen) {
      LST(apply(LREP_OP_B, na, Wsol, BWr));
      LST(apply(LREP_OP_B, na, Zsol, BZr));
      LST(gram(seg1(Wsol, ld, na), seg1(BWr, ld, na), G2, na));
      diag_copy_kernel<<<1, 64, 0, st>>>(na, G2, na, refw2); LREP_COUNT_LAUNCH();
      LST(gram(seg1(Zsol, ld, na), seg1(BZr, ld, na), G2, na));
      diag_copy_kernel<<<1, 64, 0, st>>>(na, G2, na, refz2); LREP_COUNT_LAUNCH();
      LCK(cudaGetLastError());
    } else {
      LST(timed(LREP_PC_OTHER, [&] {
        LCK(colnorm2_f64(n, na, Wsol, ld, refw2, part, counters + 1, st));
        LCK(colnorm2_f64(n, na, Zsol, ld, refz2, part, counters + 1, st));
        return LREP_OK;
      }));
    }
    // P~ = U P^, Q~ = V Q^ and their products by the same combinations
    LCK(cudaEventSynchronize(evp));
    const int pc = h->cnt[1];
    const Segs sU = seg1(Ucur(), ld, d), sV = seg1(Vcur(), ld, d);
    const Segs sKU = seg1(KUcur(), ld, d), sMV = seg1(MVcur(), ld, d);
    if (pc > 0) {
      LST(update(pc, 0.0, sU, Ph, dmax, 1.0, TX + (int64_t)end * ld));
      LST(update(pc, 0.0, sV, Qh, dmax, 1.0, TY + (int64_t)end * ld));
      LST(update(pc, 0.0, sKU, Ph, dmax, 1.0, TK + (int64_t)end * ld));
      LST(update(pc, 0.0, sMV, Qh, dmax, 1.0, TM + (int64_t)end * ld));
      if (gen) {
        LST(update(pc, 0.0, seg1(BUcur(), ld, d), Ph, dmax, 1.0, BU[t] + (int64_t)end * ld));
        LST(update(pc, 0.0, seg1(BVcur(), ld, d), Qh, dmax, 1.0, BV[t] + (int64_t)end * ld));
      }
    }
    // eq. update_W / update_Z against [X0, X_locked, X~, P~] (applied twice)
    const int nw = wv + pc;
    const Segs SA = seg_push(seg1(Dx, ld, r + ell), TX + (int64_t)win0 * ld, ld, nw);
    const Segs SB = seg_push(seg1(Dy, ld, r + ell), TY + (int64_t)win0 * ld, ld, nw);
    // B-companions: [B Dx, B X~, B P~], [B Dy, B Y~, B Q~]
    const Segs SAb = seg_push(seg1(bdx(), ld, r + ell), bux(t) + (int64_t)win0 * ld, ld, nw);
    const Segs SBb = seg_push(seg1(bdy(), ld, r + ell), bvy(t) + (int64_t)win0 * ld, ld, nw);
    const int L = r + ell + nw;
    for (int pass = 0; pass < 2; ++pass) {
      LST(gram(SBb, seg1(Wsol, ld, na), Cproj, L));
      LST(update(na, 1.0, SA, Cproj, L, -1.0, Wsol));
      if (gen) LST(update(na, 1.0, SAb, Cproj, L, -1.0, BWr));
      LST(gram(SAb, seg1(Zsol, ld, na), Cproj, L));
      LST(update(na, 1.0, SB, Cproj, L, -1.0, Zsol));
      if (gen) LST(update(na, 1.0, SBb, Cproj, L, -1.0, BZr));
    }
    // Alg. 1 on (W~, Z~) with the discard rule, into place after P~
    const int wpos = end + pc;
    int m = 0;
    if (gen)
      LST(biorth_block(Wsol, Zsol, na, nullptr, nullptr, TW, TZ, nullptr, nullptr,
                       TX + (int64_t)wpos * ld, TY + (int64_t)wpos * ld, nullptr, nullptr,
                       refw2, refz2, &m, BWr, BZr, BTW, BTZ, BU[t] + (int64_t)wpos * ld,
                       BV[t] + (int64_t)wpos * ld));
    else
      LST(biorth_block(Wsol, Zsol, na, nullptr, nullptr, TW, TZ, nullptr, nullptr,
                       TX + (int64_t)wpos * ld, TY + (int64_t)wpos * ld, nullptr, nullptr,
                       refw2, refz2, &m));
    // fresh products K W~, M Z~
    LST(apply(LREP_OP_K, m, TX + (int64_t)wpos * ld, TK + (int64_t)wpos * ld));
    LST(apply(LREP_OP_M, m, TY + (int64_t)wpos * ld, TM + (int64_t)wpos * ld));
    if (events) LCK(cudaEventRecord(ev[4], st));
    LST(sync());
    if (events) {
      float a = 0, b = 0, c2 = 0, e2 = 0;
      cudaEventElapsedTime(&a, ev[0], ev[1]);
      cudaEventElapsedTime(&b, ev[1], ev[2]);
      cudaEventElapsedTime(&c2, ev[2], ev[3]);
      cudaEventElapsedTime(&e2, ev[3], ev[4]);
      p->timings[1] += a * 1e-3; p->timings[2] += b * 1e-3;
      p->timings[3] += c2 * 1e-3; p->timings[4] += e2 * 1e-3;
    }
    // Step 7: U = [X~, P~, W~], V = [Y~, Q~, Z~]
    cur = t;
    off = win0;
    d = wv + pc + m;
    w_prev = wv;
    stale = true;
    return LREP_OK;
  }

  lrep_status finalize() {
    const int nc = ell;
    p->nconv = nc;
    p->lam = locked;
    p->Xres = Dx + (int64_t)r * ld;
    p->Yres = Dy + (int64_t)r * ld;
    p->res_ld = ld;
    p->resid.assign(nc, 0.0);
    p->biorth_err = 0.0;
    if (nc == 0) return LREP_OK;
    // biorthogonality of the result (X^T B Y; before the sign fix, which
    // flips X, Y but not their B-companions)
    if (nc <= 512) {
      double* G = (2 * dmax * 2 * dmax >= nc * nc) ? G2 : nullptr;
      if (G) {
        LST(gram(seg1(p->Xres, ld, nc), seg1(bdy() + (int64_t)r * ld, ld, nc), G, nc));
        LCK(biorth_error(nc, G, nc, berr_d, st));
        LCK(cudaMemcpyAsync(&h->berr, berr_d, sizeof(double), cudaMemcpyDeviceToHost, st));
        LST(sync());
        p->biorth_err = h->berr;
      }
    }
    LCK(fix_sign(n, nc, p->Xres, p->Yres, ld, st));
    LCK(cudaMemcpyAsync(lam_lock, locked.data(), sizeof(double) * nc, cudaMemcpyHostToDevice, st));
    // final residuals with fresh float64 products (eq. tol)
    for (int c0 = 0; c0 < nc; c0 += C) {
      const int cc = std::min(C, nc - c0);
      double* X = p->Xres + (int64_t)c0 * ld;
      double* Y = p->Yres + (int64_t)c0 * ld;
      LST(apply(LREP_OP_K, cc, X, KX[0]));
      LST(apply(LREP_OP_M, cc, Y, MY[0]));
      if (gen) {  // fresh B X, B Y into the free U, V buffers
        LST(apply(LREP_OP_B, cc, X, UX[0]));
        LST(apply(LREP_OP_B, cc, Y, UY[0]));
      }
      LCK(residuals_f64(n, cc, X, Y, KX[0], MY[0], ld, lam_lock + c0, eps_d, part,
                        counters, st, gen ? UX[0] : nullptr, gen ? UY[0] : nullptr));
      LCK(cudaMemcpyAsync(h->eps, eps_d, sizeof(double) * cc, cudaMemcpyDeviceToHost, st));
      LST(sync());
      for (int i = 0; i < cc; ++i) p->resid[c0 + i] = h->eps[i];
    }
    return LREP_OK;
  }
};

}  // namespace

static void configure(Solver& S, lrep_problem p, int nev, int nb, double tol) {
  S.p = p;
  S.st = p->stream;
  S.n = p->op.n;
  S.r = p->r;
  S.nev = nev;
  S.nb = std::min(nb, nev);
  S.moving = S.nb < nev;
  S.w = (int)std::min<int64_t>(S.moving ? (int64_t)p->opts.s * S.nb : nev, S.n - S.r);
  S.dmax = S.w + 2 * S.nb;
  S.C = S.w + 4 * S.nb;
  S.Lmax = S.r + nev + S.dmax;
  S.tol = tol;
}

size_t bosp_footprint(lrep_problem p, int nev, int nb) {
  Solver S{};
  configure(S, p, nev, nb, 1.0);
  return S.bytes_needed();
}

// A solve in progress (lrep_solve_begin / lrep_solve_advance): the solver
// lives on the heap between calls and owns its pinned mirror and events.
struct ActiveSolve {
  Solver S{};
};

void bosp_abort(lrep_problem p) {
  if (!p->active) return;
  ActiveSolve* a = static_cast<ActiveSolve*>(p->active);
  a->S.release_host();
  delete a;
  p->active = nullptr;
}

static lrep_status bosp_end(lrep_problem p, lrep_status s, int nev) {
  bosp_abort(p);
  p->solved = (s == LREP_OK || s == LREP_NOT_CONVERGED);
  p->nev_solved = nev;
  return s;
}

lrep_status bosp_begin(lrep_problem p, int nev, int nb, double tol, SmallBatcher* batcher) {
  bosp_abort(p);
  ActiveSolve* a = new ActiveSolve();
  Solver& S = a->S;
  configure(S, p, nev, nb, tol);
  S.batcher = batcher;
  for (double& v : p->prof) v = 0.0;
  for (double& v : p->prof_cg) v = 0.0;
  for (double& v : p->prof_class) v = 0.0;
  p->solved = false;
  if (S.dmax > 256) {
    delete a;
    return p->fail(LREP_ERR_ARG, "window + 2*block exceeds 256 columns");
  }
  if (S.nb > 64) {
    delete a;
    return p->fail(LREP_ERR_ARG, "block exceeds 64");
  }
  if ((int64_t)S.dmax > S.n - S.r) {
    delete a;
    return p->fail(LREP_ERR_ARG, "n too small for nev/block");
  }
  p->history.clear();
  p->iters = 0;
  p->matvecs = 0;
  p->rebiorths = 0;
  p->nconv = 0;
  for (double& t : p->timings) t = 0.0;
  p->active = a;
  lrep_status s = S.alloc();
  if (s == LREP_OK) {
    S.events = true;
    for (auto& e : S.ev)
      if (cudaEventCreate(&e) != cudaSuccess) S.events = false;
    s = S.begin();
  }
  if (s != LREP_OK) return bosp_end(p, s, nev);
  return LREP_OK;
}

lrep_status bosp_advance(lrep_problem p, int max_locks, bool* ended, int* locked) {
  *ended = false;
  *locked = 0;
  if (!p->active) return p->fail(LREP_ERR_STATE, "no solve in progress (lrep_solve_begin)");
  ActiveSolve* a = static_cast<ActiveSolve*>(p->active);
  const int nev = a->S.nev;
  bool done = false;
  lrep_status s = a->S.iterate(max_locks < 1 ? 1 : max_locks, &done);
  *locked = a->S.ell;
  if (done || (s != LREP_OK && s != LREP_NOT_CONVERGED)) {
    *ended = true;
    return bosp_end(p, s, nev);
  }
  return LREP_OK;
}

lrep_status bosp_solve(lrep_problem p, int nev, int nb, double tol, SmallBatcher* batcher) {
  LST(bosp_begin(p, nev, nb, tol, batcher));
  bool ended = false;
  int locked = 0;
  return bosp_advance(p, 1 << 30, &ended, &locked);
}

}  // namespace lrep
