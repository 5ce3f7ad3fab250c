// lrep_op_gram_noalloc: the tall-skinny Gram G = A^T B without any device
// allocation.
//
// Some callers cannot allocate device memory when they call us: a process
// whose device memory has been reserved up front by another allocator (a
// framework's caching allocator holding nearly all of HBM, so cudaMalloc can
// fail mid-run), or a latency-critical loop that cannot accept cudaMalloc /
// cudaFree (which may synchronise the device and stall other streams).  This
// entry point keeps the Gram's split-K partials in a fixed array in device
// memory that is part of the library image, so the call itself allocates
// nothing; the caller still passes A, B and G.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/lrep_ops.h"
#include "kernels.h"

namespace lrep {
void set_global_error(const char* msg);  // capi.cu (lrep_last_error(NULL))
}

namespace {

// 2^19 doubles = 4 MiB of partials per device, held by every GPU that loads
// the library until the process exits.
constexpr size_t kGramScratchElems = (size_t)1 << 19;
static __device__ __align__(256) double lrep_gram_scratch[kGramScratchElems];

std::mutex g_scratch_mu;
double* g_scratch_addr[64] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (host code cannot use the symbol itself as a device pointer).
lrep_status scratch_address(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) {
    lrep::set_global_error("lrep_op_gram_noalloc: no current CUDA device");
    return LREP_ERR_CUDA;
  }
  std::lock_guard<std::mutex> g(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, lrep_gram_scratch);
    if (e != cudaSuccess || p == nullptr) {
      lrep::set_global_error("lrep_op_gram_noalloc: cudaGetSymbolAddress failed");
      return LREP_ERR_CUDA;
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return LREP_OK;
}

}  // namespace

extern "C" lrep_status lrep_op_gram_noalloc(int64_t n, int32_t a, int32_t b, const double* A,
                                            int64_t lda, const double* B, int64_t ldb,
                                            double* G, int64_t ldg, void* stream) {
  if (n < 0 || a < 0 || b < 0 || (a > 0 && (!A || lda < n)) || (b > 0 && (!B || ldb < n)) ||
      !G || ldg < a) {
    lrep::set_global_error("lrep_op_gram_noalloc: invalid argument");
    return LREP_ERR_ARG;
  }
  if ((int64_t)a * b > LREP_GRAM_NOALLOC_MAX_AB) {
    lrep::set_global_error(
        "lrep_op_gram_noalloc: a * b exceeds the static scratch limit "
        "LREP_GRAM_NOALLOC_MAX_AB (65536); use lrep_op_gram");
    return LREP_ERR_ARG;
  }
  if (a == 0 || b == 0) return LREP_OK;
  double* ws = nullptr;
  lrep_status s = scratch_address(&ws);
  if (s != LREP_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  // an error left by an earlier, unrelated call is not this call's failure
  (void)cudaGetLastError();
  cudaError_t e;
  if (n == 0)
    e = cudaMemset2DAsync(G, ldg * sizeof(double), 0, a * sizeof(double), b, st);
  else
    e = lrep::gram_f64_capped(n, lrep::seg1(A, lda, a), lrep::seg1(B, ldb, b), G, ldg, ws,
                              kGramScratchElems, st);
  if (e != cudaSuccess) {
    const std::string msg = std::string("lrep_op_gram_noalloc: kernel launch failed: ") +
                            cudaGetErrorString(e);
    lrep::set_global_error(msg.c_str());
    return LREP_ERR_CUDA;
  }
  return LREP_OK;
}
