// A variant of mbar_lse_pass for callers that must not allocate device
// memory: its per-CTA partial sums and completion counter live in a fixed
// array compiled into this library instead of a caller-provided buffer.
#include "common.cuh"
#include "kernels.cuh"

namespace bumbar {
namespace {

// 1 MiB, 256-byte aligned; every GPU that loads the library holds it until
// the process exits. The first 256 bytes hold the completion counter and the
// error word, the rest the partial row sums.
constexpr size_t kStaticScratchBytes = size_t(1) << 20;
static __device__ __align__(256) unsigned char g_lse_scratch[kStaticScratchBytes];

// Device address of g_lse_scratch on the current device (the host-side name
// g_lse_scratch is only a stand-in, not a device address). Looked up on
// every call: the lookup allocates nothing, and a cached address would go
// stale if the device's primary context were reset and the module reloaded.
mbar_status static_scratch(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_lse_scratch);
  if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(g_lse_scratch)");
  *out = p;
  return MBAR_OK;
}

}  // namespace
}  // namespace bumbar

using namespace bumbar;

extern "C" {

size_t mbar_lse_static_scratch_bytes(void) { return kStaticScratchBytes; }

mbar_status mbar_lse_pass_static(const void* v, int32_t dtype_bytes, int64_t K, int64_t n, int64_t ld,
                                 const double* f, const double* log_N, const int32_t* H, double* Q, void* logden,
                                 void* stream) {
  cudaGetLastError();  // drop stale errors of earlier, unrelated runtime calls
  if (dtype_bytes != 4 && dtype_bytes != 8) {
    set_error("mbar_lse_pass_static: dtype_bytes must be 4 or 8");
    return MBAR_EINVAL;
  }
  if (K < 1 || K > 1024 || n < 1) {
    set_error("mbar_lse_pass_static: bad sizes K=%lld n=%lld", (long long)K, (long long)n);
    return (K > 1024) ? MBAR_EUNSUPPORTED : MBAR_EINVAL;
  }
  const size_t need = mbar_lse_scratch_bytes(K, n, dtype_bytes);
  if (need == 0 || need > kStaticScratchBytes) {
    set_error("mbar_lse_pass_static: this K=%lld n=%lld pass needs %zu bytes of scratch; the built-in array holds "
              "%zu bytes (use mbar_lse_pass with a caller-provided buffer)",
              (long long)K, (long long)n, need, kStaticScratchBytes);
    return MBAR_EUNSUPPORTED;
  }
  void* scratch = nullptr;
  BUMBAR_TRY(static_scratch(&scratch));
  // counter and error word must start at zero (the array keeps the last
  // call's contents)
  BUMBAR_CUDA(cudaMemsetAsync(scratch, 0, 256, static_cast<cudaStream_t>(stream)));
  return mbar_lse_pass(v, dtype_bytes, K, n, ld, f, log_N, H, Q, logden, scratch, kStaticScratchBytes, stream);
}

}  // extern "C"
