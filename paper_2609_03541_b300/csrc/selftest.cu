// Self-test of the failure path every bounded device-side wait shares: a
// kernel waits on an mbarrier that nothing arrives on, gives up after its
// time limit, records the timeout in an error word and returns, so the host
// gets MBAR_ETIMEOUT and the device stays usable. No fault, no trap, no
// unbounded loop.
#include "common.cuh"
#include "kernels.cuh"

namespace bumbar {
namespace {

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void wait_selftest_kernel(unsigned long long limit_ns, unsigned* err, unsigned long long* waited_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);  // expects one arrival, which never comes
    fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long t0 = now_ns();
    bool ok = false;
    while (now_ns() - t0 < limit_ns) {
      if (mbar_try_wait(&bar, 0)) {
        ok = true;
        break;
      }
    }
    *waited_ns = now_ns() - t0;
    if (!ok) atomicAdd(err, 1u);
  }
}

}  // namespace
}  // namespace bumbar

using namespace bumbar;

extern "C" {

mbar_status mbar_selftest_wait_timeout(int64_t limit_us, double* waited_s) {
  if (limit_us < 1 || limit_us > 2000000) {
    set_error("mbar_selftest_wait_timeout: limit must be 1 us .. 2 s");
    return MBAR_EINVAL;
  }
  cudaGetLastError();
  unsigned* err = nullptr;
  unsigned long long* waited = nullptr;
  BUMBAR_CUDA(cudaMalloc(&err, sizeof(unsigned) + sizeof(unsigned long long) + 8));
  waited = reinterpret_cast<unsigned long long*>(reinterpret_cast<unsigned char*>(err) + 8);
  mbar_status s = MBAR_OK;
  if (cudaMemset(err, 0, 16) != cudaSuccess) s = MBAR_ECUDA;
  if (s == MBAR_OK) {
    wait_selftest_kernel<<<1, 32>>>(static_cast<unsigned long long>(limit_us) * 1000ull, err, waited);
    count_launches(1);
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) s = cuda_status(e, "wait self-test");
  }
  unsigned h_err = 0;
  unsigned long long h_waited = 0;
  if (s == MBAR_OK && (cudaMemcpy(&h_err, err, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess ||
                       cudaMemcpy(&h_waited, waited, sizeof(h_waited), cudaMemcpyDeviceToHost) != cudaSuccess))
    s = MBAR_ECUDA;
  cudaFree(err);
  if (s != MBAR_OK) return s;
  if (waited_s) *waited_s = static_cast<double>(h_waited) * 1e-9;
  if (h_err) {
    set_error("a bounded device-side wait gave up after %.3f s (self-test)", static_cast<double>(h_waited) * 1e-9);
    return MBAR_ETIMEOUT;
  }
  return MBAR_OK;
}

}  // extern "C"
