// Shared tail of the fused LSE pass kernels: each CTA writes its FP64
// partial row sums; the reduction over CTAs and the SCI epilogue (Eq. 1
// update, gauge f_0 = 0, gradient Q - N, relative step of Eq. 2, absolute
// step, and the device-side loop control of Algorithm 1) run in
// lse_epilogue_kernel (lse.cu), one warp per state, launched right after the
// pass on the same stream.
#pragma once

#include "common.cuh"
#include "kernels.cuh"

namespace bumbar {

// rowsum[j] is this thread's FP64 row sum of row tid + j*THREADS.
template <int THREADS, int ROWS_PT>
__device__ __forceinline__ void lse_write_partials(const LseParams& p, const double* rowsum) {
  double* part = p.partials + static_cast<size_t>(blockIdx.x) * p.K;
#pragma unroll
  for (int j = 0; j < ROWS_PT; ++j) {
    const int k = threadIdx.x + j * THREADS;
    if (k < p.K) part[k] = rowsum[j];
  }
}

}  // namespace bumbar
