// Shared tail of the fused LSE pass kernels: per-CTA partial row sums, the
// fixed-order reduction by the last CTA to finish, and the SCI epilogue
// (Eq. 1 update, gauge f_0 = 0, gradient Q - N, relative step of Eq. 2,
// absolute step, and the device-side loop control of Algorithm 1).
#pragma once

#include <cmath>

#include "common.cuh"
#include "kernels.cuh"

namespace bumbar {

// rowsum[j] is this thread's FP64 row sum of row tid + j*THREADS.
// red_s: K doubles of shared memory.
template <int THREADS, int ROWS_PT>
__device__ __forceinline__ void lse_finish(const LseParams& p, const double* rowsum, double* red_s) {
  const int K = p.K;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  double* part = p.partials + static_cast<size_t>(blockIdx.x) * K;
#pragma unroll
  for (int j = 0; j < ROWS_PT; ++j) {
    const int k = tid + j * THREADS;
    if (k < K) part[k] = rowsum[j];
  }
  __threadfence();
  __syncthreads();
  __shared__ unsigned int is_last;
  if (tid == 0) {
    const unsigned int ticket = atomicAdd(p.counter, 1u);
    is_last = (ticket == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();

  double* fnew_s = red_s;
  for (int k = tid; k < K; k += THREADS) {
    double qk = 0.0;
    for (int b = 0; b < static_cast<int>(gridDim.x); ++b) qk += p.partials[static_cast<size_t>(b) * K + k];
    p.Q[k] = qk;
    fnew_s[k] = p.f[k] + p.logN[k] - log(qk);
  }
  __syncthreads();
  if (p.mode == kLseModeSci) {
    const double f0 = fnew_s[0];
    const double fin0 = p.f[0];
    double smax = -1.0;  // -1 = no f_k != 0 seen
    double dmax = 0.0;
    bool finite = true;
    for (int k = tid; k < K; k += THREADS) {
      const double fo = fnew_s[k] - f0;
      const double fi = p.f[k];
      if (p.f_out) p.f_out[k] = fo;
      if (p.g_out) p.g_out[k] = p.Q[k] - p.Nk[k];
      if (!isfinite(fo)) finite = false;
      if (fi != 0.0) smax = fmax(smax, fabs(fo / fi - 1.0));
      dmax = fmax(dmax, fabs(fo - (fi - fin0)));
    }
    __shared__ double red[THREADS / 32];
    __shared__ double redd[THREADS / 32];
    __shared__ int fin[THREADS / 32];
    for (int o = 16; o >= 1; o >>= 1) {
      smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
      dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    }
    const int allfin = __all_sync(0xffffffffu, finite);
    if (lane == 0) {
      red[warp] = smax;
      redd[warp] = dmax;
      fin[warp] = allfin;
    }
    __syncthreads();
    if (tid == 0) {
      double sm = -1.0, dm = 0.0;
      int okf = 1;
      for (int w = 0; w < THREADS / 32; ++w) {
        sm = fmax(sm, red[w]);
        dm = fmax(dm, redd[w]);
        okf &= fin[w];
      }
      const double s = (sm < 0.0) ? INFINITY : sm;
      if (p.s_out) *p.s_out = s;
      if (p.d_out) *p.d_out = dm;
      if (p.ctrl) {
        p.ctrl->iters += 1;
        p.ctrl->last_s = s;
        if (!okf) p.ctrl->nonfinite = 1;
        if ((p.eps > 0.0 && s < p.eps) || (p.noise > 0.0 && dm < p.noise)) p.ctrl->done = 1;
      }
    }
  }
  if (tid == 0) *p.counter = 0u;  // leave the scratch counter zeroed
}

}  // namespace bumbar
