// The arithmetic of one lane group on two samples of a sample-major FP32
// tile (the per-sample work of Eq. 1): for sample columns c0, c1 (Kp
// consecutive floats each) the lane's entries k = 4 (lig + LPS i) + t give
//     x_k = a_k log2(e) - v_k log2(e)     (FP32 pairs (ahi, alo), (kLog2e, kLog2eLo)),
// the group's maxima m0, m1 and sums s0, s1 of 2^(x - m) by shuffles within
// the group of LPS lanes, and x0, x1 overwritten with 2^(x - m).
#pragma once

#include "common.cuh"

namespace bumbar {

template <int LPS, int NK>
__device__ __forceinline__ void smaj_pair(const float* c0, const float* c1, int lig, int Kp, const float (&ahi)[4 * NK],
                                          const float (&alo)[4 * NK], float (&x0)[4 * NK], float (&x1)[4 * NK],
                                          float& m0, float& m1, float& s0, float& s1) {
  constexpr int E = 4 * NK;
  m0 = -INFINITY;
  m1 = -INFINITY;
#pragma unroll
  for (int i = 0; i < NK; ++i) {
    const int k4 = 4 * (lig + LPS * i);
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
    if (k4 < Kp) {
      a = *reinterpret_cast<const float4*>(c0 + k4);
      b = *reinterpret_cast<const float4*>(c1 + k4);
    }
    const float va[4] = {a.x, a.y, a.z, a.w}, vb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int e = 4 * i + t;
      x0[e] = fmaf(-va[t], kLog2e, ahi[e]) + fmaf(-va[t], kLog2eLo, alo[e]);
      x1[e] = fmaf(-vb[t], kLog2e, ahi[e]) + fmaf(-vb[t], kLog2eLo, alo[e]);
      m0 = fmaxf(m0, x0[e]);
      m1 = fmaxf(m1, x1[e]);
    }
  }
  if constexpr (LPS == 32) {
    m0 = warp_max_f32(m0);  // the whole warp holds each sample
    m1 = warp_max_f32(m1);
  } else {
#pragma unroll
    for (int o = LPS / 2; o >= 1; o >>= 1) {
      m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, o));
      m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
    }
  }
  s0 = 0.f;
  s1 = 0.f;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    x0[e] = ex2_approx(x0[e] - m0);
    x1[e] = ex2_approx(x1[e] - m1);
    s0 += x0[e];
    s1 += x1[e];
  }
#pragma unroll
  for (int o = LPS / 2; o >= 1; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
}

}  // namespace bumbar
