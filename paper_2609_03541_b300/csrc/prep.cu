// Data preparation on the device: validation of u_kn, the per-sample shift
// of the mixed-precision store, and small vector updates.
//
// Mixed precision keeps v_kn = fl32(u_kn - c_n) with c_n = min_k u_kn: the
// free energies are unchanged by any per-sample shift (the shift cancels
// between numerator and denominator of Eq. 1), the stored magnitudes stay
// small for the entries that carry weight, and every v_kn >= 0.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace bumbar {

namespace {

// Persistent blocks, each handling strips of 32 columns: 8 row groups x 32
// columns, eight rows in flight per thread. Pass 1 takes the column minimum with integer comparisons on an
// order-preserving image of the binary64 bits (FP64 arithmetic is slow on
// this part); pass 2 re-reads the same 32 x K block -- few enough blocks are
// resident that it is still in L2 -- and writes fl32(u - min).
__device__ __forceinline__ unsigned long long ordered_bits(double x) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double from_ordered(unsigned long long k) {
  const unsigned long long b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
  return __longlong_as_double(static_cast<long long>(b));
}

// Binary64 -> binary32 with round-to-nearest-even using integer operations
// only (the FP64 pipe is the bottleneck of this kernel): keep the top 23 of
// the 52 fraction bits and round on the 29 dropped ones; a carry out of the
// fraction moves into the exponent (up to infinity), as IEEE rounding does.
// Results that would be subnormal or zero in binary32 take the hardware
// conversion (rare for shifted energies).
__device__ __forceinline__ float f64_to_f32_rn(double x) {
  const unsigned long long d = static_cast<unsigned long long>(__double_as_longlong(x));
  const unsigned int hi = static_cast<unsigned int>(d >> 32), lo = static_cast<unsigned int>(d);
  const int e = static_cast<int>((hi >> 20) & 0x7FFu) - 1023 + 127;
  if (e <= 0 || e >= 255) return __double2float_rn(x);  // zero, subnormal, overflow, inf/nan
  const unsigned int sign = hi & 0x80000000u;
  const unsigned int mant = ((hi & 0xFFFFFu) << 3) | (lo >> 29);  // top 23 fraction bits
  const unsigned int rest = lo & 0x1FFFFFFFu;                     // the 29 dropped bits
  const unsigned int half = 0x10000000u;
  const unsigned int up = (rest > half || (rest == half && (mant & 1u))) ? 1u : 0u;
  const unsigned int bits = ((static_cast<unsigned int>(e) << 23) | mant) + up;
  return __uint_as_float(sign | bits);
}

// Splits a binary64 x into hi = RN32(x) and lo ~ x - hi with integer
// operations only: the residual is (dropped 29 fraction bits - the rounding
// increment) x 2^(E - 1075), formed as an int -> float conversion and a
// power-of-two scale. False when hi or the scale would leave the normal
// binary32 range (the caller then uses FP64 arithmetic).
__device__ __forceinline__ bool split_f64(double x, float& hi, float& lo) {
  const unsigned long long d = static_cast<unsigned long long>(__double_as_longlong(x));
  const unsigned int dh = static_cast<unsigned int>(d >> 32), dl = static_cast<unsigned int>(d);
  const int E = static_cast<int>((dh >> 20) & 0x7FFu);
  const int e = E - 1023 + 127;
  const int s = E - 1075;  // weight of the last binary64 fraction bit
  if (e <= 0 || e >= 254 || s < -126) return false;
  const unsigned int sign = dh & 0x80000000u;
  const unsigned int mant = ((dh & 0xFFFFFu) << 3) | (dl >> 29);
  const unsigned int rest = dl & 0x1FFFFFFFu;
  const unsigned int half = 0x10000000u;
  const unsigned int up = (rest > half || (rest == half && (mant & 1u))) ? 1u : 0u;
  hi = __uint_as_float(sign | (((static_cast<unsigned int>(e) << 23) | mant) + up));
  const int r = static_cast<int>(rest) - (up ? (1 << 29) : 0);
  const float scale = __uint_as_float(static_cast<unsigned int>(s + 127) << 23);
  lo = __uint_as_float(sign ^ __float_as_uint(__int2float_rn(r) * scale));
  return true;
}

__global__ void __launch_bounds__(256) shift_fp32_kernel(const double* __restrict__ u, int64_t K, int64_t N,
                                                         int64_t ldu, double* __restrict__ c, float* __restrict__ v,
                                                         int64_t ldv, int* bad) {
  __shared__ unsigned long long part[8][32];
  __shared__ int okp[8][32];
  const int lane = threadIdx.x & 31, rg = threadIdx.x >> 5;
  const int64_t nstrips = (N + 31) / 32;
  for (int64_t strip = blockIdx.x; strip < nstrips; strip += gridDim.x) {
    const int64_t n = strip * 32 + lane;
    unsigned long long m = ~0ull;
    bool ok = true;
    if (n < N) {
      // eight independent loads in flight per thread
      int64_t k = rg;
      for (; k + 56 < K; k += 64) {
        double x[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = u[(k + 8 * j) * ldu + n];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const unsigned long long bx = static_cast<unsigned long long>(__double_as_longlong(x[j]));
          ok &= ((bx >> 52) & 0x7FF) != 0x7FF;
          const unsigned long long kx = ordered_bits(x[j]);
          m = kx < m ? kx : m;
        }
      }
      for (; k < K; k += 8) {
        const double x = u[k * ldu + n];
        const unsigned long long bx = static_cast<unsigned long long>(__double_as_longlong(x));
        ok &= ((bx >> 52) & 0x7FF) != 0x7FF;
        const unsigned long long kx = ordered_bits(x);
        m = kx < m ? kx : m;
      }
    }
    part[rg][lane] = m;
    okp[rg][lane] = ok ? 1 : 0;
    __syncthreads();
    unsigned long long mm = part[0][lane];
    int allok = okp[0][lane];
#pragma unroll
    for (int g = 1; g < 8; ++g) {
      mm = part[g][lane] < mm ? part[g][lane] : mm;
      allok &= okp[g][lane];
    }
    __syncthreads();
    if (n < N) {
      double cm = from_ordered(mm);
      if (!allok) {
        if (rg == 0) atomicOr(bad, 1);
        cm = 0.0;
      }
      if (rg == 0) c[n] = cm;
      // v = (uh - mh) + (ul - ml) in FP32 from the hi/lo splits of u and of
      // the column minimum (no FP64 arithmetic in the common case); FP64
      // subtraction for values outside the split's range
      float mh = 0.f, ml = 0.f;
      const bool msplit = split_f64(cm, mh, ml) || cm == 0.0;
      auto shifted = [&](double x) -> float {
        float xh, xl;
        if (msplit && split_f64(x, xh, xl)) return __fadd_rn(__fsub_rn(xh, mh), __fsub_rn(xl, ml));
        return f64_to_f32_rn(x - cm);
      };
      int64_t k = rg;
      for (; k + 56 < K; k += 64) {
        double x[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = u[(k + 8 * j) * ldu + n];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[(k + 8 * j) * ldv + n] = shifted(x[j]);
      }
      for (; k < K; k += 8) v[k * ldv + n] = shifted(u[k * ldu + n]);
    }
  }
}

__global__ void copy_checked_kernel(const double* __restrict__ u, int64_t K, int64_t N, int64_t ldu,
                                    double* __restrict__ v, int64_t ldv, int* bad) {
  const int64_t n = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t k = blockIdx.y;
  if (n >= N) return;
  const double x = u[k * ldu + n];
  if (!isfinite(x)) atomicOr(bad, 1);
  v[k * ldv + n] = x;
}

__global__ void finite_kernel(const double* __restrict__ x, int64_t n, int* bad) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n && !isfinite(x[i])) atomicOr(bad, 1);
}

__global__ void add_gauge_kernel(const double* __restrict__ f, const double* __restrict__ d, double* __restrict__ out,
                                 int64_t K) {
  __shared__ double base;
  if (threadIdx.x == 0) base = f[0] + d[0];
  __syncthreads();
  for (int64_t k = threadIdx.x; k < K; k += blockDim.x) out[k] = (f[k] + d[k]) - base;
}

}  // namespace

mbar_status shift_to_fp32(const double* u, int64_t K, int64_t N, int64_t ldu, double* c, float* v, int64_t ldv,
                          int* bad, cudaStream_t st) {
  const int64_t strips = ceil_div(N, 32);
  const unsigned grid = static_cast<unsigned>(std::min<int64_t>(strips, 4 * static_cast<int64_t>(num_sms())));
  shift_fp32_kernel<<<grid, 256, 0, st>>>(u, K, N, ldu, c, v, ldv, bad);
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

mbar_status copy_fp64_checked(const double* u, int64_t K, int64_t N, int64_t ldu, double* v, int64_t ldv, int* bad,
                              cudaStream_t st) {
  const dim3 g(static_cast<unsigned>(ceil_div(N, kThreads)), static_cast<unsigned>(K));
  copy_checked_kernel<<<g, kThreads, 0, st>>>(u, K, N, ldu, v, ldv, bad);
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

mbar_status check_finite(const double* x, int64_t n, int* bad, cudaStream_t st) {
  finite_kernel<<<static_cast<unsigned>(ceil_div(n, kThreads)), kThreads, 0, st>>>(x, n, bad);
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

mbar_status vec_add_gauge(const double* f, const double* d, double* out, int64_t K, cudaStream_t st) {
  add_gauge_kernel<<<1, kThreads, 0, st>>>(f, d, out, K);
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

}  // namespace bumbar
