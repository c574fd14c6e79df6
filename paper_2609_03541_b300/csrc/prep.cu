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
      int64_t k = rg;
      for (; k + 56 < K; k += 64) {
        double x[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = u[(k + 8 * j) * ldu + n];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[(k + 8 * j) * ldv + n] = static_cast<float>(x[j] - cm);
      }
      for (; k < K; k += 8) v[k * ldv + n] = static_cast<float>(u[k * ldu + n] - cm);
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
