// Reweighting to a target state (Eqs. 5-6) and the weighted 2-D histogram
// that the paper's free-energy surface (Fig. 1) is drawn from.
//
//   log p~_n = -u0_n - logden_n,   logden_n = log sum_m N_m exp(f_m - u_mn)
//   C        = sum_n p~_n,         p_n = p~_n / C
//
// logden comes from an LSE pass over the stored (possibly shifted, FP32)
// data: with v_mn = u_mn - c_n, logden(u)_n = logden(v)_n - c_n. The log of
// C is a log-sum-exp over the samples, reduced per block and then in block
// order (deterministic).
#include <cmath>

#include "common.cuh"
#include "kernels.cuh"

namespace bumbar {

namespace {

constexpr int kRwThreads = 256;

__device__ __forceinline__ void lse_combine(double& m, double& s, double m2, double s2) {
  if (m2 == -INFINITY) return;
  if (m == -INFINITY) {
    m = m2;
    s = s2;
    return;
  }
  if (m2 > m) {
    s = s * exp(m - m2) + s2;
    m = m2;
  } else {
    s += s2 * exp(m2 - m);
  }
}

// lp[i] = -u0[perm[i]] - (logden_i - c_i) in the stored column order, and a
// per-block (max, sum exp(lp - max)).
template <typename T>
__global__ void __launch_bounds__(kRwThreads) reweight_logp(const double* __restrict__ u0,
                                                            const int32_t* __restrict__ perm,
                                                            const T* __restrict__ logden,
                                                            const double* __restrict__ shift, int64_t N,
                                                            double* __restrict__ lp, double* __restrict__ part) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * kRwThreads + threadIdx.x;
  double m = -INFINITY, s = 0.0;
  if (i < N) {
    const double ld = static_cast<double>(logden[i]) - (shift ? shift[i] : 0.0);
    const double x = -u0[perm[i]] - ld;
    lp[i] = x;
    m = x;
    s = 1.0;
  }
  __shared__ double sm[kRwThreads], ss[kRwThreads];
  sm[threadIdx.x] = m;
  ss[threadIdx.x] = s;
  __syncthreads();
  for (int o = kRwThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      double a = sm[threadIdx.x], b = ss[threadIdx.x];
      lse_combine(a, b, sm[threadIdx.x + o], ss[threadIdx.x + o]);
      sm[threadIdx.x] = a;
      ss[threadIdx.x] = b;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sm[0];
    part[2 * blockIdx.x + 1] = ss[0];
  }
}

// log C from the block partials, combined in block order by one thread per
// stride and then a fixed tree.
__global__ void __launch_bounds__(kRwThreads) reweight_logc(const double* __restrict__ part, int64_t nblocks,
                                                            double* __restrict__ log_c) {
  double m = -INFINITY, s = 0.0;
  for (int64_t b = threadIdx.x; b < nblocks; b += kRwThreads) lse_combine(m, s, part[2 * b], part[2 * b + 1]);
  __shared__ double sm[kRwThreads], ss[kRwThreads];
  sm[threadIdx.x] = m;
  ss[threadIdx.x] = s;
  __syncthreads();
  for (int o = kRwThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      double a = sm[threadIdx.x], b = ss[threadIdx.x];
      lse_combine(a, b, sm[threadIdx.x + o], ss[threadIdx.x + o]);
      sm[threadIdx.x] = a;
      ss[threadIdx.x] = b;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *log_c = sm[0] + log(ss[0]);
}

// p in the caller's original sample order.
__global__ void reweight_p(const double* __restrict__ lp, const int32_t* __restrict__ perm, int64_t N,
                           const double* __restrict__ log_c, double* __restrict__ p) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * kRwThreads + threadIdx.x;
  if (i < N) p[perm[i]] = exp(lp[i] - *log_c);
}

// out[ix * ny + iy] += p_n for bin (ix, iy) = (floor((x-x0)/dx), floor((y-y0)/dy)),
// each subtraction and division rounded to nearest in binary64; samples
// outside [0, nx) x [0, ny) are dropped.
__global__ void hist2d_kernel(const double* __restrict__ x, const double* __restrict__ y,
                              const double* __restrict__ p, int64_t N, double x0, double dx, int64_t nx, double y0,
                              double dy, int64_t ny, double* __restrict__ out) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * kRwThreads + threadIdx.x;
  if (i >= N) return;
  const double qx = floor(__ddiv_rn(__dsub_rn(x[i], x0), dx));
  const double qy = floor(__ddiv_rn(__dsub_rn(y[i], y0), dy));
  if (!(qx >= 0.0 && qx < static_cast<double>(nx) && qy >= 0.0 && qy < static_cast<double>(ny))) return;
  atomicAdd(&out[static_cast<int64_t>(qx) * ny + static_cast<int64_t>(qy)], p[i]);
}

}  // namespace

size_t reweight_tmp_bytes(int64_t N) {
  return round_up(N * 8, 256) + round_up(ceil_div(N, kRwThreads) * 16, 256) + 256;
}

mbar_status reweight_weights(const double* u0, const int32_t* perm, const void* logden, int dtype_bytes,
                             const double* shift, int64_t N, double* p, double* log_c, void* tmp, size_t tmp_bytes,
                             cudaStream_t st) {
  if (tmp_bytes < reweight_tmp_bytes(N)) {
    set_error("reweight: scratch too small");
    return MBAR_EINVAL;
  }
  unsigned char* q = static_cast<unsigned char*>(tmp);
  double* lp = reinterpret_cast<double*>(q);
  q += round_up(N * 8, 256);
  double* part = reinterpret_cast<double*>(q);
  const int64_t nb = ceil_div(N, kRwThreads);
  if (dtype_bytes == 4)
    reweight_logp<float><<<static_cast<unsigned>(nb), kRwThreads, 0, st>>>(u0, perm, static_cast<const float*>(logden),
                                                                          shift, N, lp, part);
  else
    reweight_logp<double><<<static_cast<unsigned>(nb), kRwThreads, 0, st>>>(
        u0, perm, static_cast<const double*>(logden), shift, N, lp, part);
  reweight_logc<<<1, kRwThreads, 0, st>>>(part, nb, log_c);
  reweight_p<<<static_cast<unsigned>(nb), kRwThreads, 0, st>>>(lp, perm, N, log_c, p);
  count_launches(3);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

mbar_status weighted_hist2d(const double* x, const double* y, const double* p, int64_t N, double x0, double dx,
                            int64_t nx, double y0, double dy, int64_t ny, double* out, cudaStream_t st) {
  BUMBAR_CUDA(cudaMemsetAsync(out, 0, static_cast<size_t>(nx) * ny * sizeof(double), st));
  hist2d_kernel<<<static_cast<unsigned>(ceil_div(N, kRwThreads)), kRwThreads, 0, st>>>(x, y, p, N, x0, dx, nx, y0, dy,
                                                                                      ny, out);
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

}  // namespace bumbar
