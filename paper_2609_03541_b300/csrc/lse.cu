// Fused paired log-sum-exp pass (Eq. 1): for every column p of a K x n
// matrix v (samples or bins),
//     logden_p = log sum_j exp(a_j - v_jp),          a_j = f_j + log N_j,
//     Q_i      = sum_p H_p exp(a_i - v_ip - logden_p),
// in ONE read of v from HBM. Columns are streamed in strips of 128 bytes
// (32 FP32 or 16 FP64 columns) x all K rows; each strip is brought into
// shared memory by 2-D TMA boxes (128-byte swizzle) through a multi-stage
// mbarrier pipeline. Per strip:
//   A1  column maxima over k (8 or 16 lanes per column, shuffle merge);
//   A2  e_kp = exp(a_k - v_kp - max_p), written back in place, column sums;
//   B   each thread owns whole rows and accumulates sum_p e_kp * H_p / s_p
//       from 16-byte chunks of the swizzled tile (conflict-free).
// Row sums are kept per thread (FP32 for MIXED, flushed to FP64 every few
// strips; FP64 throughout for the FP64 path) and written once per CTA to
// scratch; the last CTA to finish reduces the per-CTA partials in a fixed
// order (deterministic) and, for an SCI step, applies the update, the
// gauge, the gradient and the relative step of Eq. 2.
#include <cmath>
#include <cstdio>

#include "common.cuh"
#include "kernels.cuh"

namespace bumbar {

namespace {

constexpr int kMaxRowsPerThread = 4;      // K <= 1024 with 256 threads
constexpr int kFlushStrips = 4;           // FP32 row sums flushed to FP64 every 4 strips
constexpr uint32_t kMaxSpins = 1u << 28;  // bounded mbarrier wait

template <typename T>
struct Lane;

template <>
struct Lane<float> {
  static constexpr int C = 32;  // columns per strip (128 bytes)
  static constexpr int R = 8;   // lanes (row groups) per column
};
template <>
struct Lane<double> {
  static constexpr int C = 16;
  static constexpr int R = 16;
};

__device__ __forceinline__ float lse_exp(float x) { return ex2_approx(x); }     // x in log2 units
__device__ __forceinline__ double lse_exp(double x) { return exp(x); }         // x in natural units
__device__ __forceinline__ float lse_scale() { return kLog2e; }
__device__ __forceinline__ float lse_log(float s) { return __log2f(s); }
__device__ __forceinline__ double lse_log(double s) { return log(s); }

__device__ __forceinline__ float tmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double tmax(double a, double b) { return fmax(a, b); }

template <typename T>
__device__ __forceinline__ T shfl_xor(T v, int m) {
  return __shfl_xor_sync(0xffffffffu, v, m);
}

}  // namespace

// Shared-memory carve-up of one CTA (dynamic smem, 1024-aligned base).
template <typename T>
struct LseSmem {
  static __host__ __device__ size_t stage_bytes(int nbox, int box_rows) {
    return static_cast<size_t>(nbox) * box_rows * 128;
  }
  static __host__ __device__ size_t extra_bytes(int K) {
    // a_k (Kpad of T), w_c (C of T), mbarriers (4), epilogue scratch (K doubles + 64)
    return round_up_dev(static_cast<size_t>(K) * sizeof(T), 16) + 128 * sizeof(T) + 64 +
           round_up_dev(static_cast<size_t>(K) * sizeof(double), 16) + 512;
  }
  static __host__ __device__ size_t round_up_dev(size_t x, size_t m) { return (x + m - 1) / m * m; }
};

template <typename T>
__global__ void __launch_bounds__(kThreads) lse_pass_kernel(const __grid_constant__ CUtensorMap tmap,
                                                            LseParams p) {
  constexpr int C = Lane<T>::C;
  constexpr int R = Lane<T>::R;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // align base to 1024 for the 128-byte swizzle atoms
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));

  const int K = p.K;
  const int tid = threadIdx.x;

  if (p.ctrl != nullptr && p.skip_if_done && p.ctrl->done) return;

  const size_t sbytes = LseSmem<T>::stage_bytes(p.nbox, p.box_rows);
  unsigned char* stage_base = smem;
  T* a_s = reinterpret_cast<T*>(smem + p.stages * sbytes);
  T* w_s = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(a_s) +
                                LseSmem<T>::round_up_dev(static_cast<size_t>(K) * sizeof(T), 16));
  uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(w_s) + 128 * sizeof(T));
  double* red_s = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(bars) + 64);

  const int num_strips = p.num_strips;
  const int my_first = blockIdx.x;
  const int stride = gridDim.x;
  const int my_count = (my_first < num_strips) ? (num_strips - 1 - my_first) / stride + 1 : 0;

  if (tid == 0) {
    prefetch_tmap(&tmap);
    for (int s = 0; s < p.stages; ++s) mbar_init(&bars[s], 1);
    fence_barrier_init();
  }
  // a_k = f_k + log N_k (FP32 path: in log2 units)
  for (int k = tid; k < K; k += kThreads) {
    double a = p.f[k] + p.logN[k];
    if constexpr (sizeof(T) == 4) {
      a_s[k] = static_cast<T>(a * 1.4426950408889634);
    } else {
      a_s[k] = static_cast<T>(a);
    }
  }
  __syncthreads();

  const uint32_t tx_bytes = static_cast<uint32_t>(sbytes);
  // prologue: fill the pipeline
  if (tid == 0) {
    for (int s = 0; s < p.stages && s < my_count; ++s) {
      const int strip = my_first + s * stride;
      unsigned char* dst = stage_base + s * sbytes;
      mbar_expect_tx(&bars[s], tx_bytes);
      for (int b = 0; b < p.nbox; ++b)
        tma_load_2d(dst + static_cast<size_t>(b) * p.box_rows * 128, &tmap, &bars[s], strip * C, b * p.box_rows);
    }
  }

  // Per-thread row ownership for phase B.
  double acc64[kMaxRowsPerThread];
  float acc32[kMaxRowsPerThread];
#pragma unroll
  for (int j = 0; j < kMaxRowsPerThread; ++j) {
    acc64[j] = 0.0;
    acc32[j] = 0.f;
  }

  const int col = tid / R;  // phase-A column within the strip
  const int rg = tid % R;   // phase-A row group
  int it_fail = -1;

  for (int it = 0; it < my_count; ++it) {
    const int s = it % p.stages;
    const uint32_t parity = static_cast<uint32_t>((it / p.stages) & 1);
    const int strip = my_first + it * stride;
    unsigned char* tile = stage_base + s * sbytes;
    const bool ok = mbar_wait_bounded(&bars[s], parity, kMaxSpins);
    if (__syncthreads_or(!ok)) {  // uniform decision across the CTA
      it_fail = it;
      break;
    }
    const int gcol = strip * C + col;
    const bool valid = gcol < p.n;

    // ---- A1: column maximum of x = a_k - v_kp ----
    T m = -INFINITY;
    for (int k = rg; k < K; k += R) {
      const uint32_t off = swz128(k, (col * sizeof(T)) / 16) + (col * sizeof(T)) % 16;
      const T v = *reinterpret_cast<const T*>(tile + off);
      T x;
      if constexpr (sizeof(T) == 4) {
        x = fmaf(-v, lse_scale(), a_s[k]);
      } else {
        x = a_s[k] - v;
      }
      m = tmax(m, x);
    }
#pragma unroll
    for (int o = R / 2; o >= 1; o >>= 1) m = tmax(m, shfl_xor(m, o));

    // ---- A2: e = exp(x - m) in place, column sum ----
    T ssum = T(0);
    for (int k = rg; k < K; k += R) {
      const uint32_t off = swz128(k, (col * sizeof(T)) / 16) + (col * sizeof(T)) % 16;
      T* ptr = reinterpret_cast<T*>(tile + off);
      T x;
      if constexpr (sizeof(T) == 4) {
        x = fmaf(-*ptr, lse_scale(), a_s[k]);
      } else {
        x = a_s[k] - *ptr;
      }
      const T e = lse_exp(x - m);
      *ptr = e;
      ssum += e;
    }
#pragma unroll
    for (int o = R / 2; o >= 1; o >>= 1) ssum += shfl_xor(ssum, o);
    if (rg == 0) {
      T w = T(0);
      if (valid) {
        const T h = p.H ? static_cast<T>(p.H[gcol]) : T(1);
        w = h / ssum;
        if (p.logden != nullptr) {
          T ld;
          if constexpr (sizeof(T) == 4) {
            ld = (m + lse_log(ssum)) * kLn2;
          } else {
            ld = m + lse_log(ssum);
          }
          static_cast<T*>(p.logden)[gcol] = ld;
        }
      }
      w_s[col] = w;
    }
    __syncthreads();

    // ---- B: row sums over the strip ----
#pragma unroll
    for (int j = 0; j < kMaxRowsPerThread; ++j) {
      const int k = tid + j * kThreads;
      if (k < K) {
        if constexpr (sizeof(T) == 4) {
          float part = 0.f;
#pragma unroll
          for (int ch = 0; ch < 8; ++ch) {
            const float4 e4 = *reinterpret_cast<const float4*>(tile + swz128(k, ch));
            const float4 w4 = *reinterpret_cast<const float4*>(w_s + ch * 4);
            part = fmaf(e4.x, w4.x, part);
            part = fmaf(e4.y, w4.y, part);
            part = fmaf(e4.z, w4.z, part);
            part = fmaf(e4.w, w4.w, part);
          }
          acc32[j] += part;
        } else {
          double part = 0.0;
#pragma unroll
          for (int ch = 0; ch < 8; ++ch) {
            const double2 e2 = *reinterpret_cast<const double2*>(tile + swz128(k, ch));
            const double2 w2 = *reinterpret_cast<const double2*>(w_s + ch * 2);
            part = fma(e2.x, w2.x, part);
            part = fma(e2.y, w2.y, part);
          }
          acc64[j] += part;
        }
      }
    }
    if constexpr (sizeof(T) == 4) {
      if ((it + 1) % kFlushStrips == 0) {
#pragma unroll
        for (int j = 0; j < kMaxRowsPerThread; ++j) {
          acc64[j] += static_cast<double>(acc32[j]);
          acc32[j] = 0.f;
        }
      }
    }
    // all reads/writes of this stage are done: hand it back to TMA
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0 && it + p.stages < my_count) {
      const int nstrip = my_first + (it + p.stages) * stride;
      mbar_expect_tx(&bars[s], tx_bytes);
      for (int b = 0; b < p.nbox; ++b)
        tma_load_2d(tile + static_cast<size_t>(b) * p.box_rows * 128, &tmap, &bars[s], nstrip * C, b * p.box_rows);
    }
  }

  if (it_fail >= 0) {
    // record the timeout, then wait (bounded) for the copies this CTA may
    // still have in flight before its shared memory goes away
    if (tid == 0) {
      atomicAdd(p.err, 1u);
      for (int j = it_fail; j < my_count && j < it_fail + p.stages; ++j)
        (void)mbar_wait_bounded(&bars[j % p.stages], static_cast<uint32_t>((j / p.stages) & 1), kMaxSpins);
    }
    __syncthreads();
  }

  // ---- per-CTA partials ----
  double* part = p.partials + static_cast<size_t>(blockIdx.x) * K;
#pragma unroll
  for (int j = 0; j < kMaxRowsPerThread; ++j) {
    const int k = tid + j * kThreads;
    if (k < K) {
      double v = acc64[j];
      if constexpr (sizeof(T) == 4) v += static_cast<double>(acc32[j]);
      part[k] = v;
    }
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

  // ---- last CTA: fixed-order reduction and the SCI epilogue ----
  double* fnew_s = red_s;  // K doubles
  for (int k = tid; k < K; k += kThreads) {
    double q = 0.0;
    for (int b = 0; b < static_cast<int>(gridDim.x); ++b) q += p.partials[static_cast<size_t>(b) * K + k];
    p.Q[k] = q;
    fnew_s[k] = p.f[k] + p.logN[k] - log(q);
  }
  __syncthreads();
  if (p.mode == kLseModeSci) {
    const double f0 = fnew_s[0];
    double smax = -1.0;  // -1 = no f_k != 0 seen
    bool finite = true;
    for (int k = tid; k < K; k += kThreads) {
      const double fo = fnew_s[k] - f0;
      const double fi = p.f[k];
      if (p.f_out) p.f_out[k] = fo;
      if (p.g_out) p.g_out[k] = p.Q[k] - p.Nk[k];
      if (!isfinite(fo)) finite = false;
      if (fi != 0.0) smax = fmax(smax, fabs(fo / fi - 1.0));
    }
    // block max
    __shared__ double red[kThreads / 32];
    __shared__ int fin[kThreads / 32];
    for (int o = 16; o >= 1; o >>= 1) {
      smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    }
    const int allfin = __all_sync(0xffffffffu, finite);
    if ((tid & 31) == 0) {
      red[tid >> 5] = smax;
      fin[tid >> 5] = allfin;
    }
    __syncthreads();
    if (tid == 0) {
      double sm = -1.0;
      int ok = 1;
      for (int w = 0; w < kThreads / 32; ++w) {
        sm = fmax(sm, red[w]);
        ok &= fin[w];
      }
      const double s = (sm < 0.0) ? INFINITY : sm;
      if (p.s_out) *p.s_out = s;
      if (p.ctrl) {
        p.ctrl->iters += 1;
        p.ctrl->last_s = s;
        if (!ok) p.ctrl->nonfinite = 1;
        if (p.eps > 0.0 && s < p.eps) p.ctrl->done = 1;
      }
    }
  }
  if (tid == 0) *p.counter = 0u;  // leave the scratch counter zeroed
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

LsePlan lse_plan(int64_t K, int64_t n, int dtype_bytes) {
  LsePlan pl{};
  const int C = 128 / dtype_bytes;
  pl.C = C;
  pl.num_strips = static_cast<int>(ceil_div(n, C));
  pl.box_rows = static_cast<int>(std::min<int64_t>(256, round_up(K, 8)));
  pl.nbox = static_cast<int>(ceil_div(K, pl.box_rows));
  const size_t sb = static_cast<size_t>(pl.nbox) * pl.box_rows * 128;
  pl.stages = sb <= 48 * 1024 ? 4 : (sb <= 64 * 1024 ? 3 : (sb <= 96 * 1024 ? 2 : 1));
  const size_t extra = (dtype_bytes == 4) ? LseSmem<float>::extra_bytes(static_cast<int>(K))
                                          : LseSmem<double>::extra_bytes(static_cast<int>(K));
  pl.smem = pl.stages * sb + extra + 1024;  // + alignment slack
  static int occ_cache[2][1025] = {};
  int* occ = &occ_cache[dtype_bytes == 4 ? 0 : 1][std::min<int64_t>(K, 1024)];
  if (*occ == 0) {
    int blocks = 1;
    if (dtype_bytes == 4) {
      cudaFuncSetAttribute(lse_pass_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, lse_pass_kernel<float>, kThreads, pl.smem);
    } else {
      cudaFuncSetAttribute(lse_pass_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, lse_pass_kernel<double>, kThreads, pl.smem);
    }
    *occ = std::max(1, blocks);
  }
  pl.grid = static_cast<int>(std::min<int64_t>(pl.num_strips, static_cast<int64_t>(*occ) * num_sms()));
  pl.grid = std::max(pl.grid, 1);
  return pl;
}

size_t lse_scratch_bytes(int64_t K, int64_t n, int dtype_bytes) {
  LsePlan pl = lse_plan(K, n, dtype_bytes);
  return static_cast<size_t>(pl.grid) * K * sizeof(double) + 256;
}

mbar_status lse_launch(const CUtensorMap& tmap, const LsePlan& pl, LseParams prm, int dtype_bytes,
                       cudaStream_t stream) {
  prm.num_strips = pl.num_strips;
  prm.box_rows = pl.box_rows;
  prm.nbox = pl.nbox;
  prm.stages = pl.stages;
  if (dtype_bytes == 4) {
    lse_pass_kernel<float><<<pl.grid, kThreads, pl.smem, stream>>>(tmap, prm);
    count_launches(1);
  } else {
    lse_pass_kernel<double><<<pl.grid, kThreads, pl.smem, stream>>>(tmap, prm);
    count_launches(1);
  }
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

}  // namespace bumbar
