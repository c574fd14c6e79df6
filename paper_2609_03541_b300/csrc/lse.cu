// Fused paired log-sum-exp pass (Eq. 1): for every column p of a K x n
// matrix v (samples or bins),
//     logden_p = log sum_j exp(a_j - v_jp),          a_j = f_j + log N_j,
//     Q_i      = sum_p H_p exp(a_i - v_ip - logden_p),
// in ONE read of v from HBM.
//
// Layout and schedule (persistent CTAs, one per SM or more):
//   * columns are streamed in strips of 128 bytes (32 FP32 or 16 FP64
//     columns) x all K rows; each strip is fetched into shared memory by 2-D
//     TMA boxes (<= 256 rows each, 128-byte swizzle) through a multi-stage
//     mbarrier pipeline, so HBM reads of later strips overlap the arithmetic;
//   * A1: column maxima of x = a_k - v_kp. A warp covers one 16-byte chunk
//     of the swizzled row (4 FP32 / 2 FP64 columns) and 8 / 16 row residues,
//     so its shared-memory reads are conflict-free; G warps split the rows
//     and merge through shared memory;
//   * A2: e_kp = exp(x - max_p) written back in place, column sums;
//   * B: each thread owns whole rows and accumulates sum_p e_kp H_p / s_p
//     from 16-byte chunks of the swizzled tile.
// Row sums are kept per thread (FP32 partial sums flushed to FP64 every few
// strips for MIXED; FP64 throughout for FP64) and written once per CTA to
// scratch; the last CTA to finish reduces the per-CTA partials in a fixed
// order (deterministic) and, for an SCI step, applies the update, the gauge,
// the gradient and the relative step of Eq. 2.
#include <cmath>
#include <cstdio>

#include "common.cuh"
#include "kernels.cuh"
#include "lse_common.cuh"

namespace bumbar {

namespace {

constexpr int kFlushStrips = 4;           // FP32 row sums flushed to FP64 every 4 strips
constexpr uint32_t kMaxSpins = 1u << 28;  // bounded mbarrier wait

template <typename T, int G>
struct Cfg {
  static constexpr int THREADS = 256 * G;
  static constexpr int C = 128 / static_cast<int>(sizeof(T));  // columns per strip
  static constexpr int CPW = C / 8;                             // columns per 16-byte chunk
  static constexpr int LW = 32 / CPW;                           // lanes per column inside a warp
  static constexpr int R = LW * G;                              // row groups per column
  static constexpr int ROWS_PT = (1024 + THREADS - 1) / THREADS;  // phase-B rows per thread
};

__device__ __forceinline__ float lse_exp(float x) { return ex2_approx(x); }  // x in log2 units
__device__ __forceinline__ double lse_exp(double x) { return exp(x); }      // x in natural units
__device__ __forceinline__ float lse_log(float s) { return __log2f(s); }
__device__ __forceinline__ double lse_log(double s) { return log(s); }
__device__ __forceinline__ float tmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double tmax(double a, double b) { return fmax(a, b); }

// x = a - v in the kernel's exponent units (log2 for FP32, natural for FP64)
__device__ __forceinline__ float expo(float a, float v) { return fmaf(-v, kLog2e, a); }
__device__ __forceinline__ double expo(double a, double v) { return a - v; }

template <typename T>
__device__ __forceinline__ T shfl_xor(T v, int m) {
  return __shfl_xor_sync(0xffffffffu, v, m);
}

__host__ __device__ inline size_t rup(size_t x, size_t m) { return (x + m - 1) / m * m; }

}  // namespace

// Shared-memory carve-up (dynamic, base aligned up to 1024 in the kernel):
//   stages x stage bytes | a_k [K] (FP32: hi [K], lo [K]) | w_c [32] | column partials [2][G][32] |
//   mbarriers [8]
template <typename T, int G>
struct LseSmem {
  static __host__ __device__ size_t stage_bytes(int nbox, int box_rows) {
    return static_cast<size_t>(nbox) * box_rows * 128;
  }
  // FP32: a_k log2(e) as an unevaluated pair, hi [K] then lo [K]
  static __host__ __device__ size_t a_bytes(int K) {
    return rup(static_cast<size_t>(K) * sizeof(T) * (sizeof(T) == 4 ? 2 : 1), 16);
  }
  static constexpr size_t kW = 32 * sizeof(T);
  static constexpr size_t kParts = 2 * G * 32 * sizeof(T);
  static constexpr size_t kBars = 64;
  static __host__ __device__ size_t extra_bytes(int K) {
    return a_bytes(K) + kW + kParts + kBars;
  }
};

template <typename T, int G>
__global__ void __launch_bounds__(Cfg<T, G>::THREADS, 1) lse_pass_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                     LseParams p) {
  using CF = Cfg<T, G>;
  constexpr int THREADS = CF::THREADS, C = CF::C, CPW = CF::CPW, LW = CF::LW, R = CF::R;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));

  const int K = p.K;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;

  if (lse_skip(p)) return;

  const size_t sbytes = LseSmem<T, G>::stage_bytes(p.nbox, p.box_rows);
  unsigned char* stage_base = smem;
  unsigned char* cur = smem + p.stages * sbytes;
  T* a_s = reinterpret_cast<T*>(cur);
  cur += LseSmem<T, G>::a_bytes(K);
  T* w_s = reinterpret_cast<T*>(cur);
  cur += LseSmem<T, G>::kW;
  T* colm = reinterpret_cast<T*>(cur);         // [G][32] partial maxima
  T* cols = colm + G * 32;                     // [G][32] partial sums
  cur += LseSmem<T, G>::kParts;
  uint64_t* bars = reinterpret_cast<uint64_t*>(cur);

  const int num_strips = p.num_strips;
  const int my_first = blockIdx.x;
  const int stride = gridDim.x;
  const int my_count = (my_first < num_strips) ? (num_strips - 1 - my_first) / stride + 1 : 0;

  if (tid == 0) {
    prefetch_tmap(&tmap);
    for (int s = 0; s < p.stages; ++s) mbar_init(&bars[s], 1);
    fence_barrier_init();
  }
  // FP32 keeps the rounding of a_k log2(e) beside it (lo), and of log2(e)
  // in kLog2eLo, so the state offsets are not quantised to the FP32 spacing
  // at |a_k| and v carries no systematic scale error: x_kp is rounded once
  // per entry, not once per row for every column alike
  T* a_lo = a_s + K;
  for (int k = tid; k < K; k += THREADS) {
    const double a = p.f[k] + p.logN[k];
    if constexpr (sizeof(T) == 4) {
      const double al = a * 1.4426950408889634;
      a_s[k] = static_cast<T>(al);
      a_lo[k] = isfinite(a_s[k]) ? static_cast<T>(al - static_cast<double>(a_s[k])) : T(0);
    } else {
      a_s[k] = static_cast<T>(a);
    }
  }
  auto xk = [&](int k, T v) -> T {
    if constexpr (sizeof(T) == 4) {
      return expo(a_s[k], v) + fmaf(-v, kLog2eLo, a_lo[k]);
    } else {
      return expo(a_s[k], v);
    }
  };
  __syncthreads();

  const uint32_t tx_bytes = static_cast<uint32_t>(sbytes);
  if (tid == 0) {
    for (int s = 0; s < p.stages && s < my_count; ++s) {
      const int strip = my_first + s * stride;
      unsigned char* dst = stage_base + s * sbytes;
      mbar_expect_tx(&bars[s], tx_bytes);
      for (int b = 0; b < p.nbox; ++b)
        tma_load_2d(dst + static_cast<size_t>(b) * p.box_rows * 128, &tmap, &bars[s], strip * C, b * p.box_rows);
    }
  }

  double acc64[CF::ROWS_PT];
  float acc32[CF::ROWS_PT];
#pragma unroll
  for (int j = 0; j < CF::ROWS_PT; ++j) {
    acc64[j] = 0.0;
    acc32[j] = 0.f;
  }

  // phase-A geometry of this thread
  const int q = warp & 7;                    // 16-byte chunk (column group) of the strip
  const int h = warp >> 3;                   // row half (0..G-1)
  const int col = q * CPW + lane / LW;       // column within the strip
  const int r0 = h * LW + (lane % LW);       // first row; rows r0, r0 + R, ...
  // byte offset of (row r0, col) inside the swizzled tile; rows r0 + R*j keep
  // the same swizzle phase (R is a multiple of 8), so the stride is R*128 bytes
  const uint32_t off0 = static_cast<uint32_t>(r0) * 128u + ((static_cast<uint32_t>(q) ^ (r0 & 7u)) << 4) +
                        static_cast<uint32_t>((col % CPW) * sizeof(T));
  constexpr uint32_t kRowStep = R * 128u;
  int it_fail = -1;

  for (int it = 0; it < my_count; ++it) {
    const int s = it % p.stages;
    const uint32_t parity = static_cast<uint32_t>((it / p.stages) & 1);
    const int strip = my_first + it * stride;
    unsigned char* tile = stage_base + s * sbytes;
    const bool ok = mbar_wait_bounded(&bars[s], parity, kMaxSpins);
    if (__syncthreads_or(!ok)) {
      it_fail = it;
      break;
    }
    const int gcol = strip * C + col;
    const bool valid = gcol < p.n;

    // ---- A1: column maximum of x = a_k - v_kp ----
    T m0 = -INFINITY, m1 = -INFINITY;
    {
      int k = r0;
      uint32_t off = off0;
      for (; k + R < K; k += 2 * R, off += 2 * kRowStep) {
        const T v0 = *reinterpret_cast<const T*>(tile + off);
        const T v1 = *reinterpret_cast<const T*>(tile + off + kRowStep);
        m0 = tmax(m0, xk(k, v0));
        m1 = tmax(m1, xk(k + R, v1));
      }
      if (k < K) m0 = tmax(m0, xk(k, *reinterpret_cast<const T*>(tile + off)));
    }
    T m = tmax(m0, m1);
#pragma unroll
    for (int o = LW / 2; o >= 1; o >>= 1) m = tmax(m, shfl_xor(m, o));
    if constexpr (G > 1) {
      if ((lane % LW) == 0) colm[h * 32 + col] = m;
      __syncthreads();
#pragma unroll
      for (int g = 0; g < G; ++g) m = tmax(m, colm[g * 32 + col]);
    }

    // ---- A2: e = exp(x - m) in place, column sum ----
    T s0 = T(0), s1 = T(0);
    {
      int k = r0;
      uint32_t off = off0;
      for (; k + R < K; k += 2 * R, off += 2 * kRowStep) {
        T* p0 = reinterpret_cast<T*>(tile + off);
        T* p1 = reinterpret_cast<T*>(tile + off + kRowStep);
        const T e0 = lse_exp(xk(k, *p0) - m);
        const T e1 = lse_exp(xk(k + R, *p1) - m);
        *p0 = e0;
        *p1 = e1;
        s0 += e0;
        s1 += e1;
      }
      if (k < K) {
        T* p0 = reinterpret_cast<T*>(tile + off);
        const T e0 = lse_exp(xk(k, *p0) - m);
        *p0 = e0;
        s0 += e0;
      }
    }
    T ssum = s0 + s1;
#pragma unroll
    for (int o = LW / 2; o >= 1; o >>= 1) ssum += shfl_xor(ssum, o);
    if constexpr (G > 1) {
      if ((lane % LW) == 0) cols[h * 32 + col] = ssum;
      __syncthreads();
    }
    if (h == 0 && (lane % LW) == 0) {
      if constexpr (G > 1) {
        ssum = T(0);
#pragma unroll
        for (int g = 0; g < G; ++g) ssum += cols[g * 32 + col];
      }
      T w = T(0);
      if (valid) {
        const T hc = p.H ? static_cast<T>(p.H[gcol]) : T(1);
        w = hc / ssum;
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
    for (int j = 0; j < CF::ROWS_PT; ++j) {
      const int k = tid + j * THREADS;
      if (k < K) {
        if constexpr (sizeof(T) == 4) {
          float pa = 0.f, pb = 0.f;
#pragma unroll
          for (int ch = 0; ch < 8; ch += 2) {
            const float4 ea = *reinterpret_cast<const float4*>(tile + swz128(k, ch));
            const float4 wa = *reinterpret_cast<const float4*>(w_s + ch * 4);
            const float4 eb = *reinterpret_cast<const float4*>(tile + swz128(k, ch + 1));
            const float4 wb = *reinterpret_cast<const float4*>(w_s + ch * 4 + 4);
            pa = fmaf(ea.x, wa.x, pa);
            pb = fmaf(eb.x, wb.x, pb);
            pa = fmaf(ea.y, wa.y, pa);
            pb = fmaf(eb.y, wb.y, pb);
            pa = fmaf(ea.z, wa.z, pa);
            pb = fmaf(eb.z, wb.z, pb);
            pa = fmaf(ea.w, wa.w, pa);
            pb = fmaf(eb.w, wb.w, pb);
          }
          acc32[j] += pa + pb;
        } else {
          double pa = 0.0, pb = 0.0;
#pragma unroll
          for (int ch = 0; ch < 8; ch += 2) {
            const double2 ea = *reinterpret_cast<const double2*>(tile + swz128(k, ch));
            const double2 wa = *reinterpret_cast<const double2*>(w_s + ch * 2);
            const double2 eb = *reinterpret_cast<const double2*>(tile + swz128(k, ch + 1));
            const double2 wb = *reinterpret_cast<const double2*>(w_s + ch * 2 + 2);
            pa = fma(ea.x, wa.x, pa);
            pb = fma(eb.x, wb.x, pb);
            pa = fma(ea.y, wa.y, pa);
            pb = fma(eb.y, wb.y, pb);
          }
          acc64[j] += pa + pb;
        }
      }
    }
    if constexpr (sizeof(T) == 4) {
      if ((it + 1) % kFlushStrips == 0) {
#pragma unroll
        for (int j = 0; j < CF::ROWS_PT; ++j) {
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

  // ---- per-CTA partials, then the last CTA's reduction and SCI epilogue ----
  double rowsum[CF::ROWS_PT];
#pragma unroll
  for (int j = 0; j < CF::ROWS_PT; ++j) {
    rowsum[j] = acc64[j];
    if constexpr (sizeof(T) == 4) rowsum[j] += static_cast<double>(acc32[j]);
  }
  lse_write_partials<THREADS, CF::ROWS_PT>(p, rowsum);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

namespace {

// CTA width per element type: FP32 runs 512 threads (G = 2), FP64 256 (G = 1).
constexpr int kGf32 = 2;
constexpr int kGf64 = 1;

template <typename T, int G>
int lse_occupancy(size_t smem) {
  std::lock_guard<std::recursive_mutex> lock(init_mutex());
  static size_t max_dyn = 0;
  if (max_dyn == 0) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, lse_pass_kernel<T, G>);
    max_dyn = static_cast<size_t>(optin) - fa.sharedSizeBytes;
    cudaFuncSetAttribute(lse_pass_kernel<T, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(max_dyn));
  }
  if (smem > max_dyn) return 0;
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, lse_pass_kernel<T, G>, Cfg<T, G>::THREADS, smem) !=
      cudaSuccess)
    blocks = 0;
  return blocks;
}

}  // namespace

LsePlan lse_plan(int64_t K, int64_t n, int dtype_bytes) {
  if (lse_regs_supported(K, dtype_bytes)) return lse_regs_plan(K, n);
  LsePlan pl{};
  const int C = 128 / dtype_bytes;
  pl.C = C;
  pl.threads = dtype_bytes == 4 ? Cfg<float, kGf32>::THREADS : Cfg<double, kGf64>::THREADS;
  pl.num_strips = static_cast<int>(ceil_div(n, C));
  pl.box_rows = static_cast<int>(std::min<int64_t>(256, round_up(K, 8)));
  pl.nbox = static_cast<int>(ceil_div(K, pl.box_rows));
  const size_t sb = static_cast<size_t>(pl.nbox) * pl.box_rows * 128;
  pl.stages = sb <= 48 * 1024 ? 4 : (sb <= 64 * 1024 ? 3 : (sb <= 96 * 1024 ? 2 : 1));
  const size_t extra = (dtype_bytes == 4) ? LseSmem<float, kGf32>::extra_bytes(static_cast<int>(K))
                                          : LseSmem<double, kGf64>::extra_bytes(static_cast<int>(K));
  pl.smem = pl.stages * sb + extra + 1024;  // + alignment slack
  static int occ_cache[2][1025] = {};
  int occ = 0;
  {
    std::lock_guard<std::recursive_mutex> lock(init_mutex());
    int* slot = &occ_cache[dtype_bytes == 4 ? 0 : 1][std::min<int64_t>(K, 1024)];
    if (*slot == 0) {
      *slot = (dtype_bytes == 4) ? lse_occupancy<float, kGf32>(pl.smem) : lse_occupancy<double, kGf64>(pl.smem);
      cudaGetLastError();  // the probes above report through their return values
    }
    occ = *slot;
  }
  pl.grid = static_cast<int>(std::min<int64_t>(pl.num_strips, static_cast<int64_t>(std::max(occ, 1)) * num_sms()));
  pl.grid = std::max(pl.grid, 1);
  pl.ok = occ > 0;
  return pl;
}

namespace {

constexpr int kEpiWarps = 4;  // states per epilogue CTA (one warp each)

// Reduction over the CTAs of the pass and the SCI epilogue, one warp per
// state k: the lanes add the partials of CTAs lane, lane + 32, ... in order,
// a shuffle tree combines them (a fixed order); lane 0 finishes the state.
// Each CTA also evaluates state 0's update for the gauge. The new f goes to
// a scratch vector first (f_out may be f itself, which other CTAs are still
// reading). Per-CTA maxima of the step sizes go to scratch slots, and the
// last CTA to finish combines them with all its threads (shuffle trees, no
// long dependent FP64 chains), updates the loop control and copies the new
// f out.
__global__ void __launch_bounds__(32 * kEpiWarps) lse_epilogue_kernel(LseParams p) {
  if (lse_skip(p)) return;  // same guard as the pass
  const int K = p.K;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int k = blockIdx.x * kEpiWarps + warp;
  const bool sci = p.mode == kLseModeSci;
  // the lane's partials b = lane, lane + 32, ... added in that order; eight
  // loads are issued before their adds (past the end: exact zeros)
  auto rowsum = [&](int row) {
    double q = 0.0;
    for (int b0 = lane; b0 < p.nparts; b0 += 32 * 8) {
      double x[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int b = b0 + 32 * j;
        x[j] = b < p.nparts ? p.partials[static_cast<size_t>(b) * K + row] : 0.0;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) q += x[j];
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    return q;
  };
  __shared__ double f0new_s;
  __shared__ double smax_s[kEpiWarps], dmax_s[kEpiWarps];
  __shared__ int fin_s[kEpiWarps], unf_s[kEpiWarps];
  if (sci && warp == 0) {
    const double q0 = rowsum(0);
    if (lane == 0) f0new_s = p.f[0] + p.logN[0] - log(q0);
  }
  double qk = 0.0, fnew = 0.0;
  if (k < K) {
    qk = rowsum(k);
    if (lane == 0) {
      p.Q[k] = qk;
      if (sci) fnew = p.f[k] + p.logN[k] - log(qk);
    }
  }
  if (!sci) return;
  __syncthreads();
  double smax = -1.0, dmax = 0.0;  // smax -1: no f_k != 0 seen
  int finite = 1, under = 0;
  if (k < K && lane == 0) {
    // a state whose expected count fell below 1e-20 N_k lost (part of) its
    // sum to the linear-domain exponentials: the step is redone exactly
    under = (qk >= 1e-20 * p.Nk[k]) ? 0 : 1;
    const double fo = fnew - f0new_s;
    const double fi = p.f[k];
    p.epi[k] = fo;
    if (p.g_out) p.g_out[k] = qk - p.Nk[k];
    if (!isfinite(fo)) finite = 0;
    if (fi != 0.0) smax = fabs(fo / fi - 1.0);
    dmax = fabs(fo - (fi - p.f[0]));
  }
  if (lane == 0) {
    smax_s[warp] = smax;
    dmax_s[warp] = dmax;
    fin_s[warp] = finite;
    unf_s[warp] = under;
  }
  __syncthreads();
  __shared__ unsigned int is_last;
  if (threadIdx.x == 0) {
    double sm = -1.0, dm = 0.0;
    int ok = 1, un = 0;
#pragma unroll
    for (int w = 0; w < kEpiWarps; ++w) {
      sm = fmax(sm, smax_s[w]);
      dm = fmax(dm, dmax_s[w]);
      ok &= fin_s[w];
      un |= unf_s[w];
    }
    double* slot = p.epi + K + 3 * static_cast<size_t>(blockIdx.x);
    slot[0] = sm;
    slot[1] = dm;
    slot[2] = (ok ? 1.0 : 0.0) + (un ? 2.0 : 0.0);
    __threadfence();
    const unsigned int ticket = atomicAdd(p.counter, 1u);
    is_last = (ticket == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double sm = -1.0, dm = 0.0;
  int okm = 1, unm = 0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
    const double* slot = p.epi + K + 3 * static_cast<size_t>(b);
    sm = fmax(sm, slot[0]);
    dm = fmax(dm, slot[1]);
    okm &= (static_cast<int>(slot[2]) & 1);
    unm |= (static_cast<int>(slot[2]) >> 1) & 1;
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    sm = fmax(sm, __shfl_xor_sync(0xffffffffu, sm, o));
    dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
    okm &= __shfl_xor_sync(0xffffffffu, okm, o);
    unm |= __shfl_xor_sync(0xffffffffu, unm, o);
  }
  if (lane == 0) {
    smax_s[warp] = sm;
    dmax_s[warp] = dm;
    fin_s[warp] = okm;
    unf_s[warp] = unm;
  }
  __syncthreads();
  int unf = 0;
#pragma unroll
  for (int w = 0; w < kEpiWarps; ++w) unf |= unf_s[w];
  if (unf && p.ctrl) {  // keep f; the host redoes this step in the log domain
    if (threadIdx.x == 0) {
      p.ctrl->underflow = 1;
      if (p.s_out) *p.s_out = INFINITY;
      *p.counter = 0u;
    }
    return;
  }
  if (p.f_out)
    for (int j = threadIdx.x; j < K; j += blockDim.x) p.f_out[j] = p.epi[j];
  if (threadIdx.x != 0) return;
  double smf = -1.0, dmf = 0.0;
  int okf = 1;
#pragma unroll
  for (int w = 0; w < kEpiWarps; ++w) {
    smf = fmax(smf, smax_s[w]);
    dmf = fmax(dmf, dmax_s[w]);
    okf &= fin_s[w];
  }
  const double sv = (smf < 0.0) ? INFINITY : smf;
  const double dv = dmf;
  if (p.s_out) *p.s_out = sv;
  if (p.d_out) *p.d_out = dv;
  if (p.ctrl) {
    p.ctrl->iters += 1;
    p.ctrl->last_s = sv;
    if (!okf) p.ctrl->nonfinite = 1;
    if ((p.eps > 0.0 && sv < p.eps) || (p.noise > 0.0 && dv < p.noise)) p.ctrl->done = 1;
  }
  *p.counter = 0u;  // leave the scratch counter zeroed
}

}  // namespace

// ---------------------------------------------------------------------------
// exact log-domain SCI step (steps whose linear-domain row sums underflowed)
// ---------------------------------------------------------------------------
namespace {

constexpr int kLogThreads = 256;
constexpr int64_t kLogCols = 8192;  // columns per block

template <typename A>
__device__ __forceinline__ void lse_acc(A& m, A& s, A m2, A s2) {
  if (m2 == -INFINITY) return;
  if (m == -INFINITY) {
    m = m2;
    s = s2;
  } else if (m2 > m) {
    s = s * exp(m - m2) + s2;
    m = m2;
  } else {
    s += s2 * exp(m2 - m);
  }
}

// (max, sum) of t_kp = a_k - v_kp - logden_p + log H_p over one chunk of
// columns of row k = blockIdx.y, in the data's precision.
template <typename T>
__global__ void __launch_bounds__(kLogThreads) row_logsum_partial(const T* __restrict__ v, int64_t ld, int64_t n,
                                                                  const double* __restrict__ f,
                                                                  const double* __restrict__ logN,
                                                                  const T* __restrict__ logden,
                                                                  const int32_t* __restrict__ H,
                                                                  double* __restrict__ part, int64_t nchunks) {
  const int64_t k = blockIdx.y;
  const double ad = f[k] + logN[k];
  const T a = static_cast<T>(ad);
  const T a_lo = isfinite(a) ? static_cast<T>(ad - static_cast<double>(a)) : T(0);  // 0 for FP64
  const int64_t c0 = static_cast<int64_t>(blockIdx.x) * kLogCols;
  const int64_t c1 = (c0 + kLogCols < n) ? c0 + kLogCols : n;
  T m = -INFINITY, s = T(0);
  for (int64_t c = c0 + threadIdx.x; c < c1; c += kLogThreads) {
    T t = (a - v[k * ld + c] - logden[c]) + a_lo;
    if (H) t += log(static_cast<T>(H[c]));
    lse_acc(m, s, t, T(1));
  }
  __shared__ double sm[kLogThreads], ss[kLogThreads];
  sm[threadIdx.x] = static_cast<double>(m);
  ss[threadIdx.x] = static_cast<double>(s);
  __syncthreads();
  for (int o = kLogThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      double x = sm[threadIdx.x], y = ss[threadIdx.x];
      lse_acc(x, y, sm[threadIdx.x + o], ss[threadIdx.x + o]);
      sm[threadIdx.x] = x;
      ss[threadIdx.x] = y;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * (k * nchunks + blockIdx.x)] = sm[0];
    part[2 * (k * nchunks + blockIdx.x) + 1] = ss[0];
  }
}

// logQ_k from the chunk partials (in chunk order), then Eq. 1, gauge, the
// gradient, Eq. 2 and the loop control, as lse_epilogue_kernel does. One
// block, K <= 1024 threads.
__global__ void __launch_bounds__(1024) log_sci_finish_kernel(LseParams p, const double* __restrict__ part,
                                                              int64_t nchunks) {
  const int K = p.K, k = threadIdx.x;
  __shared__ double fnew_s[1024];
  __shared__ double red_s[32], red_d[32];
  __shared__ int red_f[32];
  __shared__ double f00;
  double fi = 0.0, fn = 0.0;
  if (k < K) {
    double m = -INFINITY, s = 0.0;
    for (int64_t b = 0; b < nchunks; ++b) lse_acc(m, s, part[2 * (k * nchunks + b)], part[2 * (k * nchunks + b) + 1]);
    const double logq = m + log(s);
    fi = p.f[k];
    fn = fi + p.logN[k] - logq;
    fnew_s[k] = fn;
    p.Q[k] = exp(logq);
    if (p.g_out) p.g_out[k] = exp(logq) - p.Nk[k];
  }
  if (k == 0) f00 = p.f[0];
  __syncthreads();
  double smax = -1.0, dmax = 0.0;
  int finite = 1;
  if (k < K) {
    const double fo = fn - fnew_s[0];
    if (!isfinite(fo)) finite = 0;
    if (fi != 0.0) smax = fabs(fo / fi - 1.0);
    dmax = fabs(fo - (fi - f00));
    fnew_s[k] = fo;
  }
  for (int o = 16; o >= 1; o >>= 1) {
    smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    finite &= __shfl_xor_sync(0xffffffffu, finite, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red_s[threadIdx.x >> 5] = smax;
    red_d[threadIdx.x >> 5] = dmax;
    red_f[threadIdx.x >> 5] = finite;
  }
  __syncthreads();  // every read of f is done: f_out may be f
  if (k < K && p.f_out) p.f_out[k] = fnew_s[k];
  if (threadIdx.x == 0) {
    double sm = -1.0, dm = 0.0;
    int ok = 1;
    for (int w = 0; w < static_cast<int>((blockDim.x + 31) / 32); ++w) {
      sm = fmax(sm, red_s[w]);
      dm = fmax(dm, red_d[w]);
      ok &= red_f[w];
    }
    const double sv = (sm < 0.0) ? INFINITY : sm;
    if (p.s_out) *p.s_out = sv;
    if (p.d_out) *p.d_out = dm;
    if (p.ctrl) {
      p.ctrl->iters += 1;
      p.ctrl->last_s = sv;
      if (!ok) p.ctrl->nonfinite = 1;
      if ((p.eps > 0.0 && sv < p.eps) || (p.noise > 0.0 && dm < p.noise)) p.ctrl->done = 1;
    }
  }
}

}  // namespace

size_t log_sci_tmp_bytes(int64_t K, int64_t n) { return round_up(K * ceil_div(n, kLogCols) * 16, 256) + 256; }

mbar_status log_sci_finish(const void* v, int dtype_bytes, int64_t K, int64_t n, int64_t ld, const LseParams& p,
                           void* tmp, size_t tmp_bytes, cudaStream_t st) {
  if (K > 1024 || tmp_bytes < log_sci_tmp_bytes(K, n)) {
    set_error("log_sci_finish: bad sizes");
    return MBAR_EINVAL;
  }
  const int64_t nchunks = ceil_div(n, kLogCols);
  double* part = static_cast<double*>(tmp);
  const dim3 g(static_cast<unsigned>(nchunks), static_cast<unsigned>(K));
  if (dtype_bytes == 4)
    row_logsum_partial<float><<<g, kLogThreads, 0, st>>>(static_cast<const float*>(v), ld, n, p.f, p.logN,
                                                         static_cast<const float*>(p.logden), p.H, part, nchunks);
  else
    row_logsum_partial<double><<<g, kLogThreads, 0, st>>>(static_cast<const double*>(v), ld, n, p.f, p.logN,
                                                          static_cast<const double*>(p.logden), p.H, part, nchunks);
  log_sci_finish_kernel<<<1, static_cast<unsigned>(round_up(K, 32)), 0, st>>>(p, part, nchunks);
  count_launches(2);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

size_t lse_scratch_for_grid(int64_t K, int grid) {
  return 256 + static_cast<size_t>(grid) * K * sizeof(double) + sizeof(double) * K +
         3 * sizeof(double) * ceil_div(K, kEpiWarps);
}

size_t lse_scratch_bytes(int64_t K, int64_t n, int dtype_bytes) {
  LsePlan pl = lse_plan(K, n, dtype_bytes);
  return lse_scratch_for_grid(K, pl.grid);
}

mbar_status lse_epilogue_launch(const LseParams& prm, cudaStream_t stream) {
  // same shared-memory carveout as the pass kernels it alternates with, so the
  // SMs need not repartition L1 / shared memory between the two launches
  static bool carveout = false;
  {
    std::lock_guard<std::recursive_mutex> lock(init_mutex());
    if (!carveout) {
      cudaFuncSetAttribute(lse_epilogue_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                           static_cast<int>(cudaSharedmemCarveoutMaxShared));
      cudaGetLastError();
      carveout = true;
    }
  }
  lse_epilogue_kernel<<<static_cast<unsigned>(ceil_div(prm.K, kEpiWarps)), 32 * kEpiWarps, 0, stream>>>(prm);
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

mbar_status lse_launch(const CUtensorMap& tmap, const LsePlan& pl, LseParams prm, int dtype_bytes,
                       cudaStream_t stream) {
  if (!pl.ok) {
    set_error("lse pass: %zu bytes of shared memory per CTA exceed the device limit", pl.smem);
    return MBAR_EUNSUPPORTED;
  }
  prm.num_strips = pl.num_strips;
  prm.box_rows = pl.box_rows;
  prm.nbox = pl.nbox;
  prm.stages = pl.stages;
  prm.nparts = pl.grid;
  prm.epi = prm.partials + static_cast<size_t>(pl.grid) * prm.K;
  if (pl.variant == 1) {
    BUMBAR_TRY(lse_regs_launch(tmap, pl, prm, stream));
    return lse_epilogue_launch(prm, stream);
  }
  if (dtype_bytes == 4) {
    lse_pass_kernel<float, kGf32><<<pl.grid, pl.threads, pl.smem, stream>>>(tmap, prm);
  } else {
    lse_pass_kernel<double, kGf64><<<pl.grid, pl.threads, pl.smem, stream>>>(tmap, prm);
  }
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return lse_epilogue_launch(prm, stream);
}

}  // namespace bumbar
