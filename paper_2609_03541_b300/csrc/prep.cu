// Data preparation on the device: validation of u_kn, the per-sample shift
// of the mixed-precision store, and small vector updates.
//
// Mixed precision keeps v_kn = fl32(u_kn - c_n) with c_n = min_k u_kn: the
// free energies are unchanged by any per-sample shift (the shift cancels
// between numerator and denominator of Eq. 1), the stored magnitudes stay
// small for the entries that carry weight, and every v_kn >= 0.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace bumbar {

namespace {

// Column minima are taken with integer comparisons on an order-preserving
// image of the binary64 bits (FP64 arithmetic is slow on this part).
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

// x = hi + lo for the per-sample shift: hi = x truncated toward zero to 24
// significant bits (the sign, the exponent and the top 23 fraction bits of
// x, moved by integer operations) and lo = the 29 dropped fraction bits as
// an FP32 value (one integer-to-float rounding: |lo - exact| <= 2^-48 |x|).
// About half the integer work of the round-to-nearest split_f64 (no
// rounding increment, no carry into the exponent). False when hi or the
// scale of lo would leave the normal binary32 range (|x| outside
// [2^-74, 2^128)); the caller then uses FP64 arithmetic.
__device__ __forceinline__ bool split_f64_trunc(double x, float& hi, float& lo) {
  const unsigned long long d = static_cast<unsigned long long>(__double_as_longlong(x));
  const unsigned int dh = static_cast<unsigned int>(d >> 32), dl = static_cast<unsigned int>(d);
  const unsigned int E = (dh >> 20) & 0x7FFu;
  if (E - 949u > 1150u - 949u) return false;
  const unsigned int sign = dh & 0x80000000u;
  hi = __uint_as_float(sign | (((dh & 0x7FFFFFFFu) - 0x38000000u) << 3) | (dl >> 29));
  const float scale = __uint_as_float((E - 948u) << 23);  // 2^(E - 1075)
  lo = __uint_as_float(sign ^ __float_as_uint(__uint2float_rn(dl & 0x1FFFFFFFu) * scale));
  return true;
}

// Staging at creation, sample-major: block b takes the kStageCols samples
// n0 = b * kStageCols .. n0 + kStageCols - 1 with all K rows into shared
// memory (one read of u, 128-byte row pieces), takes each column's minimum
// there (MIXED) and writes the samples out as contiguous K-vectors,
// vst[n * stage_pitch(K) + k], padded with zeros to a multiple of 4 entries
// so every sample starts 16-byte aligned. The later reordering by the bin
// coordinate then moves whole contiguous samples (gather_transpose in
// binning.cu) instead of single elements of K separate rows, and the
// unbinned LSE passes of MIXED stream it as contiguous runs (lse_smaj.cu).
constexpr int kStageCols = 16;
constexpr int kStageThreads = 256;
constexpr int kStageRows = kStageThreads / kStageCols;  // row residues covered at once
constexpr int kStagePitch = kStageCols + 1;             // shared-memory row pitch (doubles)

size_t stage_smem_bytes(int64_t K) { return static_cast<size_t>(K) * kStagePitch * sizeof(double); }

template <bool kShift>
__global__ void __launch_bounds__(kStageThreads) stage_kernel(const double* __restrict__ u, int64_t K, int64_t N,
                                                              int64_t ldu, double* __restrict__ c,
                                                              void* __restrict__ vst, int* bad) {
  extern __shared__ double xs[];  // [K][kStagePitch]
  __shared__ unsigned long long part[kStageRows][kStageCols];
  __shared__ int okp[kStageRows][kStageCols];
  __shared__ double cmin[kStageCols];
  __shared__ float mhs[kStageCols], mls[kStageCols];
  __shared__ int msp[kStageCols];
  const int t = threadIdx.x;
  const int j = t % kStageCols, g = t / kStageCols;
  const int64_t n0 = static_cast<int64_t>(blockIdx.x) * kStageCols;
  const int64_t n = n0 + j;
  const bool inb = n < N;
  unsigned long long m = ~0ull;
  bool ok = true;
  auto take = [&](int64_t k, double x) {
    xs[k * kStagePitch + j] = x;
    const unsigned long long bx = static_cast<unsigned long long>(__double_as_longlong(x));
    ok &= ((bx >> 52) & 0x7FF) != 0x7FF;
    if constexpr (kShift) {
      const unsigned long long kx = ordered_bits(x);
      m = kx < m ? kx : m;
    }
  };
  if (inb) {
    // sixteen independent loads in flight per thread (K <= 256 in one batch)
    for (int64_t k0 = g; k0 < K; k0 += 16 * kStageRows) {
      double x[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int64_t k = k0 + r * kStageRows;
        if (k < K) x[r] = __ldg(u + k * ldu + n);
      }
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int64_t k = k0 + r * kStageRows;
        if (k < K) take(k, x[r]);
      }
    }
  }
  part[g][j] = m;
  okp[g][j] = ok ? 1 : 0;
  __syncthreads();
  if (t < kStageCols && n0 + t < N) {
    unsigned long long mm = part[0][t];
    int allok = okp[0][t];
#pragma unroll
    for (int r = 1; r < kStageRows; ++r) {
      mm = part[r][t] < mm ? part[r][t] : mm;
      allok &= okp[r][t];
    }
    if (!allok) atomicOr(bad, 1);
    if constexpr (kShift) {
      const double cm = allok ? from_ordered(mm) : 0.0;
      c[n0 + t] = cm;
      cmin[t] = cm;
      float mh = 0.f, ml = 0.f;
      msp[t] = (split_f64_trunc(cm, mh, ml) || cm == 0.0) ? 1 : 0;
      mhs[t] = mh;
      mls[t] = ml;
    }
  }
  __syncthreads();
  // sample-major write-out: the block's samples form one contiguous run
  const int64_t Kp = stage_pitch(K);
  const int ncols = static_cast<int>(N - n0 < kStageCols ? N - n0 : kStageCols);
  for (int jj = 0; jj < ncols; ++jj) {
    if constexpr (kShift) {
      // v = (uh - mh) + (ul - ml) in FP32 from the hi/lo splits of u and of
      // the column minimum (no FP64 arithmetic in the common case); FP64
      // subtraction for values outside the split's range
      const double cm = cmin[jj];
      const float mh = mhs[jj], ml = mls[jj];
      const bool msplit = msp[jj] != 0;
      float* out = static_cast<float*>(vst) + (n0 + jj) * Kp;
      for (int64_t k = t; k < Kp; k += kStageThreads) {
        float r = 0.f;
        if (k < K) {
          const double x = xs[k * kStagePitch + jj];
          float xh, xl;
          if (msplit && split_f64_trunc(x, xh, xl))
            r = __fadd_rn(__fsub_rn(xh, mh), __fsub_rn(xl, ml));
          else
            r = f64_to_f32_rn(x - cm);
        }
        out[k] = r;
      }
    } else {
      double* out = static_cast<double*>(vst) + (n0 + jj) * Kp;
      for (int64_t k = t; k < Kp; k += kStageThreads) out[k] = k < K ? xs[k * kStagePitch + jj] : 0.0;
    }
  }
}

// TMA-fed variant of the MIXED staging for K <= 512 (u 16-byte aligned, row
// pitch a multiple of 16 bytes): persistent CTAs take strips of 16 samples
// (one 128-byte line of each of the K rows) through a two-stage ring of 2-D
// TMA loads; the column minima are taken over the swizzled tile, the
// converted samples are written to a padded shared-memory tile and leave by
// 1-D bulk stores (one contiguous K-vector per sample), so the threads only
// do the arithmetic. Same results as stage_kernel<true>.
constexpr int kStThreads = 512;
constexpr int kStCols = 16;                    // FP64 samples per strip
constexpr int kStRows = kStThreads / kStCols;  // row residues covered at once
constexpr uint32_t kStSpin = 1u << 28;

__device__ __forceinline__ void bulk_store_1d(void* gdst, const void* ssrc, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(smem_u32(ssrc)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// shared-memory pitch (floats) of one converted sample: Kp, or Kp + 4 when
// Kp / 4 is even, so the 16 samples written by one warp spread over the banks
__host__ __device__ inline int64_t stage_tma_ypitch(int64_t Kp) { return ((Kp / 4) & 1) ? Kp : Kp + 4; }

struct StageTmaSmem {
  static __host__ __device__ size_t xbytes(int nbox, int box_rows) {
    return static_cast<size_t>(nbox) * box_rows * 128;
  }
  static __host__ __device__ size_t ybytes(int64_t K) {
    return static_cast<size_t>(kStCols) * stage_tma_ypitch(stage_pitch(K)) * 4;
  }
  static __host__ __device__ size_t total(int64_t K, int nbox, int box_rows) {
    return 2 * xbytes(nbox, box_rows) + 2 * ybytes(K) + 1024 /* alignment */ + 64 /* barriers */;
  }
};

__global__ void __launch_bounds__(kStThreads, 1) stage_tma_kernel(const __grid_constant__ CUtensorMap tmap, int64_t K,
                                                                  int64_t N, int nbox, int box_rows,
                                                                  double* __restrict__ c, float* __restrict__ vst,
                                                                  int* bad, unsigned* err) {
  extern __shared__ __align__(1024) unsigned char st_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(st_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  __shared__ unsigned long long part[kStRows][kStCols + 1];  // padded: a warp reads one column
  __shared__ int nonfinite[kStCols];                         // set by any thread that met one
  __shared__ double cmin[kStCols];
  __shared__ float mhs[kStCols], mls[kStCols];
  __shared__ int msp[kStCols];
  const size_t xb = StageTmaSmem::xbytes(nbox, box_rows);
  const size_t yb = StageTmaSmem::ybytes(K);
  unsigned char* xs = smem;
  float* ys = reinterpret_cast<float*>(smem + 2 * xb);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * xb + 2 * yb);
  const int64_t Kp = stage_pitch(K), Yp = stage_tma_ypitch(Kp);
  const int tid = threadIdx.x, jj = tid % kStCols, r0 = tid / kStCols;
  const int64_t nstrips = (N + kStCols - 1) / kStCols;
  const int64_t first = blockIdx.x, stride = gridDim.x;
  const int count = first < nstrips ? static_cast<int>((nstrips - 1 - first) / stride + 1) : 0;
  const uint32_t tx = static_cast<uint32_t>(xb);
  auto issue = [&](int s, int it) {
    const int64_t strip = first + static_cast<int64_t>(it) * stride;
    mbar_expect_tx(&bars[s], tx);
    for (int b = 0; b < nbox; ++b)
      tma_load_2d(xs + s * xb + static_cast<size_t>(b) * box_rows * 128, &tmap, &bars[s],
                  static_cast<int>(strip * kStCols), b * box_rows);
  };
  if (tid < kStCols) nonfinite[tid] = 0;
  if (tid == 0) {
    prefetch_tmap(&tmap);
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_barrier_init();
    for (int s = 0; s < 2 && s < count; ++s) issue(s, s);
  }
  __syncthreads();
  int it_fail = -1;
  for (int it = 0; it < count; ++it) {
    const int s = it & 1;
    const bool ok_wait = mbar_wait_bounded(&bars[s], static_cast<uint32_t>((it >> 1) & 1), kStSpin);
    if (__syncthreads_or(!ok_wait)) {
      it_fail = it;
      break;
    }
    const int64_t n0 = (first + static_cast<int64_t>(it) * stride) * kStCols;
    const int ns = static_cast<int>(N - n0 < kStCols ? N - n0 : kStCols);
    const unsigned char* X = xs + s * xb;
    // rows k = r0 + 32 i share the swizzle phase k & 7 = r0 & 7: one base
    // address per thread, 32 rows (4096 bytes) per step
    const unsigned char* xp = X + r0 * 128 + (((jj >> 1) ^ (r0 & 7)) << 4) + (jj & 1) * 8;
    const int Ki = static_cast<int>(K), Kpi = static_cast<int>(Kp);
    // pass 1: column minimum (order-preserving integer image) and finiteness
    unsigned long long m = ~0ull;
    bool ok = true;
#pragma unroll 4
    for (int k = r0; k < Ki; k += kStRows) {
      const double x = *reinterpret_cast<const double*>(xp + (k - r0) * 128);
      const unsigned long long bx = static_cast<unsigned long long>(__double_as_longlong(x));
      ok &= ((bx >> 52) & 0x7FF) != 0x7FF;
      const unsigned long long kx = ordered_bits(x);
      m = kx < m ? kx : m;
    }
    part[r0][jj] = m;
    if (!ok) nonfinite[jj] = 1;
    // the bulk stores of two strips ago must have read their tile
    if (tid == 0) bulk_wait_read1();
    __syncthreads();
    // warp w reduces the kStRows partials of column w: kStRows / 32 per
    // lane, then the 64-bit minimum as the minimum of the high words and of
    // the low words among the lanes that hold that high word (one redux each)
    {
      const int w = tid >> 5, l = tid & 31;
      static_assert(kStRows % 32 == 0 && kStThreads / 32 >= kStCols, "one warp per column");
      if (w < ns) {
        unsigned long long pv = part[l][w];
#pragma unroll
        for (int q = l + 32; q < kStRows; q += 32) pv = part[q][w] < pv ? part[q][w] : pv;
        const unsigned ph = static_cast<unsigned>(pv >> 32), pl = static_cast<unsigned>(pv);
        const unsigned mh32 = __reduce_min_sync(0xffffffffu, ph);
        const unsigned ml32 = __reduce_min_sync(0xffffffffu, ph == mh32 ? pl : 0xffffffffu);
        if (l == 0) {
          const unsigned long long mm = (static_cast<unsigned long long>(mh32) << 32) | ml32;
          const bool allok = nonfinite[w] == 0;
          nonfinite[w] = 0;  // read by this lane only; set again after the next barrier
          if (!allok) atomicOr(bad, 1);
          const double cm = allok ? from_ordered(mm) : 0.0;
          c[n0 + w] = cm;
          cmin[w] = cm;
          float mh = 0.f, ml = 0.f;
          msp[w] = (split_f64_trunc(cm, mh, ml) || cm == 0.0) ? 1 : 0;
          mhs[w] = mh;
          mls[w] = ml;
        }
      }
    }
    __syncthreads();
    // pass 2: fl32(u - c) as (uh - ch) + (ul - cl), into the sample-major tile
    float* Y = ys + static_cast<size_t>(it & 1) * (yb / 4);
    if (jj < ns) {
      const double cm = cmin[jj];
      const float mh = mhs[jj], ml = mls[jj];
      const bool msplit = msp[jj] != 0;
      float* yp = Y + jj * Yp;
#pragma unroll 4
      for (int k = r0; k < Kpi; k += kStRows) {
        float r = 0.f;
        if (k < Ki) {
          const double x = *reinterpret_cast<const double*>(xp + (k - r0) * 128);
          float xh, xl;
          if (msplit && split_f64_trunc(x, xh, xl))
            r = __fadd_rn(__fsub_rn(xh, mh), __fsub_rn(xl, ml));
          else
            r = f64_to_f32_rn(x - cm);
        }
        yp[k] = r;
      }
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      for (int q = 0; q < ns; ++q)
        bulk_store_1d(vst + (n0 + q) * Kp, Y + q * Yp, static_cast<uint32_t>(Kp * 4));
      bulk_commit();
      if (it + 2 < count) issue(s, it + 2);  // the tile of stage s is no longer read
    }
  }
  if (tid == 0) {
    if (it_fail >= 0) {
      atomicAdd(err, 1u);
      for (int j = it_fail; j < count && j < it_fail + 2; ++j)
        (void)mbar_wait_bounded(&bars[j & 1], static_cast<uint32_t>((j >> 1) & 1), kStSpin);
    }
    bulk_wait_all();
  }
  __syncthreads();
}

// Row-major K x n (pitch ld) -> sample-major n x Kp through 32 x 32 tiles.
__global__ void level_to_samples_kernel(const float* __restrict__ v, int64_t K, int64_t n, int64_t ld,
                                        float* __restrict__ out) {
  __shared__ float tile[32][33];
  const int64_t Kp = stage_pitch(K);
  const int64_t p0 = static_cast<int64_t>(blockIdx.x) * 32, k0 = static_cast<int64_t>(blockIdx.y) * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int64_t k = k0 + r, p = p0 + tx;
    tile[r][tx] = (k < K && p < n) ? v[k * ld + p] : 0.f;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int64_t p = p0 + r, k = k0 + tx;
    if (p < n && k < Kp) out[p * Kp + k] = tile[tx][r];
  }
}

// Per-column re-centring of a binned FP32 level at the current f: column p
// gets o_p = max_k (a_k - v_kp), a_k = f_k + ln N_k, added to every entry,
// so the exponents a_k - v_kp of its dominant states are near 0 instead of
// near the size of a_k. A per-column shift leaves Eq. 1 unchanged (it
// cancels between numerator and denominator); the FP32 rounding of the
// shifted values is a fixed perturbation of the level's data, while the
// rounding of the exponents, which moves with f from step to step, is then
// that of numbers near 0.
constexpr int kRecCols = 32;
constexpr int kRecGroups = 8;  // row groups (warps) per block
__global__ void __launch_bounds__(kRecCols * kRecGroups) recenter_kernel(float* __restrict__ v, int64_t K, int64_t n,
                                                                         int64_t ld, const double* __restrict__ f,
                                                                         const double* __restrict__ logN) {
  __shared__ float a_s[1024];
  __shared__ float part[kRecGroups][kRecCols];
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  for (int64_t k = threadIdx.x; k < K; k += kRecCols * kRecGroups) a_s[k] = static_cast<float>(f[k] + logN[k]);
  __syncthreads();
  const int64_t p = static_cast<int64_t>(blockIdx.x) * kRecCols + lane;
  float m = -INFINITY;
  if (p < n) {
    // rows grp, grp + 8, ...; eight loads in flight
    for (int64_t k0 = grp; k0 < K; k0 += 8 * kRecGroups) {
      float x[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int64_t k = k0 + r * kRecGroups;
        x[r] = k < K ? a_s[k] - v[k * ld + p] : -INFINITY;
      }
#pragma unroll
      for (int r = 0; r < 8; ++r) m = fmaxf(m, x[r]);
    }
  }
  part[grp][lane] = m;
  __syncthreads();
#pragma unroll
  for (int g = 0; g < kRecGroups; ++g) m = fmaxf(m, part[g][lane]);
  if (p >= n) return;
  for (int64_t k = grp; k < K; k += kRecGroups) v[k * ld + p] += m;
}

__global__ void finite_kernel(const double* __restrict__ x, int64_t n, int* bad) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n && !isfinite(x[i])) atomicOr(bad, 1);
}

// out = (f + t d) - (f_0 + t d_0); t = 1 gives f + d exactly
__global__ void add_gauge_kernel(const double* __restrict__ f, const double* __restrict__ d, double* __restrict__ out,
                                 int64_t K, double t) {
  __shared__ double base;
  if (threadIdx.x == 0) base = fma(t, d[0], f[0]);
  __syncthreads();
  for (int64_t k = threadIdx.x; k < K; k += blockDim.x) out[k] = fma(t, d[k], f[k]) - base;
}

}  // namespace

mbar_status stage_samples(const double* u, int64_t K, int64_t N, int64_t ldu, double* c, void* vst, int dtype_bytes,
                          int* bad, unsigned* err, cudaStream_t st) {
  if (dtype_bytes == 4 && K <= 512 && (reinterpret_cast<uintptr_t>(u) & 15) == 0 && (ldu * 8) % 16 == 0) {
    const int box_rows = static_cast<int>(std::min<int64_t>(256, round_up(K, 8)));
    const int nbox = static_cast<int>(ceil_div(K, box_rows));
    CUtensorMap map;
    if (make_tmap_2d(&map, u, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, K, N, ldu, kStCols, box_rows) == MBAR_OK) {
      const size_t smem = StageTmaSmem::total(K, nbox, box_rows);
      static bool init = false;
      {
        std::lock_guard<std::recursive_mutex> lock(init_mutex());
        if (!init) {
          int dev = 0, optin = 0;
          cudaGetDevice(&dev);
          cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
          cudaFuncAttributes fa = {};
          BUMBAR_CUDA(cudaFuncGetAttributes(&fa, stage_tma_kernel));
          // the dynamic part may take what the static arrays leave
          BUMBAR_CUDA(cudaFuncSetAttribute(stage_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           optin - static_cast<int>(fa.sharedSizeBytes)));
          init = true;
        }
      }
      const int64_t strips = ceil_div(N, kStCols);
      const unsigned grid = static_cast<unsigned>(std::min<int64_t>(strips, num_sms()));
      stage_tma_kernel<<<grid, kStThreads, smem, st>>>(map, K, N, nbox, box_rows, c, static_cast<float*>(vst), bad,
                                                       err);
      count_launches(1);
      BUMBAR_CUDA(cudaGetLastError());
      return MBAR_OK;
    }
    cudaGetLastError();
  }
  const size_t smem = stage_smem_bytes(K);
  {
    std::lock_guard<std::recursive_mutex> lock(init_mutex());
    static bool init = false;
    if (!init) {
      int dev = 0, optin = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      const int lim = optin - 8 * 1024;  // room for the static arrays
      cudaFuncSetAttribute(stage_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
      cudaFuncSetAttribute(stage_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
      init = true;
    }
  }
  const unsigned grid = static_cast<unsigned>(ceil_div(N, kStageCols));
  if (dtype_bytes == 4)
    stage_kernel<true><<<grid, kStageThreads, smem, st>>>(u, K, N, ldu, c, vst, bad);
  else
    stage_kernel<false><<<grid, kStageThreads, smem, st>>>(u, K, N, ldu, c, vst, bad);
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

mbar_status level_to_samples(const float* v, int64_t K, int64_t n, int64_t ld, float* out, cudaStream_t st) {
  if (n < 1) return MBAR_OK;
  const dim3 g(static_cast<unsigned>(ceil_div(n, 32)), static_cast<unsigned>(ceil_div(stage_pitch(K), 32)));
  level_to_samples_kernel<<<g, dim3(32, 8), 0, st>>>(v, K, n, ld, out);
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

mbar_status recenter_columns(float* v, int64_t K, int64_t n, int64_t ld, const double* f, const double* logN,
                             cudaStream_t st) {
  if (n < 1) return MBAR_OK;
  recenter_kernel<<<static_cast<unsigned>(ceil_div(n, kRecCols)), kRecCols * kRecGroups, 0, st>>>(v, K, n, ld, f,
                                                                                                 logN);
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

mbar_status vec_add_gauge(const double* f, const double* d, double* out, int64_t K, cudaStream_t st, double t) {
  add_gauge_kernel<<<1, kThreads, 0, st>>>(f, d, out, K, t);
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

// u_kn = a_k + b_k phi_n (factorised potentials, K x N row-major, pitch N),
// the product and the sum each rounded to nearest in binary64 (no FMA), as
// a host evaluating a + b * phi gets them.
__global__ void factorised_u_kernel(const double* __restrict__ a, const double* __restrict__ b,
                                    const double* __restrict__ phi, int64_t K, int64_t N, double* __restrict__ u) {
  const int64_t k = blockIdx.y;
  const double ak = a[k], bk = b[k];
  double* row = u + k * N;
  for (int64_t n = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; n < N;
       n += static_cast<int64_t>(gridDim.x) * blockDim.x)
    row[n] = __dadd_rn(ak, __dmul_rn(bk, phi[n]));
}

mbar_status factorised_u(const double* a, const double* b, const double* phi, int64_t K, int64_t N, double* u,
                         cudaStream_t st) {
  const unsigned gx = static_cast<unsigned>(std::min<int64_t>(ceil_div(N, 256), 1024));
  factorised_u_kernel<<<dim3(gx, static_cast<unsigned>(K)), 256, 0, st>>>(a, b, phi, K, N, u);
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

// ---------------------------------------------------------------------------
// Binned levels of a factorised context (u_kp = a_k + b_k phi_p): the mean of
// the members' u is a_k + b_k phibar_b with phibar_b the mean of the members'
// coordinate, so a level's FP32 store is generated from a, b and the bin
// means of phi instead of being summed from a K x N store. Column b is
// shifted by c_b = min_k (a_k + b_k phibar_b) like the unbinned MIXED store
// (v >= 0, 0 at the minimum; any per-column shift leaves Eq. 1 unchanged).
// The sums are unevaluated FP32 pairs (about 44 significant bits), so no
// FP64 arithmetic runs per entry.
namespace {

struct Pair {
  float hi, lo;
};

__device__ __forceinline__ Pair pair_of(double x) {
  Pair p;
  p.hi = static_cast<float>(x);
  p.lo = static_cast<float>(x - static_cast<double>(p.hi));
  return p;
}

// a + b phi as an unevaluated pair (the dropped b_lo phi_lo term is 2^-48 of
// the product)
// (explicitly rounded operations: contracting the product into the sum
// would break the error-free transformations)
__device__ __forceinline__ Pair affine_pair(Pair a, Pair b, Pair ph) {
  const float pr = __fmul_rn(b.hi, ph.hi);
  const float pe = __fmaf_rn(b.hi, ph.hi, -pr);
  const float small = __fadd_rn(__fmaf_rn(b.hi, ph.lo, __fmaf_rn(b.lo, ph.hi, pe)), a.lo);
  const float s = __fadd_rn(a.hi, pr);
  const float bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(pr, bb));  // TwoSum error of a.hi + pr
  Pair r;
  r.hi = s;
  r.lo = __fadd_rn(e, small);
  return r;
}

__device__ __forceinline__ bool pair_less(Pair x, Pair y) {
  return __fadd_rn(__fsub_rn(x.hi, y.hi), __fsub_rn(x.lo, y.lo)) < 0.f;
}

// (a_k, b_k) as FP32 pairs, once per level
__global__ void fact_state_pairs(const double* __restrict__ a, const double* __restrict__ b, int64_t K,
                                 float4* __restrict__ ab) {
  const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const Pair pa = pair_of(a[k]), pb = pair_of(b[k]);
  ab[k] = make_float4(pa.hi, pa.lo, pb.hi, pb.lo);
}

__device__ __forceinline__ Pair state_a(float4 v) { return Pair{v.x, v.y}; }
__device__ __forceinline__ Pair state_b(float4 v) { return Pair{v.z, v.w}; }

// c_b = min_k (a_k + b_k phibar_b), one thread per bin
__global__ void fact_level_min(const float4* __restrict__ ab, const double* __restrict__ phibar, int64_t K,
                               int64_t nb, float2* __restrict__ cmin) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  const Pair ph = pair_of(phibar[j]);
  float4 s0 = ab[0];
  Pair m = affine_pair(state_a(s0), state_b(s0), ph);
  for (int64_t k = 1; k < K; ++k) {
    const float4 sk = ab[k];
    const Pair u = affine_pair(state_a(sk), state_b(sk), ph);
    if (pair_less(u, m)) m = u;
  }
  cmin[j] = make_float2(m.hi, m.lo);
}

// v_kb = fl32(a_k + b_k phibar_b - c_b): block rows = states, columns = bins
__global__ void fact_level_fill(const float4* __restrict__ ab, const double* __restrict__ phibar,
                                const float2* __restrict__ cmin, int64_t K, int64_t nb, float* __restrict__ out,
                                int64_t ld) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t k = blockIdx.y;
  if (j >= nb || k >= K) return;
  const float4 sk = ab[k];
  const Pair u = affine_pair(state_a(sk), state_b(sk), pair_of(phibar[j]));
  const float2 c = cmin[j];
  const float d = __fsub_rn(u.hi, c.x);
  const float bb = __fsub_rn(d, u.hi);
  const float e = __fadd_rn(__fsub_rn(u.hi, __fsub_rn(d, bb)), __fsub_rn(-c.x, bb));  // TwoSum error of u.hi - c.hi
  const float v = __fadd_rn(d, __fsub_rn(__fadd_rn(e, u.lo), c.y));
  out[k * ld + j] = v > 0.f ? v : 0.f;  // >= 0 up to the pairs' rounding
}

}  // namespace

size_t fact_level_tmp_bytes(int64_t K, int64_t nb) {
  return static_cast<size_t>(round_up(K * 16, 256)) + static_cast<size_t>(round_up(nb * 8, 256));
}

mbar_status fact_level_store(const double* a, const double* b, const double* phibar, int64_t K, int64_t nb,
                             float* out, int64_t ld, void* tmp, cudaStream_t st) {
  if (nb <= 0) return MBAR_OK;
  float4* ab = static_cast<float4*>(tmp);
  float2* cmin = reinterpret_cast<float2*>(static_cast<unsigned char*>(tmp) + round_up(K * 16, 256));
  const unsigned gx = static_cast<unsigned>(ceil_div(nb, 256));
  fact_state_pairs<<<static_cast<unsigned>(ceil_div(K, 256)), 256, 0, st>>>(a, b, K, ab);
  fact_level_min<<<gx, 256, 0, st>>>(ab, phibar, K, nb, cmin);
  fact_level_fill<<<dim3(gx, static_cast<unsigned>(K)), 256, 0, st>>>(ab, phibar, cmin, K, nb, out, ld);
  count_launches(3);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

}  // namespace bumbar
