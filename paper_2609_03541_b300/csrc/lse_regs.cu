// Register-resident variant of the fused paired-LSE pass for FP32 data and
// K <= 512 (the mixed-precision hot path; the tiled variant in lse.cu
// covers FP64 and larger K).
//
// Same strip pipeline as lse.cu (2-D TMA boxes, 128-byte swizzle, mbarrier
// stages), but each thread keeps its slice of a strip in registers instead
// of writing e back to shared memory. A stage holds SUB sub-tiles of 32
// columns x all K rows; 16 warps cover them as 8 column chunks x H row
// halves x SUB sub-tiles (H * SUB = 2):
//   * thread (warp w, lane l) owns column c = 4 (w % 8) + l / 8 of its
//     sub-tile and rows k_j = 8 h + l % 8 + 8 H j, j < J (J = ceil(K / 8H));
//   * A1 reads v once from shared memory (conflict-free: a warp reads one
//     16-byte chunk of 8 rows whose swizzle phases differ) and keeps
//     x_j = a_kj - v log2(e) in registers; column max by 8-lane shuffles
//     (plus one shared-memory exchange between row halves when H = 2); the
//     stage is then released and its next TMA load issued at once;
//   * A2 turns x_j into e_j = 2^(x_j - max) in place; column sum likewise;
//   * B accumulates e_j * H_c / s_c into per-thread row partials acc_j.
// Every 64 stages the four column lanes that share rows are combined by
// shuffles and added by TwoSum into one slot per warp and row in shared
// memory, an unevaluated FP32 sum hi + lo (fixed order, deterministic; FP64
// adds there stall every warp on B300's slow FP64 pipe, as all warps fold
// in the same stage); at the end a row's slots are summed in order in FP64
// and the common epilogue (lse_common.cuh) runs. 1 / column sum by
// rcp.approx (1 ulp). H = 1 (two 32-column
// sub-tiles per stage, no cross-warp exchange) serves K <= 256; H = 2 serves
// K <= 512. Per entry: one shared-memory read of v and one of a, two FFMA
// and an add for x, one max, one SFU ex2, two adds and one FFMA.
//
// x_kp = a_k log2(e) - v_kp log2(e) is formed from unevaluated FP32 pairs,
// (a_hi, a_lo) for the state offset and (kLog2e, kLog2eLo) for the scale.
// A single FP32 offset would be quantised to the FP32 spacing at |a_k|
// (about 1e-4 kT at |a_k| ~ 700, as on tempering data spread over hundreds
// of kT), the same rounding for every column, which turns the SCI map into
// a step function of f; a single FP32 scale multiplies every v by the same
// relative error (1.3e-8), which moves the fixed point by 1.3e-8 times the
// energy differences. With the pairs x_kp is rounded once per entry, at
// positions that differ from column to column.
#include <cmath>

#include "common.cuh"
#include "kernels.cuh"
#include "lse_common.cuh"

namespace bumbar {

namespace {

constexpr int kRThreads = 512;
constexpr int kFlush = 64;  // stages between folds of the FP32 row partials
constexpr uint32_t kSpin = 1u << 28;

__host__ __device__ inline size_t rupr(size_t x, size_t m) { return (x + m - 1) / m * m; }

}  // namespace

// shared memory: stages | a [Kpad] (hi, lo) f32 pairs | slots [16][Kpad] (hi, lo) f32 | colm[2][32] |
//                cols[2][32] | mbarriers[8]
struct RegsSmem {
  static __host__ __device__ size_t kpad(int K) { return rupr(static_cast<size_t>(K), 16); }
  static __host__ __device__ size_t extra(int K, int nslots) {
    return kpad(K) * 8 + nslots * kpad(K) * 8 + 2 * 32 * 4 * 2 + 64;
  }
};

template <int J, int H>
__global__ void __launch_bounds__(kRThreads, 1) lse_regs_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                LseParams p) {
  constexpr int SUB = 2 / H;             // 32-column sub-tiles per stage
  constexpr int CS = 32 * SUB;           // columns per stage
  constexpr int RG = 8 * H;              // row groups
  constexpr int NSLOT = 16;              // one per warp
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int K = p.K;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (lse_skip(p)) return;

  const size_t subbytes = static_cast<size_t>(p.nbox) * p.box_rows * 128;
  const size_t sbytes = SUB * subbytes;
  const size_t kp = RegsSmem::kpad(K);
  unsigned char* cur = smem + p.stages * sbytes;
  float2* a_s = reinterpret_cast<float2*>(cur);
  cur += kp * 8;
  float2* slots = reinterpret_cast<float2*>(cur);  // [NSLOT][kp] unevaluated sums hi + lo
  cur += NSLOT * kp * 8;
  float* colm = reinterpret_cast<float*>(cur);     // [2][32]
  float* cols = colm + 64;                         // [2][32]
  cur += 2 * 32 * 4 * 2;
  uint64_t* bars = reinterpret_cast<uint64_t*>(cur);

  const int num_strips = p.num_strips;
  const int my_first = blockIdx.x, stride = gridDim.x;
  const int my_count = (my_first < num_strips) ? (num_strips - 1 - my_first) / stride + 1 : 0;

  if (tid == 0) {
    prefetch_tmap(&tmap);
    for (int s = 0; s < p.stages; ++s) mbar_init(&bars[s], 1);
    fence_barrier_init();
  }
  for (int k = tid; k < static_cast<int>(kp); k += kRThreads) {
    const double a = k < K ? (p.f[k] + p.logN[k]) * 1.4426950408889634 : 0.0;
    const float hi = static_cast<float>(a);
    a_s[k] = make_float2(hi, isfinite(hi) ? static_cast<float>(a - static_cast<double>(hi)) : 0.f);
  }
  for (int i = tid; i < static_cast<int>(NSLOT * kp); i += kRThreads) slots[i] = make_float2(0.f, 0.f);
  __syncthreads();

  const uint32_t tx = static_cast<uint32_t>(sbytes);
  auto issue = [&](int stage, int strip) {
    unsigned char* dst = smem + stage * sbytes;
    mbar_expect_tx(&bars[stage], tx);
#pragma unroll
    for (int sb = 0; sb < SUB; ++sb)
      for (int b = 0; b < p.nbox; ++b)
        tma_load_2d(dst + sb * subbytes + static_cast<size_t>(b) * p.box_rows * 128, &tmap, &bars[stage],
                    strip * CS + sb * 32, b * p.box_rows);
  };
  if (tid == 0) {
    for (int s = 0; s < p.stages && s < my_count; ++s) issue(s, my_first + s * stride);
  }

  const int q = warp & 7;
  const int h = (H == 2) ? (warp >> 3) : 0;
  const int sub = (H == 1) ? (warp >> 3) : 0;
  const int col = q * 4 + (lane >> 3);  // column within the sub-tile
  const int r0 = h * 8 + (lane & 7);
  const uint32_t off0 = static_cast<uint32_t>(sub * subbytes) + static_cast<uint32_t>(r0) * 128u +
                        ((static_cast<uint32_t>(q) ^ (lane & 7u)) << 4) + static_cast<uint32_t>((lane >> 3) * 4);
  constexpr uint32_t kStep = RG * 128u;
  float acc[J];
#pragma unroll
  for (int j = 0; j < J; ++j) acc[j] = 0.f;
  int it_fail = -1;

  auto flush = [&]() {
#pragma unroll
    for (int j = 0; j < J; ++j) {
      float v = acc[j];
      v += __shfl_xor_sync(0xffffffffu, v, 8);
      v += __shfl_xor_sync(0xffffffffu, v, 16);
      const int k = r0 + RG * j;
      if (lane < 8 && k < K) {
        // TwoSum (Knuth): hi + v = sum + err exactly
        const float2 c = slots[warp * kp + k];
        const float sum = c.x + v, bv = sum - c.x;
        const float err = (c.x - (sum - bv)) + (v - bv);
        slots[warp * kp + k] = make_float2(sum, c.y + err);
      }
      acc[j] = 0.f;
    }
  };

  for (int it = 0; it < my_count; ++it) {
    const int s = it % p.stages;
    const uint32_t parity = static_cast<uint32_t>((it / p.stages) & 1);
    const int strip = my_first + it * stride;
    const unsigned char* tile = smem + s * sbytes;
    const bool ok = mbar_wait_bounded(&bars[s], parity, kSpin);
    if (__syncthreads_or(!ok)) {
      it_fail = it;
      break;
    }
    const int gcol = strip * CS + sub * 32 + col;

    // A1: x_j in registers, column max
    float x[J];
    float m0 = -INFINITY, m1 = -INFINITY;
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int k = r0 + RG * j;
      if (k < K) {
        const float v = *reinterpret_cast<const float*>(tile + off0 + j * kStep);
        const float2 a = a_s[k];
        x[j] = fmaf(-v, kLog2e, a.x) + fmaf(-v, kLog2eLo, a.y);
        if (j & 1)
          m1 = fmaxf(m1, x[j]);
        else
          m0 = fmaxf(m0, x[j]);
      } else {
        x[j] = -INFINITY;
      }
    }
    float m = fmaxf(m0, m1);
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 4));
    if constexpr (H == 2) {
      if ((lane & 7) == 0) colm[h * 32 + col] = m;
    }
    fence_proxy_async_smem();
    __syncthreads();  // every warp is done reading this stage
    if (tid == 0 && it + p.stages < my_count) issue(s, my_first + (it + p.stages) * stride);
    if constexpr (H == 2) m = fmaxf(colm[col], colm[32 + col]);

    // A2: e_j = 2^(x_j - m), column sum
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int j = 0; j < J; ++j) {
      x[j] = ex2_approx(x[j] - m);
      if (j & 1)
        s1 += x[j];
      else
        s0 += x[j];
    }
    float ssum = s0 + s1;
    ssum += __shfl_xor_sync(0xffffffffu, ssum, 1);
    ssum += __shfl_xor_sync(0xffffffffu, ssum, 2);
    ssum += __shfl_xor_sync(0xffffffffu, ssum, 4);
    if constexpr (H == 2) {
      if ((lane & 7) == 0) cols[h * 32 + col] = ssum;
      __syncthreads();
      ssum = cols[col] + cols[32 + col];
    }
    const bool valid = gcol < p.n;
    float w = 0.f;
    if (valid) {
      w = (p.H ? static_cast<float>(p.H[gcol]) : 1.f) * rcp_approx(ssum);
      if (p.logden != nullptr && h == 0 && (lane & 7) == 0)
        static_cast<float*>(p.logden)[gcol] = (m + __log2f(ssum)) * kLn2;
    }

    // B: row partials
#pragma unroll
    for (int j = 0; j < J; ++j) acc[j] = fmaf(x[j], w, acc[j]);
    if ((it + 1) % kFlush == 0) flush();
  }

  if (it_fail >= 0) {
    if (tid == 0) {
      atomicAdd(p.err, 1u);
      for (int j = it_fail; j < my_count && j < it_fail + p.stages; ++j)
        (void)mbar_wait_bounded(&bars[j % p.stages], static_cast<uint32_t>((j / p.stages) & 1), kSpin);
    }
    __syncthreads();
  }
  flush();
  __syncthreads();
  constexpr int RPT = (1024 + kRThreads - 1) / kRThreads;
  double rowsum[RPT];
#pragma unroll
  for (int j = 0; j < RPT; ++j) {
    const int k = tid + j * kRThreads;
    double t = 0.0;
    if (k < K) {
#pragma unroll
      for (int g = 0; g < NSLOT; ++g) t += static_cast<double>(slots[g * kp + k].x) + static_cast<double>(slots[g * kp + k].y);
    }
    rowsum[j] = t;
  }
  lse_write_partials<kRThreads, RPT>(p, rowsum);
}

// ---------------------------------------------------------------------------

namespace {

template <int J, int H>
int regs_occupancy(size_t smem) {
  std::lock_guard<std::recursive_mutex> lock(init_mutex());
  static size_t max_dyn = 0;
  if (max_dyn == 0) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, lse_regs_kernel<J, H>);
    max_dyn = static_cast<size_t>(optin) - fa.sharedSizeBytes;
    cudaFuncSetAttribute(lse_regs_kernel<J, H>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(max_dyn));
  }
  if (smem > max_dyn) return 0;
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, lse_regs_kernel<J, H>, kRThreads, smem) != cudaSuccess)
    blocks = 0;
  return blocks;
}

// (J, H) for a given K: H = 1 while J = ceil(K/8) <= 32, else H = 2.
void regs_shape(int64_t K, int* J, int* H) {
  const int64_t j1 = ceil_div(K, 8);
  *H = j1 <= 32 ? 1 : 2;
  const int64_t j = ceil_div(K, 8 * (*H));
  *J = j <= 4 ? 4 : j <= 8 ? 8 : j <= 16 ? 16 : j <= 32 ? 32 : 0;
}

int regs_occ_dispatch(int J, int H, size_t smem) {
  if (H == 1) {
    switch (J) {
      case 4: return regs_occupancy<4, 1>(smem);
      case 8: return regs_occupancy<8, 1>(smem);
      case 16: return regs_occupancy<16, 1>(smem);
      case 32: return regs_occupancy<32, 1>(smem);
    }
  } else {
    switch (J) {
      case 16: return regs_occupancy<16, 2>(smem);
      case 32: return regs_occupancy<32, 2>(smem);
    }
  }
  return 0;
}

}  // namespace

bool lse_regs_supported(int64_t K, int dtype_bytes) {
  if (dtype_bytes != 4 || K < 1) return false;
  int J = 0, H = 0;
  regs_shape(K, &J, &H);
  return J > 0;
}

LsePlan lse_regs_plan(int64_t K, int64_t n) {
  LsePlan pl{};
  int J = 0, H = 0;
  regs_shape(K, &J, &H);
  const int SUB = 2 / H;
  pl.variant = 1;
  pl.J = J;
  pl.H = H;
  pl.C = 32 * SUB;
  pl.threads = kRThreads;
  pl.num_strips = static_cast<int>(ceil_div(n, pl.C));
  pl.box_rows = static_cast<int>(std::min<int64_t>(256, round_up(K, 8)));
  pl.nbox = static_cast<int>(ceil_div(K, pl.box_rows));
  const size_t sb = static_cast<size_t>(SUB) * pl.nbox * pl.box_rows * 128;
  const size_t extra = RegsSmem::extra(static_cast<int>(K), 16) + 1024;
  pl.stages = 4;
  while (pl.stages > 2 && pl.stages * sb + extra > 220 * 1024) --pl.stages;
  pl.smem = pl.stages * sb + extra;
  static int occ_cache[1025] = {};
  int occ = 0;
  {
    std::lock_guard<std::recursive_mutex> lock(init_mutex());
    int* slot = &occ_cache[std::min<int64_t>(K, 1024)];
    if (*slot == 0) {
      *slot = regs_occ_dispatch(J, H, pl.smem);
      cudaGetLastError();
    }
    occ = *slot;
  }
  pl.grid = static_cast<int>(std::min<int64_t>(pl.num_strips, static_cast<int64_t>(std::max(occ, 1)) * num_sms()));
  pl.grid = std::max(pl.grid, 1);
  pl.ok = occ > 0;
  return pl;
}

mbar_status lse_regs_launch(const CUtensorMap& tmap, const LsePlan& pl, const LseParams& prm, cudaStream_t st) {
  const dim3 g(pl.grid), b(kRThreads);
  if (pl.H == 1) {
    switch (pl.J) {
      case 4: lse_regs_kernel<4, 1><<<g, b, pl.smem, st>>>(tmap, prm); break;
      case 8: lse_regs_kernel<8, 1><<<g, b, pl.smem, st>>>(tmap, prm); break;
      case 16: lse_regs_kernel<16, 1><<<g, b, pl.smem, st>>>(tmap, prm); break;
      case 32: lse_regs_kernel<32, 1><<<g, b, pl.smem, st>>>(tmap, prm); break;
      default: set_error("lse_regs_launch: unsupported J=%d", pl.J); return MBAR_EUNSUPPORTED;
    }
  } else {
    switch (pl.J) {
      case 16: lse_regs_kernel<16, 2><<<g, b, pl.smem, st>>>(tmap, prm); break;
      case 32: lse_regs_kernel<32, 2><<<g, b, pl.smem, st>>>(tmap, prm); break;
      default: set_error("lse_regs_launch: unsupported J=%d", pl.J); return MBAR_EUNSUPPORTED;
    }
  }
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

}  // namespace bumbar
