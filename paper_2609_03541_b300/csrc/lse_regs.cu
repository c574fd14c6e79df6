// Register-resident variant of the fused paired-LSE pass for FP32 data and
// K <= 512 (the mixed-precision hot path; the tiled variant in lse.cu
// covers FP64 and larger K).
//
// Same strip pipeline as lse.cu (2-D TMA boxes, 128-byte swizzle, mbarrier
// stages), but each thread keeps its slice of a strip in registers instead
// of writing e back to shared memory:
//   * thread (warp w, lane l) owns column c = 4 (w % 8) + l / 8 of the strip
//     and rows k_j = 8 (w / 8) + l % 8 + 16 j, j < J (J = ceil(K / 16));
//   * A1 reads v once from shared memory (conflict-free: a warp reads one
//     16-byte chunk of 8 different rows whose swizzle phases differ) and
//     keeps x_j = a_kj - v log2(e) in registers; column max by 8-lane
//     shuffles and one shared-memory exchange between the two row halves;
//     the stage is then released and its next TMA load issued at once;
//   * A2 turns x_j into e_j = 2^(x_j - max) in place; column sum the same way;
//   * B accumulates e_j * H_c / s_c into per-thread row partials acc_j.
// Every 32 strips the four column lanes that share rows are combined by
// shuffles and added into one FP64 slot per (warp column group, row) in
// shared memory (fixed order, deterministic); at the end the eight slots of
// a row are summed in order and the common epilogue (lse_common.cuh) runs.
// Per entry: one shared-memory read of v and one (broadcast-friendly) of a,
// one FFMA, one max, one SFU ex2, two adds and one FFMA.
#include <cmath>

#include "common.cuh"
#include "kernels.cuh"
#include "lse_common.cuh"

namespace bumbar {

namespace {

constexpr int kRThreads = 512;
constexpr int kRowGroups = 16;     // 2 row halves x 8 lane residues
constexpr int kFlush = 32;         // strips between FP32 -> FP64 flushes
constexpr uint32_t kSpin = 1u << 28;

__host__ __device__ inline size_t rupr(size_t x, size_t m) { return (x + m - 1) / m * m; }

}  // namespace

// shared memory: stages | a [Kpad] f32 | slots [8][Kpad] f64 | colm[2][32] |
//                cols[2][32] | mbarriers[8] | epilogue [K] f64
struct RegsSmem {
  static __host__ __device__ size_t kpad(int K) { return rupr(static_cast<size_t>(K), 16); }
  static __host__ __device__ size_t extra(int K) {
    return kpad(K) * 4 + 8 * kpad(K) * 8 + 2 * 32 * 4 * 2 + 64 + rupr(static_cast<size_t>(K) * 8, 16);
  }
};

template <int J>
__global__ void __launch_bounds__(kRThreads, 1) lse_regs_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                LseParams p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int K = p.K;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (p.ctrl != nullptr && p.skip_if_done && p.ctrl->done) return;

  const size_t sbytes = static_cast<size_t>(p.nbox) * p.box_rows * 128;
  const size_t kp = RegsSmem::kpad(K);
  unsigned char* cur = smem + p.stages * sbytes;
  float* a_s = reinterpret_cast<float*>(cur);
  cur += kp * 4;
  double* slots = reinterpret_cast<double*>(cur);  // [8][kp]
  cur += 8 * kp * 8;
  float* colm = reinterpret_cast<float*>(cur);     // [2][32]
  float* cols = colm + 64;                         // [2][32]
  cur += 2 * 32 * 4 * 2;
  uint64_t* bars = reinterpret_cast<uint64_t*>(cur);
  cur += 64;
  double* red_s = reinterpret_cast<double*>(cur);

  const int num_strips = p.num_strips;
  const int my_first = blockIdx.x, stride = gridDim.x;
  const int my_count = (my_first < num_strips) ? (num_strips - 1 - my_first) / stride + 1 : 0;

  if (tid == 0) {
    prefetch_tmap(&tmap);
    for (int s = 0; s < p.stages; ++s) mbar_init(&bars[s], 1);
    fence_barrier_init();
  }
  for (int k = tid; k < static_cast<int>(kp); k += kRThreads)
    a_s[k] = k < K ? static_cast<float>((p.f[k] + p.logN[k]) * 1.4426950408889634) : 0.f;
  for (int i = tid; i < static_cast<int>(8 * kp); i += kRThreads) slots[i] = 0.0;
  __syncthreads();

  const uint32_t tx = static_cast<uint32_t>(sbytes);
  if (tid == 0) {
    for (int s = 0; s < p.stages && s < my_count; ++s) {
      unsigned char* dst = smem + s * sbytes;
      mbar_expect_tx(&bars[s], tx);
      for (int b = 0; b < p.nbox; ++b)
        tma_load_2d(dst + static_cast<size_t>(b) * p.box_rows * 128, &tmap, &bars[s], (my_first + s * stride) * 32,
                    b * p.box_rows);
    }
  }

  const int q = warp & 7, h = warp >> 3;
  const int col = q * 4 + (lane >> 3);
  const int r0 = h * 8 + (lane & 7);
  const uint32_t off0 = static_cast<uint32_t>(r0) * 128u + ((static_cast<uint32_t>(q) ^ (lane & 7u)) << 4) +
                        static_cast<uint32_t>((lane >> 3) * 4);
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
      const int k = r0 + kRowGroups * j;
      if (lane < 8 && k < K) slots[q * kp + k] += static_cast<double>(v);
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
    const int gcol = strip * 32 + col;

    // A1: x_j in registers, column max
    float x[J];
    float m0 = -INFINITY, m1 = -INFINITY;
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int k = r0 + kRowGroups * j;
      if (k < K) {
        const float v = *reinterpret_cast<const float*>(tile + off0 + j * (kRowGroups * 128u));
        x[j] = fmaf(-v, kLog2e, a_s[k]);
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
    if ((lane & 7) == 0) colm[h * 32 + col] = m;
    fence_proxy_async_smem();
    __syncthreads();  // also: every warp is done reading this stage
    if (tid == 0 && it + p.stages < my_count) {
      unsigned char* dst = smem + s * sbytes;
      mbar_expect_tx(&bars[s], tx);
      for (int b = 0; b < p.nbox; ++b)
        tma_load_2d(dst + static_cast<size_t>(b) * p.box_rows * 128, &tmap, &bars[s],
                    (my_first + (it + p.stages) * stride) * 32, b * p.box_rows);
    }
    m = fmaxf(colm[col], colm[32 + col]);

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
    if ((lane & 7) == 0) cols[h * 32 + col] = ssum;
    __syncthreads();
    const float S = cols[col] + cols[32 + col];
    const bool valid = gcol < p.n;
    float w = 0.f;
    if (valid) {
      w = (p.H ? static_cast<float>(p.H[gcol]) : 1.f) / S;
      if (p.logden != nullptr && h == 0 && (lane & 7) == 0)
        static_cast<float*>(p.logden)[gcol] = (m + __log2f(S)) * kLn2;
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
  double rowsum[(1024 + kRThreads - 1) / kRThreads];
#pragma unroll
  for (int j = 0; j < (1024 + kRThreads - 1) / kRThreads; ++j) {
    const int k = tid + j * kRThreads;
    double t = 0.0;
    if (k < K) {
#pragma unroll
      for (int g = 0; g < 8; ++g) t += slots[g * kp + k];
    }
    rowsum[j] = t;
  }
  lse_finish<kRThreads, (1024 + kRThreads - 1) / kRThreads>(p, rowsum, red_s);
}

// ---------------------------------------------------------------------------

namespace {

template <int J>
int regs_occupancy(size_t smem) {
  static size_t max_dyn = 0;
  if (max_dyn == 0) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, lse_regs_kernel<J>);
    max_dyn = static_cast<size_t>(optin) - fa.sharedSizeBytes;
    cudaFuncSetAttribute(lse_regs_kernel<J>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(max_dyn));
  }
  if (smem > max_dyn) return 0;
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, lse_regs_kernel<J>, kRThreads, smem) != cudaSuccess)
    blocks = 0;
  return blocks;
}

int regs_J(int64_t K) {
  const int64_t j = ceil_div(K, kRowGroups);
  if (j <= 4) return 4;
  if (j <= 8) return 8;
  if (j <= 16) return 16;
  if (j <= 32) return 32;
  return 0;  // larger K: the tiled variant (the FP64 row slots would not fit next to two stages)
}

}  // namespace

bool lse_regs_supported(int64_t K, int dtype_bytes) { return dtype_bytes == 4 && regs_J(K) > 0; }

LsePlan lse_regs_plan(int64_t K, int64_t n) {
  LsePlan pl{};
  pl.C = 32;
  pl.variant = 1;
  pl.J = regs_J(K);
  pl.threads = kRThreads;
  pl.num_strips = static_cast<int>(ceil_div(n, 32));
  pl.box_rows = static_cast<int>(std::min<int64_t>(256, round_up(K, 8)));
  pl.nbox = static_cast<int>(ceil_div(K, pl.box_rows));
  const size_t sb = static_cast<size_t>(pl.nbox) * pl.box_rows * 128;
  const size_t extra = RegsSmem::extra(static_cast<int>(K)) + 1024;
  // as many stages (2..4) as fit next to the slots
  pl.stages = 4;
  while (pl.stages > 2 && pl.stages * sb + extra > 220 * 1024) --pl.stages;
  pl.smem = pl.stages * sb + extra;
  static int occ_cache[1025] = {};
  int* occ = &occ_cache[std::min<int64_t>(K, 1024)];
  if (*occ == 0) {
    switch (pl.J) {
      case 4: *occ = regs_occupancy<4>(pl.smem); break;
      case 8: *occ = regs_occupancy<8>(pl.smem); break;
      case 16: *occ = regs_occupancy<16>(pl.smem); break;
      case 32: *occ = regs_occupancy<32>(pl.smem); break;
      case 48: *occ = regs_occupancy<48>(pl.smem); break;
      default: *occ = 0;
    }
    cudaGetLastError();
  }
  pl.grid = static_cast<int>(std::min<int64_t>(pl.num_strips, static_cast<int64_t>(std::max(*occ, 1)) * num_sms()));
  pl.grid = std::max(pl.grid, 1);
  pl.ok = *occ > 0;
  return pl;
}

mbar_status lse_regs_launch(const CUtensorMap& tmap, const LsePlan& pl, const LseParams& prm, cudaStream_t st) {
  switch (pl.J) {
    case 4: lse_regs_kernel<4><<<pl.grid, kRThreads, pl.smem, st>>>(tmap, prm); break;
    case 8: lse_regs_kernel<8><<<pl.grid, kRThreads, pl.smem, st>>>(tmap, prm); break;
    case 16: lse_regs_kernel<16><<<pl.grid, kRThreads, pl.smem, st>>>(tmap, prm); break;
    case 32: lse_regs_kernel<32><<<pl.grid, kRThreads, pl.smem, st>>>(tmap, prm); break;
    case 48: lse_regs_kernel<48><<<pl.grid, kRThreads, pl.smem, st>>>(tmap, prm); break;
    default:
      set_error("lse_regs_launch: unsupported J=%d", pl.J);
      return MBAR_EUNSUPPORTED;
  }
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

}  // namespace bumbar
