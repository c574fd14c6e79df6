// Overlap matrix G = P~ P~^T on the 5th-generation tensor cores (tcgen05),
// the contraction of the Newton Hessian (H = Laplacian of G, see hessian.cu):
//     P~_ip = sqrt(H_p) exp(f_i + log N_i - v_ip - logden_p)   (FP16),
//     G_ij  = sum_p P~_ip P~_jp                                 (FP32 in TMEM).
//
// Work decomposition: the K states are padded to 128-row tiles. A work item
// is one 128-row A tile (tile bi) and up to four 128-row B tiles
// (bj0 .. bj0+nt-1, bj0 >= bi: upper triangle only), so its accumulator,
// 128 lanes x nt*128 FP32 columns, fits the 512 TMEM columns of one SM. The
// sample axis is split into slices; each CTA owns one (item, slice), with
// the number of slices per item proportional to its work.
//
// Per 64-sample chunk every thread computes P~ for its rows and 8 samples
// (FP32 exponent, SFU ex2), converts to FP16 and stores 16-byte pieces into a
// shared-memory tile in the canonical K-major 128-byte-swizzle layout that
// the UMMA descriptors describe (row r, 16-byte chunk c at r*128 + ((c ^
// r%8) * 16)). One elected thread then issues nt x 4 tcgen05.mma
// (M = 128, N = 128, K = 16) and commits them to an mbarrier; the tile is
// double buffered so the P~ of the next chunk is built while the tensor core
// consumes the current one. The epilogue reads the accumulator with
// tcgen05.ld and writes FP32 partial tiles; a second kernel reduces the
// slices in a fixed order in FP64 and mirrors the upper triangle.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace bumbar {

namespace {

constexpr int kTcThreads = 512;
constexpr int kRowStride = kTcThreads / 8;  // threads per 8-sample group column
constexpr int kChunkCols = 64;                 // samples per chunk = one 128-byte FP16 row
constexpr int kMaxRows = 640;                  // A tile + 4 B tiles
constexpr int kStageBytes = kMaxRows * 128;    // 80 KB per buffer
constexpr int kMaxCtas = 1024;
constexpr uint32_t kMaxSpins = 1u << 28;

struct TcCta {
  int item;     // work item index
  int bi, bj0, nt;
  int64_t c_begin, c_end;
};

struct TcParams {
  const void* v;
  int64_t ld;
  int K;
  int64_t n;
  const double* a;      // f + log N  [K]
  const void* logden;   // [n]
  const int32_t* H;     // [n] or nullptr
  const TcCta* ctas;    // [gridDim.x]
  float* out;           // [gridDim.x][128][512]
  unsigned* err;
};

// ---- tcgen05 / UMMA helpers (inline PTX) ----

// Shared-memory matrix descriptor, K-major, 128-byte swizzle: start address
// >> 4, leading byte offset 16 (not used by this layout), stride byte offset
// 1024 (eight 128-byte rows), descriptor version 1, layout SWIZZLE_128B.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>(16u >> 4) << 16;
  d |= static_cast<uint64_t>(1024u >> 4) << 32;
  d |= static_cast<uint64_t>(1u) << 46;
  d |= static_cast<uint64_t>(2u) << 61;
  return d;
}

// Instruction descriptor of kind::f16: D = F32, A = B = F16, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
  return (1u << 4) | (0u << 7) | (0u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void umma_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* r) {
  uint32_t u[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
        "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15]),
        "=r"(u[16]), "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23]),
        "=r"(u[24]), "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) r[i] = __uint_as_float(u[i]);
}

__device__ __forceinline__ uint32_t pack_half2(float lo, float hi) {
  const __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}

template <typename T>
__global__ void __launch_bounds__(kTcThreads, 1) overlap_tc_kernel(TcParams p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  unsigned char* buf0 = smem;
  float* a2_s = reinterpret_cast<float*>(smem + 2 * kStageBytes);             // [kMaxRows]
  uint64_t* bars = reinterpret_cast<uint64_t*>(a2_s + kMaxRows);             // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2);

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const TcCta job = p.ctas[blockIdx.x];
  const bool a_sep = job.bj0 != job.bi;
  const int rowsA = a_sep ? 128 : 0;
  const int rows = rowsA + job.nt * 128;
  const uint32_t ncols = job.nt == 1 ? 128u : (job.nt == 2 ? 256u : 512u);

  if (warp == 0) tmem_alloc(tmem_slot, ncols);
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_barrier_init();
  }
  for (int lr = tid; lr < rows; lr += kTcThreads) {
    const int row = lr < rowsA ? job.bi * 128 + lr : job.bj0 * 128 + (lr - rowsA);
    a2_s[lr] = row < p.K ? static_cast<float>(p.a[row] * 1.4426950408889634) : -INFINITY;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int64_t nchunks = (job.c_end - job.c_begin + kChunkCols - 1) / kChunkCols;
  const int g = tid & 7;         // 8-sample group of the chunk
  const int rsub = tid >> 3;     // first local row; rows rsub, rsub + kRowStride, ...
  constexpr uint32_t idesc = idesc_f16(128, 128);
  const T* vv = static_cast<const T*>(p.v);
  const T* ld_in = static_cast<const T*>(p.logden);
  bool failed = false;

  for (int64_t c = 0; c < nchunks; ++c) {
    const int b = static_cast<int>(c & 1);
    unsigned char* buf = buf0 + b * kStageBytes;
    if (c >= 2) {
      const bool ok = mbar_wait_bounded(&bars[b], static_cast<uint32_t>(((c - 2) >> 1) & 1), kMaxSpins);
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
    }
    // per-thread column parameters (8 consecutive samples)
    const int64_t col0 = job.c_begin + c * kChunkCols + g * 8;
    float l2[8], sh[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t col = col0 + j;
      if (col < job.c_end) {
        l2[j] = static_cast<float>(static_cast<double>(ld_in[col]) * 1.4426950408889634);
        sh[j] = p.H ? sqrtf(static_cast<float>(p.H[col])) : 1.f;
      } else {
        l2[j] = INFINITY;  // exp2(-inf) = 0: padding samples contribute nothing
        sh[j] = 0.f;
      }
    }
    const bool full8 = col0 + 8 <= job.c_end;
    // four rows per round: issue all loads first, then the SFU work
    constexpr int kRowsPerRound = 4;
    for (int lr0 = rsub; lr0 < rows; lr0 += kRowStride * kRowsPerRound) {
      float x[kRowsPerRound][8];
#pragma unroll
      for (int u = 0; u < kRowsPerRound; ++u) {
        const int lr = lr0 + kRowStride * u;
        const int row = lr < rowsA ? job.bi * 128 + lr : job.bj0 * 128 + (lr - rowsA);
        if (lr < rows && row < p.K) {
          const T* src = vv + static_cast<int64_t>(row) * p.ld + col0;
          if constexpr (sizeof(T) == 4) {
            if (full8) {
              const float4 v0 = *reinterpret_cast<const float4*>(src);
              const float4 v1 = *reinterpret_cast<const float4*>(src + 4);
              x[u][0] = v0.x; x[u][1] = v0.y; x[u][2] = v0.z; x[u][3] = v0.w;
              x[u][4] = v1.x; x[u][5] = v1.y; x[u][6] = v1.z; x[u][7] = v1.w;
            } else {
#pragma unroll
              for (int j = 0; j < 8; ++j) x[u][j] = (col0 + j < job.c_end) ? src[j] : 0.f;
            }
          } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) x[u][j] = (col0 + j < job.c_end) ? static_cast<float>(src[j]) : 0.f;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) x[u][j] = 0.f;
        }
      }
#pragma unroll
      for (int u = 0; u < kRowsPerRound; ++u) {
        const int lr = lr0 + kRowStride * u;
        if (lr < rows) {
          const float a2 = a2_s[lr];
          float pv[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) pv[j] = ex2_approx(fmaf(-x[u][j], kLog2e, a2) - l2[j]) * sh[j];
          uint4 packed;
          packed.x = pack_half2(pv[0], pv[1]);
          packed.y = pack_half2(pv[2], pv[3]);
          packed.z = pack_half2(pv[4], pv[5]);
          packed.w = pack_half2(pv[6], pv[7]);
          *reinterpret_cast<uint4*>(buf + lr * 128 + ((g ^ (lr & 7)) << 4)) = packed;
        }
      }
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t base = smem_u32(buf);
      for (int t = 0; t < job.nt; ++t) {
        const uint32_t a_addr = base;  // A tile: first 128 rows (separate A, or the B tile bi == bj0)
        const uint32_t b_addr = base + static_cast<uint32_t>((rowsA + t * 128) * 128);
#pragma unroll
        for (int k4 = 0; k4 < 4; ++k4) {
          umma_f16(tmem + static_cast<uint32_t>(t * 128), sdesc_sw128(a_addr + k4 * 32),
                   sdesc_sw128(b_addr + k4 * 32), idesc, (c > 0 || k4 > 0) ? 1u : 0u);
        }
      }
      umma_commit(&bars[b]);
    }
  }

  // wait for the last two commits: the last one covers every MMA issued
  // before it, and waiting for both leaves no arrive pending on either barrier
  if (!failed && nchunks > 0) {
    bool ok = true;
    for (int64_t last = nchunks - 1; last >= 0 && last >= nchunks - 2; --last)
      ok = ok && mbar_wait_bounded(&bars[last & 1], static_cast<uint32_t>((last >> 1) & 1), kMaxSpins);
    if (__syncthreads_or(!ok)) failed = true;
  }
  if (failed && tid == 0) atomicAdd(p.err, 1u);
  tc_fence_after();

  // epilogue: warp w reads TMEM lanes 32*(w%4) .. +31; the four warps of a
  // lane quarter split the columns
  float* out = p.out + static_cast<int64_t>(blockIdx.x) * 128 * 512;
  const int sub = warp & 3;
  const int quarter = warp >> 2;  // 0..3
  const int used = job.nt * 128;
  const int row_local = sub * 32 + lane;
  for (int c0 = quarter * 32; c0 < used; c0 += 128) {
    float r[32];
    if (nchunks > 0 && !failed) {
      tmem_ld32(tmem + (static_cast<uint32_t>(sub * 32) << 16) + static_cast<uint32_t>(c0), r);
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i) r[i] = 0.f;
    }
    float4* dst = reinterpret_cast<float4*>(out + row_local * 512 + c0);
#pragma unroll
    for (int i = 0; i < 8; ++i) dst[i] = make_float4(r[4 * i], r[4 * i + 1], r[4 * i + 2], r[4 * i + 3]);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, ncols);
  }
}

// Fixed-order FP64 reduction of the slices of each item into G (upper
// triangle computed, mirrored into the lower one).
__global__ void reduce_tc(const float* __restrict__ part, const TcCta* __restrict__ ctas, int stride,
                          const int* __restrict__ item_first, const int* __restrict__ item_count, int K,
                          double* __restrict__ G) {
  const int item = blockIdx.y;
  const int first = item_first[item], count = item_count[item];
  const TcCta job = ctas[first];
  const int used = job.nt * 128;
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= static_cast<int64_t>(128) * used) return;
  const int rl = static_cast<int>(e / used), cl = static_cast<int>(e % used);
  double s = 0.0;
  for (int i = 0; i < count; ++i)
    s += part[static_cast<int64_t>(first + i * stride) * 128 * 512 + rl * 512 + cl];
  const int row = job.bi * 128 + rl;
  const int col = job.bj0 * 128 + cl;
  if (row >= K || col >= K) return;
  if (job.bi == job.bj0 && cl < 128 && col < row) return;  // diagonal tile: keep one of each pair
  G[static_cast<int64_t>(row) * K + col] = s;
  G[static_cast<int64_t>(col) * K + row] = s;
}

struct TcPlan {
  std::vector<TcCta> ctas;
  std::vector<int> first, count;  // CTAs of item i: first[i] + j * stride, j < count[i]
  int stride = 1;
};

TcPlan tc_plan(int64_t K, int64_t n) {
  TcPlan pl;
  const int MT = static_cast<int>(ceil_div(K, 128));
  struct Item { int bi, bj0, nt; };
  std::vector<Item> items;
  for (int bi = 0; bi < MT; ++bi)
    for (int bj0 = bi; bj0 < MT; bj0 += 4) items.push_back({bi, bj0, std::min(4, MT - bj0)});
  const int W = static_cast<int>(items.size());
  // equal slices for every item, CTAs ordered slice-major so the CTAs that
  // read the same columns of v run together and share them through L2;
  // about four CTAs per SM even out the unequal item sizes
  const int64_t nch = ceil_div(n, kChunkCols);
  int64_t S = std::max<int64_t>(1, (4 * static_cast<int64_t>(num_sms()) + W - 1) / W);
  S = std::min<int64_t>(S, std::max<int64_t>(1, kMaxCtas / W));
  S = std::min<int64_t>(S, nch);
  const int64_t per = ceil_div(nch, S) * kChunkCols;
  S = ceil_div(n, per);
  pl.first.assign(W, 0);
  pl.count.assign(W, 0);
  // item i's CTAs are i, i + W, i + 2W, ... : record them as a strided run
  for (int64_t sl = 0; sl < S; ++sl)
    for (int i = 0; i < W; ++i) {
      const int64_t c0 = sl * per;
      pl.ctas.push_back({i, items[i].bi, items[i].bj0, items[i].nt, c0, std::min<int64_t>(n, c0 + per)});
    }
  for (int i = 0; i < W; ++i) {
    pl.first[i] = i;
    pl.count[i] = static_cast<int>(S);
  }
  pl.stride = W;
  return pl;
}

template <typename T>
size_t tc_smem() {
  return 2 * static_cast<size_t>(kStageBytes) + kMaxRows * sizeof(float) + 64 + 1024;
}

}  // namespace

size_t overlap_tc_tmp_bytes(int64_t K, int64_t n) {
  const TcPlan pl = tc_plan(K, n);
  const size_t nc = pl.ctas.size(), ni = pl.first.size();
  return round_up(static_cast<int64_t>(nc) * 128 * 512 * 4, 256) + round_up(nc * sizeof(TcCta), 256) +
         round_up(2 * ni * sizeof(int), 256) + 256;
}

mbar_status overlap_tc(const void* v, int dtype_bytes, int64_t K, int64_t n, int64_t ld, const double* a,
                       const void* logden, const int32_t* H, double* G, unsigned* err, void* tmp, size_t tmp_bytes,
                       cudaStream_t st) {
  const TcPlan pl = tc_plan(K, n);
  if (tmp_bytes < overlap_tc_tmp_bytes(K, n)) {
    set_error("overlap_tc: scratch too small");
    return MBAR_EINVAL;
  }
  const int nc = static_cast<int>(pl.ctas.size()), ni = static_cast<int>(pl.first.size());
  unsigned char* q = static_cast<unsigned char*>(tmp);
  float* part = reinterpret_cast<float*>(q);
  q += round_up(static_cast<int64_t>(nc) * 128 * 512 * 4, 256);
  TcCta* ctas_d = reinterpret_cast<TcCta*>(q);
  q += round_up(nc * sizeof(TcCta), 256);
  int* first_d = reinterpret_cast<int*>(q);
  int* count_d = first_d + ni;
  std::vector<int> fc(pl.first);
  fc.insert(fc.end(), pl.count.begin(), pl.count.end());
  BUMBAR_CUDA(cudaMemcpyAsync(ctas_d, pl.ctas.data(), nc * sizeof(TcCta), cudaMemcpyHostToDevice, st));
  BUMBAR_CUDA(cudaMemcpyAsync(first_d, fc.data(), fc.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  BUMBAR_CUDA(cudaMemsetAsync(G, 0, static_cast<size_t>(K) * K * sizeof(double), st));
  TcParams prm{};
  prm.v = v;
  prm.ld = ld;
  prm.K = static_cast<int>(K);
  prm.n = n;
  prm.a = a;
  prm.logden = logden;
  prm.H = H;
  prm.ctas = ctas_d;
  prm.out = part;
  prm.err = err;
  const size_t smem = dtype_bytes == 4 ? tc_smem<float>() : tc_smem<double>();
  if (dtype_bytes == 4) {
    static bool attr = false;
    if (!attr) {
      BUMBAR_CUDA(cudaFuncSetAttribute(overlap_tc_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem)));
      attr = true;
    }
    overlap_tc_kernel<float><<<nc, kTcThreads, smem, st>>>(prm);
  } else {
    static bool attr = false;
    if (!attr) {
      BUMBAR_CUDA(cudaFuncSetAttribute(overlap_tc_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem)));
      attr = true;
    }
    overlap_tc_kernel<double><<<nc, kTcThreads, smem, st>>>(prm);
  }
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  const unsigned gx = static_cast<unsigned>(ceil_div(128 * 512, 256));
  reduce_tc<<<dim3(gx, ni), 256, 0, st>>>(part, ctas_d, pl.stride, first_d, count_d, static_cast<int>(K), G);
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

}  // namespace bumbar
