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
#ifndef TC_ROWS_PER_ROUND
#define TC_ROWS_PER_ROUND 4
#endif

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

  // Each thread handles rows rsub + kRowStride * m, m = 0, 1, ..., in rounds
  // of kRowsPerRound rows; the loads of the next round (next chunk after
  // the last round) are issued before the exponentials of the current one.
  constexpr int kRowsPerRound = TC_ROWS_PER_ROUND;
  const int nrounds = (rows + kRowStride * kRowsPerRound - 1) / (kRowStride * kRowsPerRound);
  auto load_cols = [&](int64_t c, float* l2, float* sh) {
    const int64_t col0 = job.c_begin + c * kChunkCols + g * 8;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t col = col0 + j;
      if (col < job.c_end) {
        l2[j] = static_cast<float>(ld_in[col]) * kLog2e;
        sh[j] = p.H ? sqrtf(static_cast<float>(p.H[col])) : 1.f;
      } else {
        l2[j] = INFINITY;  // exp2(-inf) = 0: padding samples contribute nothing
        sh[j] = 0.f;
      }
    }
  };
  auto load_round = [&](int64_t c, int r, float (*x)[8]) {
    const int64_t col0 = job.c_begin + c * kChunkCols + g * 8;
    const bool full8 = col0 + 8 <= job.c_end;
#pragma unroll
    for (int u = 0; u < kRowsPerRound; ++u) {
      const int lr = rsub + kRowStride * (r * kRowsPerRound + u);
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
  };

  float xn[kRowsPerRound][8], l2n[8], shn[8];
  if (nchunks > 0) {
    load_cols(0, l2n, shn);
    load_round(0, 0, xn);
  }
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
    float l2[8], sh[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      l2[j] = l2n[j];
      sh[j] = shn[j];
    }
    for (int r = 0; r < nrounds; ++r) {
      float x[kRowsPerRound][8];
#pragma unroll
      for (int u = 0; u < kRowsPerRound; ++u)
#pragma unroll
        for (int j = 0; j < 8; ++j) x[u][j] = xn[u][j];
      if (r + 1 < nrounds) {
        load_round(c, r + 1, xn);
      } else if (c + 1 < nchunks) {
        load_cols(c + 1, l2n, shn);
        load_round(c + 1, 0, xn);
      }
#pragma unroll
      for (int u = 0; u < kRowsPerRound; ++u) {
        const int lr = rsub + kRowStride * (r * kRowsPerRound + u);
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

// ---------------------------------------------------------------------------
// Cluster variant for K <= 512 (FP32 data): one cluster of MT = ceil(K/128)
// CTAs per slice of samples. CTA r of a cluster builds P~ only for its own
// 128-row tile r -- every exponential is evaluated once -- and stores the
// FP16 tile into its own shared memory and into the shared memory of the
// peer CTAs that use it as a B operand (distributed shared memory). CTA r
// accumulates the tiles (r, (r + d) mod MT), d = 0 .. dmax(r), which cover
// the upper triangle of G exactly once (a circulant assignment: at most
// three 128 x 128 FP32 accumulators per CTA, within the 512 TMEM columns).
//
// Three roles per CTA, coupled only by mbarriers (no CTA-wide barrier in
// the chunk loop):
//   * a loader warp streams the CTA's 128 x 64 FP32 blocks of v into a
//     two-stage ring by TMA (vfull), refilling a stage once every producer
//     warp has read it (vempty);
//   * 16 producer warps: per 64-sample chunk each thread waits for its v
//     block and for the P~ stage to be free (pempty: every reader of the
//     tile finished its MMAs on the stage's previous chunk), forms P~ for
//     two rows and eight samples and stores the FP16 pieces to this CTA and
//     its readers. The proxy fence that makes those stores visible to the
//     tensor cores, and the per-warp arrivals on the readers' pfull
//     barriers, are issued one chunk later, after the next chunk's
//     exponentials: by then the remote stores have drained and the fence
//     does not stall;
//   * an MMA warp waits until every writer's warps have delivered a chunk
//     (pfull), issues the UMMAs and commits them to the writers' pempty.
// Every wait is bounded; a CTA that gives up records an error and still
// reaches the final cluster barrier.
constexpr int kClThreads = 512;                // threads that build P~ (16 warps)
constexpr int kClWarps = kClThreads / 32;
constexpr int kClThreadsAll = kClThreads + 64;  // + the MMA warp + the loader warp
constexpr int kClVStages = 2;
constexpr int kClPStages = 3;                 // P~ stages (chunks in flight between producers and MMAs)
constexpr int kClVStageBytes = 128 * 64 * 4;  // two 32-column 128B-swizzled boxes
constexpr int kClPSlots = 3;
constexpr int kClPSlotBytes = 128 * 128;      // one FP16 128 x 64 tile
constexpr int kClPStageBytes = kClPSlots * kClPSlotBytes;
constexpr int kClMaxTiles = 4;                // MT <= 4, i.e. K <= 512
constexpr int kClMaxFactTiles = 8;            // factorised form: MT <= 8 (K <= 1024) in distance windows
constexpr int kClWindow = 3;                  // tile distances per launch of the factorised kernel

__host__ __device__ inline int cl_dmax(int q, int MT) {
  return (MT - 1) / 2 + ((MT % 2 == 0 && q < MT / 2) ? 1 : 0);
}
__host__ __device__ inline int cl_tile_base(int q, int MT) {
  int t = 0;
  for (int i = 0; i < q; ++i) t += cl_dmax(i, MT) + 1;
  return t;
}

struct ClParams {
  int K;
  int MT;
  int T;          // accumulator tiles per cluster
  int64_t n;
  int64_t per;    // samples per slice (multiple of 64)
  const double* a;
  const float* logden;
  const int32_t* H;
  float* out;     // [slices][T][128][128]
  unsigned* err;
  int dlo;        // factorised kernel: this launch forms the tiles at distances dlo .. dlo + kClWindow - 1
};

__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t mapa_shared(uint32_t addr, uint32_t rank) {
  uint32_t o;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(o) : "r"(addr), "r"(rank));
  return o;
}
__device__ __forceinline__ void st_cluster_v4(uint32_t addr, uint4 v) {
  asm volatile("st.shared::cluster.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z),
               "r"(v.w)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Waits bounded in time as well as in polls: gives up after about one second
// (every legitimate wait of this kernel lasts microseconds).
constexpr uint64_t kClWaitNs = 1000000000ull;
__device__ __forceinline__ bool mbar_wait_cluster_bounded(uint64_t* bar, uint32_t parity, uint32_t max_spins) {
  const uint64_t t0 = global_ns();
  for (uint32_t i = 0; i < max_spins; ++i) {
    if (mbar_try_wait_cluster(bar, parity)) return true;
    if ((i & 255u) == 255u && global_ns() - t0 > kClWaitNs) return false;
  }
  return false;
}
__device__ __forceinline__ bool mbar_wait_timed(uint64_t* bar, uint32_t parity, uint32_t max_spins) {
  const uint64_t t0 = global_ns();
  for (uint32_t i = 0; i < max_spins; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255u) == 255u && global_ns() - t0 > kClWaitNs) return false;
  }
  return false;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// generic-proxy writes to shared memory (this CTA's and the cluster peers')
// made visible to the async proxy (the tensor cores' operand reads)
__device__ __forceinline__ void fence_proxy_async_smem_cluster() {
  asm volatile("fence.proxy.async.shared::cluster;" ::: "memory");
}
__device__ __forceinline__ void umma_commit_multicast(uint64_t* bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"(mask)
      : "memory");
}

__global__ void __launch_bounds__(kClThreadsAll, 1)
    overlap_tc_cluster_kernel(const __grid_constant__ CUtensorMap tmap, ClParams p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  unsigned char* vbuf = smem;
  unsigned char* pbuf = smem + kClVStages * kClVStageBytes;
  uint64_t* vfull = reinterpret_cast<uint64_t*>(pbuf + kClPStages * kClPStageBytes);  // [kClVStages]
  uint64_t* vempty = vfull + kClVStages;                                                // [kClVStages]
  uint64_t* pfull = vempty + kClVStages;                                                // [kClPStages]
  uint64_t* pempty = pfull + kClPStages;                                                // [kClPStages]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(pempty + kClPStages);
  volatile int* fail_s = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* issued_s = reinterpret_cast<int*>(tmem_slot + 2);  // v chunks the loader sent

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const bool producer = tid < kClThreads;
  const bool mma_warp = warp == kClWarps;
  const bool loader_warp = warp == kClWarps + 1;
  const int MT = p.MT;
  const int r = static_cast<int>(cluster_ctarank());
  const int64_t slice = blockIdx.x / MT;
  const int dm = cl_dmax(r, MT);
  const int ntl = dm + 1;
  const uint32_t ncols = ntl == 1 ? 128u : (ntl == 2 ? 256u : 512u);
  // readers of tile r: CTAs q that use it (slot (r - q) mod MT there)
  uint32_t reader_mask = 0;
  for (int q = 0; q < MT; ++q)
    if ((r - q + MT) % MT <= cl_dmax(q, MT)) reader_mask |= 1u << q;
  const int nreaders = __popc(reader_mask);
  uint16_t writer_mask = 0;  // CTAs whose tiles this CTA uses
  for (int d = 0; d <= dm; ++d) writer_mask |= static_cast<uint16_t>(1u << ((r + d) % MT));
  const int64_t c_begin = slice * p.per;
  const int64_t c_end = (c_begin + p.per < p.n) ? c_begin + p.per : p.n;
  const int64_t nchunks = c_end > c_begin ? (c_end - c_begin + 63) / 64 : 0;

  if (warp == 0) tmem_alloc(tmem_slot, ncols);
  if (tid == 0) {
    for (int s = 0; s < kClVStages; ++s) {
      mbar_init(&vfull[s], 1);
      mbar_init(&vempty[s], kClWarps);
    }
    for (int b = 0; b < kClPStages; ++b) {
      mbar_init(&pfull[b], static_cast<uint32_t>((dm + 1) * kClWarps));
      mbar_init(&pempty[b], static_cast<uint32_t>(nreaders));
    }
    *fail_s = 0;
    *issued_s = 0;
    fence_barrier_init();
    prefetch_tmap(&tmap);
  }
  // this thread's rows (lr0, lr0 + 64) of tile r and 8-sample group g
  const int g = tid & 7;
  const int lr0 = (tid >> 3) & 63;
  float a2r[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int row = r * 128 + lr0 + 64 * u;
    a2r[u] = (producer && row < p.K) ? static_cast<float>(p.a[row] * 1.4426950408889634) : -INFINITY;
  }
  tc_fence_before();
  cluster_sync_all();  // barrier initialisation visible to the peers
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  constexpr uint32_t idesc = idesc_f16(128, 128);

  if (producer) {
    // per-sample log2(e) logden and sqrt(H) of this thread's 8 samples,
    // loaded one chunk ahead (padding samples: 2^-inf = 0)
    float l2n[8], shn[8];
    auto load_cols = [&](int64_t cc) {
      const int64_t col0 = c_begin + cc * 64 + g * 8;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        l2n[j] = INFINITY;
        shn[j] = 0.f;
      }
      if (col0 + 8 <= c_end) {
        const float4 d0 = *reinterpret_cast<const float4*>(p.logden + col0);
        const float4 d1 = *reinterpret_cast<const float4*>(p.logden + col0 + 4);
        const float dd[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          l2n[j] = dd[j] * kLog2e;
          shn[j] = p.H ? sqrtf(static_cast<float>(p.H[col0 + j])) : 1.f;
        }
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (col0 + j < c_end) {
            l2n[j] = p.logden[col0 + j] * kLog2e;
            shn[j] = p.H ? sqrtf(static_cast<float>(p.H[col0 + j])) : 1.f;
          }
      }
    };
    // readers' pfull barriers of stage b: arrive once per warp, after the
    // proxy fence that covers this thread's earlier P~ stores
    auto deliver = [&](int b) {
      fence_proxy_async_smem_cluster();
      __syncwarp();
      if (lane == 0)
        for (int q = 0; q < MT; ++q)
          if (reader_mask & (1u << q)) mbar_arrive_cluster(mapa_shared(smem_u32(&pfull[b]), static_cast<uint32_t>(q)));
    };
    if (nchunks > 0) load_cols(0);
    bool failed = false;
    int64_t c = 0;
    for (; c < nchunks; ++c) {
      const int s = static_cast<int>(c % kClVStages);
      const int b = static_cast<int>(c % kClPStages);
      bool ok = mbar_wait_timed(&vfull[s], static_cast<uint32_t>((c / kClVStages) & 1), kMaxSpins);
      float x[2][8];
      if (ok) {
        const unsigned char* vb = vbuf + s * kClVStageBytes + (g >> 2) * (kClVStageBytes / 2);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int lr = lr0 + 64 * u;
          const float4 x0 = *reinterpret_cast<const float4*>(vb + swz128(lr, (g & 3) * 2));
          const float4 x1 = *reinterpret_cast<const float4*>(vb + swz128(lr, (g & 3) * 2 + 1));
          x[u][0] = x0.x; x[u][1] = x0.y; x[u][2] = x0.z; x[u][3] = x0.w;
          x[u][4] = x1.x; x[u][5] = x1.y; x[u][6] = x1.z; x[u][7] = x1.w;
        }
      }
      if (__all_sync(0xffffffffu, ok)) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&vempty[s]);  // this warp is done with the v stage
      }
      if (ok && c >= kClPStages) {
        // the stage's previous chunk is consumed by every reader: one lane
        // polls, the warp follows
        if (lane == 0)
          ok = mbar_wait_cluster_bounded(&pempty[b], static_cast<uint32_t>(((c - kClPStages) / kClPStages) & 1),
                                         kMaxSpins);
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      }
      if (!__all_sync(0xffffffffu, ok && *fail_s == 0)) {
        if (lane == 0) *fail_s = 1;
        failed = true;
        break;
      }
      float l2[8], sh[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        l2[j] = l2n[j];
        sh[j] = shn[j];
      }
      uint4 packed[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        float pv[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) pv[j] = ex2_approx(fmaf(-x[u][j], kLog2e, a2r[u]) - l2[j]) * sh[j];
        packed[u].x = pack_half2(pv[0], pv[1]);
        packed[u].y = pack_half2(pv[2], pv[3]);
        packed[u].z = pack_half2(pv[4], pv[5]);
        packed[u].w = pack_half2(pv[6], pv[7]);
      }
      if (c > 0) deliver(static_cast<int>((c - 1) % kClPStages));  // the previous chunk's stores
      unsigned char* pst = pbuf + b * kClPStageBytes;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int lr = lr0 + 64 * u;
        const uint32_t off = static_cast<uint32_t>(lr * 128 + ((g ^ (lr & 7)) << 4));
#pragma unroll
        for (int q = 0; q < kClMaxTiles; ++q) {
          if (reader_mask & (1u << q)) {
            const int slot = (r - q + MT) % MT;
            if (q == r)
              *reinterpret_cast<uint4*>(pst + off) = packed[u];  // own tile: slot 0
            else
              st_cluster_v4(mapa_shared(smem_u32(pst + slot * kClPSlotBytes) + off, static_cast<uint32_t>(q)),
                            packed[u]);
          }
        }
      }
      // the next chunk's per-sample columns, issued after the fence above
      // (a proxy fence also waits for this thread's loads in flight)
      if (c + 1 < nchunks) load_cols(c + 1);
    }
    if (!failed && nchunks > 0) deliver(static_cast<int>((nchunks - 1) % kClPStages));
  } else if (mma_warp) {
    // waits until every writer has delivered chunk c, issues the UMMAs and
    // commits them to the writers' pempty barriers
    for (int64_t cm = 0; cm < nchunks; ++cm) {
      const int b = static_cast<int>(cm % kClPStages);
      bool ok = true;
      if (lane == 0)
        ok = mbar_wait_cluster_bounded(&pfull[b], static_cast<uint32_t>((cm / kClPStages) & 1), kMaxSpins);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok || *fail_s) {
        if (lane == 0) *fail_s = 1;
        break;
      }
      if (lane == 0) {
        tc_fence_after();
        const uint32_t base = smem_u32(pbuf + b * kClPStageBytes);
        for (int t = 0; t < ntl; ++t) {
#pragma unroll
          for (int k4 = 0; k4 < 4; ++k4)
            umma_f16(tmem + static_cast<uint32_t>(t * 128), sdesc_sw128(base + k4 * 32),
                     sdesc_sw128(base + static_cast<uint32_t>(t * kClPSlotBytes) + k4 * 32), idesc,
                     (cm > 0 || k4 > 0) ? 1u : 0u);
        }
        umma_commit_multicast(&pempty[b], writer_mask);
      }
      __syncwarp();
    }
  } else if (loader_warp && lane == 0) {
    // the CTA's v blocks, each stage refilled once every producer warp read it
    int64_t issued = 0;
    for (int64_t c = 0; c < nchunks; ++c) {
      const int s = static_cast<int>(c % kClVStages);
      if (c >= kClVStages &&
          !mbar_wait_timed(&vempty[s], static_cast<uint32_t>(((c - kClVStages) / kClVStages) & 1), kMaxSpins)) {
        *fail_s = 1;
        break;
      }
      if (*fail_s) break;
      unsigned char* dst = vbuf + s * kClVStageBytes;
      const int col = static_cast<int>(c_begin + c * 64);
      mbar_expect_tx(&vfull[s], kClVStageBytes);
      tma_load_2d(dst, &tmap, &vfull[s], col, r * 128);
      tma_load_2d(dst + kClVStageBytes / 2, &tmap, &vfull[s], col + 32, r * 128);
      ++issued;
    }
    *issued_s = static_cast<int>(issued);
  }
  __syncthreads();
  bool failed = *fail_s != 0;
  if (!failed && nchunks > 0) {
    // the last commits of every reader of this tile (they include this CTA's)
    bool ok = true;
    for (int64_t last = nchunks - 1; last >= 0 && last >= nchunks - kClPStages; --last)
      ok = ok && mbar_wait_cluster_bounded(&pempty[last % kClPStages], static_cast<uint32_t>((last / kClPStages) & 1),
                                           kMaxSpins);
    if (__syncthreads_or(!ok)) failed = true;
  }
  if (failed) {
    // let this CTA's own tensor copies in flight land before leaving (at
    // most one outstanding per v stage: the last kClVStages issued)
    if (tid == 0) {
      const int64_t iss = *issued_s;
      for (int64_t cc = (iss > kClVStages ? iss - kClVStages : 0); cc < iss; ++cc)
        mbar_wait_timed(&vfull[cc % kClVStages], static_cast<uint32_t>((cc / kClVStages) & 1), kMaxSpins);
      atomicAdd(p.err, 1u);
    }
  }
  tc_fence_after();

  // epilogue: warp w reads TMEM lanes 32*(w%4) .. +31, the four warps of a
  // lane quarter split the columns
  float* out = p.out + (slice * p.T + cl_tile_base(r, MT)) * 128 * 128;
  const int sub = warp & 3;
  const int quarter = warp >> 2;
  const int row_local = sub * 32 + lane;
  for (int c0 = quarter * 32; producer && c0 < ntl * 128; c0 += 128) {
    float rr[32];
    if (nchunks > 0 && !failed) {
      tmem_ld32(tmem + (static_cast<uint32_t>(sub * 32) << 16) + static_cast<uint32_t>(c0), rr);
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i) rr[i] = 0.f;
    }
    float4* dst = reinterpret_cast<float4*>(out + (c0 >> 7) * 128 * 128 + row_local * 128 + (c0 & 127));
#pragma unroll
    for (int i = 0; i < 8; ++i) dst[i] = make_float4(rr[4 * i], rr[4 * i + 1], rr[4 * i + 2], rr[4 * i + 3]);
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // no peer touches this CTA's shared memory after this point
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, ncols);
  }
}

// ---------------------------------------------------------------------------
// The same cluster contraction for unbinned FP32 data read from the
// sample-major copy vst[n][Kp] (MIXED contexts keep it for their LSE
// passes), logden in that sample order, no counts.
//
// A generic-proxy write of UMMA operands must be followed by a proxy fence
// before the tensor cores read it, and that fence is expensive (about 1,700
// cycles per warp measured on B300, whatever is outstanding), so each fence
// here covers a whole 32-state x 64-sample block per warp. The 16 producer
// warps form four groups; group q builds the chunks c = q (mod 4) into P~
// stage c mod 4 (four stages), warp w of a group the 32 states 32 w + lane of
// the CTA's tile for all 64 samples: it loads their v straight from the
// sample-major copy (a warp load is 128 contiguous bytes of one sample; the
// first 32 samples of a chunk are loaded during the group's previous chunk),
// forms P~, stores the eight 16-byte pieces of its row to this CTA and the
// tile's readers, fences once and arrives on the readers' pfull barriers.
// While one group loads or fences, the other three compute. The MMA warp
// consumes the chunks in order.
constexpr int kSmjGroups = 4;
constexpr int kSmjPStages = kSmjGroups;
constexpr int kSmjThreadsAll = kClThreads + 32;  // 16 producer warps + the MMA warp

__global__ void __launch_bounds__(kSmjThreadsAll, 1)
    overlap_tc_smaj_kernel(const float* __restrict__ vst, int Kp, ClParams p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  unsigned char* pbuf = smem;
  uint64_t* pfull = reinterpret_cast<uint64_t*>(pbuf + kSmjPStages * kClPStageBytes);  // [kSmjPStages]
  uint64_t* pempty = pfull + kSmjPStages;                                              // [kSmjPStages]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(pempty + kSmjPStages);
  volatile int* fail_s = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const bool producer = tid < kClThreads;
  const int MT = p.MT;
  const int r = static_cast<int>(cluster_ctarank());
  const int64_t slice = blockIdx.x / MT;
  const int dm = cl_dmax(r, MT);
  const int ntl = dm + 1;
  const uint32_t ncols = ntl == 1 ? 128u : (ntl == 2 ? 256u : 512u);
  uint32_t reader_mask = 0;
  for (int q = 0; q < MT; ++q)
    if ((r - q + MT) % MT <= cl_dmax(q, MT)) reader_mask |= 1u << q;
  const int nreaders = __popc(reader_mask);
  uint16_t writer_mask = 0;
  for (int d = 0; d <= dm; ++d) writer_mask |= static_cast<uint16_t>(1u << ((r + d) % MT));
  const int64_t c_begin = slice * p.per;
  const int64_t c_end = (c_begin + p.per < p.n) ? c_begin + p.per : p.n;
  const int64_t nchunks = c_end > c_begin ? (c_end - c_begin + 63) / 64 : 0;

  if (warp == 0) tmem_alloc(tmem_slot, ncols);
  if (tid == 0) {
    for (int b = 0; b < kSmjPStages; ++b) {
      // one chunk is delivered by the four warps of one group of each writer
      mbar_init(&pfull[b], static_cast<uint32_t>((dm + 1) * (kClWarps / kSmjGroups)));
      mbar_init(&pempty[b], static_cast<uint32_t>(nreaders));
    }
    *fail_s = 0;
    fence_barrier_init();
  }
  const int grp = warp / (kClWarps / kSmjGroups);   // chunk group
  const int lr = 32 * (warp % (kClWarps / kSmjGroups)) + lane;   // row (state) of tile r
  const int row = r * 128 + lr;
  const float a2 = (producer && row < p.K) ? static_cast<float>(p.a[row] * 1.4426950408889634) : -INFINITY;
  const bool row_stored = row < Kp;   // states K..Kp-1 are zero padding of the copy; beyond Kp nothing is read
  tc_fence_before();
  cluster_sync_all();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  constexpr uint32_t idesc = idesc_f16(128, 128);

  if (producer) {
    // v of samples [32 h, 32 h + 32) of chunk cc at this thread's state, and
    // log2(e) logden of samples lane and lane + 32 (padding: x = 0, +inf)
    auto load_half = [&](int64_t cc, int h, float* dst) {
      const int64_t s0 = c_begin + cc * 64;
      const int ns = static_cast<int>(c_end - s0 < 64 ? c_end - s0 : 64);
      const float* src = vst + (s0 + 32 * h) * Kp + row;
#pragma unroll
      for (int j = 0; j < 32; ++j)
        dst[j] = (row_stored && 32 * h + j < ns) ? src[static_cast<int64_t>(j) * Kp] : 0.f;
    };
    auto load_l2 = [&](int64_t cc, float& la, float& lb) {
      const int64_t s0 = c_begin + cc * 64;
      const int ns = static_cast<int>(c_end - s0 < 64 ? c_end - s0 : 64);
      la = lane < ns ? p.logden[s0 + lane] * kLog2e : INFINITY;
      lb = lane + 32 < ns ? p.logden[s0 + lane + 32] * kLog2e : INFINITY;
    };
    // the first half of each chunk is loaded during the previous chunk of
    // the group (after its fence: a proxy fence also waits for this
    // thread's loads in flight), the second half at the chunk's start
    float xa[32], xb[32], l2a = INFINITY, l2b = INFINITY;
    if (grp < nchunks) {
      load_half(grp, 0, xa);
      load_l2(grp, l2a, l2b);
    }
    for (int64_t c = grp; c < nchunks; c += kSmjGroups) {
      const int b = static_cast<int>(c % kSmjPStages);
      bool ok = true;
      if (c >= kSmjPStages) {
        if (lane == 0)
          ok = mbar_wait_cluster_bounded(&pempty[b], static_cast<uint32_t>(((c - kSmjPStages) / kSmjPStages) & 1),
                                         kMaxSpins);
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      }
      if (!__all_sync(0xffffffffu, ok && *fail_s == 0)) {
        if (lane == 0) *fail_s = 1;
        break;
      }
      load_half(c, 1, xb);
      unsigned char* pst = pbuf + b * kClPStageBytes;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        float pv[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int sj = 8 * k + j;
          const float l2 = __shfl_sync(0xffffffffu, sj < 32 ? l2a : l2b, sj & 31);
          pv[j] = ex2_approx(fmaf(-(sj < 32 ? xa[sj] : xb[sj - 32]), kLog2e, a2) - l2);
        }
        uint4 packed;
        packed.x = pack_half2(pv[0], pv[1]);
        packed.y = pack_half2(pv[2], pv[3]);
        packed.z = pack_half2(pv[4], pv[5]);
        packed.w = pack_half2(pv[6], pv[7]);
        const uint32_t off = static_cast<uint32_t>(lr * 128 + ((k ^ (lr & 7)) << 4));
#pragma unroll
        for (int q = 0; q < kClMaxTiles; ++q) {
          if (reader_mask & (1u << q)) {
            const int slot = (r - q + MT) % MT;
            if (q == r)
              *reinterpret_cast<uint4*>(pst + off) = packed;
            else
              st_cluster_v4(mapa_shared(smem_u32(pst + slot * kClPSlotBytes) + off, static_cast<uint32_t>(q)), packed);
          }
        }
      }
      fence_proxy_async_smem_cluster();
      __syncwarp();
      if (lane == 0)
        for (int q = 0; q < MT; ++q)
          if (reader_mask & (1u << q)) mbar_arrive_cluster(mapa_shared(smem_u32(&pfull[b]), static_cast<uint32_t>(q)));
      if (c + kSmjGroups < nchunks) {
        load_half(c + kSmjGroups, 0, xa);
        load_l2(c + kSmjGroups, l2a, l2b);
      }
    }
  } else {
    for (int64_t cm = 0; cm < nchunks; ++cm) {
      const int b = static_cast<int>(cm % kSmjPStages);
      bool ok = true;
      if (lane == 0)
        ok = mbar_wait_cluster_bounded(&pfull[b], static_cast<uint32_t>((cm / kSmjPStages) & 1), kMaxSpins);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok || *fail_s) {
        if (lane == 0) *fail_s = 1;
        break;
      }
      if (lane == 0) {
        tc_fence_after();
        const uint32_t base = smem_u32(pbuf + b * kClPStageBytes);
        for (int t = 0; t < ntl; ++t) {
#pragma unroll
          for (int k4 = 0; k4 < 4; ++k4)
            umma_f16(tmem + static_cast<uint32_t>(t * 128), sdesc_sw128(base + k4 * 32),
                     sdesc_sw128(base + static_cast<uint32_t>(t * kClPSlotBytes) + k4 * 32), idesc,
                     (cm > 0 || k4 > 0) ? 1u : 0u);
        }
        umma_commit_multicast(&pempty[b], writer_mask);
      }
      __syncwarp();
    }
  }
  __syncthreads();
  bool failed = *fail_s != 0;
  if (!failed && nchunks > 0) {
    bool ok = true;
    for (int64_t last = nchunks - 1; last >= 0 && last >= nchunks - kSmjPStages; --last)
      ok = ok && mbar_wait_cluster_bounded(&pempty[last % kSmjPStages],
                                           static_cast<uint32_t>((last / kSmjPStages) & 1), kMaxSpins);
    if (__syncthreads_or(!ok)) failed = true;
  }
  if (failed && tid == 0) atomicAdd(p.err, 1u);
  tc_fence_after();
  float* out = p.out + (slice * p.T + cl_tile_base(r, MT)) * 128 * 128;
  const int sub = warp & 3;
  const int quarter = warp >> 2;
  const int row_local = sub * 32 + lane;
  for (int c0 = quarter * 32; producer && c0 < ntl * 128; c0 += 128) {
    float rr[32];
    if (nchunks > 0 && !failed) {
      tmem_ld32(tmem + (static_cast<uint32_t>(sub * 32) << 16) + static_cast<uint32_t>(c0), rr);
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i) rr[i] = 0.f;
    }
    float4* dst = reinterpret_cast<float4*>(out + (c0 >> 7) * 128 * 128 + row_local * 128 + (c0 & 127));
#pragma unroll
    for (int i = 0; i < 8; ++i) dst[i] = make_float4(rr[4 * i], rr[4 * i + 1], rr[4 * i + 2], rr[4 * i + 3]);
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, ncols);
  }
}

// The same contraction for a factorised context (u_ip = a_i + b_i phi_p, no
// K x N store): P~ is formed from a, b, phi and the pass's FP64 logden (all
// in the original sample order); the exponent is FP32 at the magnitude of
// the cancelling terms (~1e-4 absolute on tempering energies), below the
// FP16 rounding of P~.
__global__ void __launch_bounds__(kSmjThreadsAll, 1)
    overlap_tc_fact_kernel(const double* __restrict__ fa, const double* __restrict__ fb,
                           const double* __restrict__ fphi, const double* __restrict__ logden, ClParams p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  unsigned char* pbuf = smem;
  uint64_t* pfull = reinterpret_cast<uint64_t*>(pbuf + kSmjPStages * kClPStageBytes);  // [kSmjPStages]
  uint64_t* pempty = pfull + kSmjPStages;                                              // [kSmjPStages]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(pempty + kSmjPStages);
  volatile int* fail_s = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const bool producer = tid < kClThreads;
  const int MT = p.MT;
  const int r = static_cast<int>(cluster_ctarank());
  const int64_t slice = blockIdx.x / MT;
  // This launch forms the tiles (q, q + d) with dlo <= d < dlo + kClWindow
  // and d <= cl_dmax(q): at most three per CTA, so the accumulators fit one
  // 512-column TMEM allocation at any MT <= 8. Slot 0 of a P~ stage holds the
  // CTA's own tile (the A operand); with dlo > 0 the window's B tiles follow
  // in slots 1 .. 2, with dlo = 0 tile d sits in slot d.
  const int dlo = p.dlo;
  const int own = dlo > 0 ? 1 : 0;
  auto ntiles = [&](int q) {
    const int hi = min(cl_dmax(q, MT), dlo + kClWindow - 1);
    return hi >= dlo ? hi - dlo + 1 : 0;
  };
  const int ntl = ntiles(r);
  const uint32_t ncols = ntl <= 1 ? 128u : (ntl == 2 ? 256u : 512u);
  uint32_t reader_mask = 0;
  for (int q = 0; q < MT; ++q) {
    const int d = (r - q + MT) % MT;
    const int nq = ntiles(q);
    if (nq > 0 && (d == 0 || (d >= dlo && d < dlo + nq))) reader_mask |= 1u << q;
  }
  const int nreaders = __popc(reader_mask);
  uint16_t writer_mask = 0;
  if (ntl > 0) {
    writer_mask = static_cast<uint16_t>(1u << r);
    for (int d = dlo; d < dlo + ntl; ++d) writer_mask |= static_cast<uint16_t>(1u << ((r + d) % MT));
  }
  const int nwriters = __popc(static_cast<uint32_t>(writer_mask));
  const int64_t c_begin = slice * p.per;
  const int64_t c_end = (c_begin + p.per < p.n) ? c_begin + p.per : p.n;
  const int64_t nchunks = c_end > c_begin ? (c_end - c_begin + 63) / 64 : 0;
  // chunks this CTA produces (none when no CTA reads its tile in this
  // window) and consumes (none when it forms no tile)
  const int64_t nprod = nreaders > 0 ? nchunks : 0;
  const int64_t ncons = ntl > 0 ? nchunks : 0;

  if (warp == 0) tmem_alloc(tmem_slot, ncols);
  if (tid == 0) {
    for (int b = 0; b < kSmjPStages; ++b) {
      // one chunk is delivered by the four warps of one group of each writer
      mbar_init(&pfull[b], static_cast<uint32_t>(max(nwriters, 1) * (kClWarps / kSmjGroups)));
      mbar_init(&pempty[b], static_cast<uint32_t>(max(nreaders, 1)));
    }
    *fail_s = 0;
    fence_barrier_init();
  }
  const int grp = warp / (kClWarps / kSmjGroups);   // chunk group
  const int lr = 32 * (warp % (kClWarps / kSmjGroups)) + lane;   // row (state) of tile r
  const int row = r * 128 + lr;
  // x_ip = (f_i + log N_i - a_i) log2(e) - b_i log2(e) phi_p - log2(e) logden_p
  const bool live = producer && row < p.K;
  const float c2 = live ? static_cast<float>((p.a[row] - fa[row]) * 1.4426950408889634) : -INFINITY;
  const float b2 = live ? static_cast<float>(fb[row] * 1.4426950408889634) : 0.f;
  tc_fence_before();
  cluster_sync_all();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  constexpr uint32_t idesc = idesc_f16(128, 128);

  if (producer) {
    // phi and log2(e) logden of samples lane and lane + 32 of chunk cc
    // (padding: logden +inf)
    auto load_cols = [&](int64_t cc, float& pa, float& pb, float& la, float& lb) {
      const int64_t s0 = c_begin + cc * 64;
      const int ns = static_cast<int>(c_end - s0 < 64 ? c_end - s0 : 64);
      pa = lane < ns ? static_cast<float>(fphi[s0 + lane]) : 0.f;
      pb = lane + 32 < ns ? static_cast<float>(fphi[s0 + lane + 32]) : 0.f;
      la = lane < ns ? static_cast<float>(logden[s0 + lane] * 1.4426950408889634) : INFINITY;
      lb = lane + 32 < ns ? static_cast<float>(logden[s0 + lane + 32] * 1.4426950408889634) : INFINITY;
    };
    // the chunk's columns are loaded during the group's previous chunk (after
    // its fence: a proxy fence also waits for this thread's loads in flight)
    float pa = 0.f, pb = 0.f, l2a = INFINITY, l2b = INFINITY;
    if (grp < nprod) load_cols(grp, pa, pb, l2a, l2b);
    for (int64_t c = grp; c < nprod; c += kSmjGroups) {
      const int b = static_cast<int>(c % kSmjPStages);
      bool ok = true;
      if (c >= kSmjPStages) {
        if (lane == 0)
          ok = mbar_wait_cluster_bounded(&pempty[b], static_cast<uint32_t>(((c - kSmjPStages) / kSmjPStages) & 1),
                                         kMaxSpins);
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      }
      if (!__all_sync(0xffffffffu, ok && *fail_s == 0)) {
        if (lane == 0) *fail_s = 1;
        break;
      }
      unsigned char* pst = pbuf + b * kClPStageBytes;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        float pv[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int sj = 8 * k + j;
          const float l2 = __shfl_sync(0xffffffffu, sj < 32 ? l2a : l2b, sj & 31);
          const float ph = __shfl_sync(0xffffffffu, sj < 32 ? pa : pb, sj & 31);
          pv[j] = ex2_approx(fmaf(-b2, ph, c2) - l2);
        }
        uint4 packed;
        packed.x = pack_half2(pv[0], pv[1]);
        packed.y = pack_half2(pv[2], pv[3]);
        packed.z = pack_half2(pv[4], pv[5]);
        packed.w = pack_half2(pv[6], pv[7]);
        const uint32_t off = static_cast<uint32_t>(lr * 128 + ((k ^ (lr & 7)) << 4));
#pragma unroll
        for (int q = 0; q < kClMaxFactTiles; ++q) {
          if (reader_mask & (1u << q)) {
            const int slot = q == r ? 0 : (r - q + MT) % MT - dlo + own;
            if (q == r)
              *reinterpret_cast<uint4*>(pst + off) = packed;
            else
              st_cluster_v4(mapa_shared(smem_u32(pst + slot * kClPSlotBytes) + off, static_cast<uint32_t>(q)), packed);
          }
        }
      }
      fence_proxy_async_smem_cluster();
      __syncwarp();
      if (lane == 0)
        for (int q = 0; q < MT; ++q)
          if (reader_mask & (1u << q)) mbar_arrive_cluster(mapa_shared(smem_u32(&pfull[b]), static_cast<uint32_t>(q)));
      if (c + kSmjGroups < nprod) load_cols(c + kSmjGroups, pa, pb, l2a, l2b);
    }
  } else {
    for (int64_t cm = 0; cm < ncons; ++cm) {
      const int b = static_cast<int>(cm % kSmjPStages);
      bool ok = true;
      if (lane == 0)
        ok = mbar_wait_cluster_bounded(&pfull[b], static_cast<uint32_t>((cm / kSmjPStages) & 1), kMaxSpins);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok || *fail_s) {
        if (lane == 0) *fail_s = 1;
        break;
      }
      if (lane == 0) {
        tc_fence_after();
        const uint32_t base = smem_u32(pbuf + b * kClPStageBytes);
        for (int t = 0; t < ntl; ++t) {
#pragma unroll
          for (int k4 = 0; k4 < 4; ++k4)
            umma_f16(tmem + static_cast<uint32_t>(t * 128), sdesc_sw128(base + k4 * 32),
                     sdesc_sw128(base + static_cast<uint32_t>((t + own) * kClPSlotBytes) + k4 * 32), idesc,
                     (cm > 0 || k4 > 0) ? 1u : 0u);
        }
        umma_commit_multicast(&pempty[b], writer_mask);
      }
      __syncwarp();
    }
  }
  __syncthreads();
  bool failed = *fail_s != 0;
  if (!failed && nprod > 0) {
    bool ok = true;
    for (int64_t last = nprod - 1; last >= 0 && last >= nprod - kSmjPStages; --last)
      ok = ok && mbar_wait_cluster_bounded(&pempty[last % kSmjPStages],
                                           static_cast<uint32_t>((last / kSmjPStages) & 1), kMaxSpins);
    if (__syncthreads_or(!ok)) failed = true;
  }
  if (failed && tid == 0) atomicAdd(p.err, 1u);
  tc_fence_after();
  float* out = p.out + (slice * p.T + cl_tile_base(r, MT) + dlo) * 128 * 128;
  const int sub = warp & 3;
  const int quarter = warp >> 2;
  const int row_local = sub * 32 + lane;
  for (int c0 = quarter * 32; producer && c0 < ntl * 128; c0 += 128) {
    float rr[32];
    if (nchunks > 0 && !failed) {
      tmem_ld32(tmem + (static_cast<uint32_t>(sub * 32) << 16) + static_cast<uint32_t>(c0), rr);
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i) rr[i] = 0.f;
    }
    float4* dst = reinterpret_cast<float4*>(out + (c0 >> 7) * 128 * 128 + row_local * 128 + (c0 & 127));
#pragma unroll
    for (int i = 0; i < 8; ++i) dst[i] = make_float4(rr[4 * i], rr[4 * i + 1], rr[4 * i + 2], rr[4 * i + 3]);
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, ncols);
  }
}

// Fixed-order FP64 sum of the slices of each accumulator tile; tile
// (q, d) is G's block (q, (q + d) mod MT), mirrored into its transpose.
__global__ void reduce_tc_cluster(const float* __restrict__ part, int S, int T, int MT, int K,
                                  double* __restrict__ G) {
  const int tile = blockIdx.y;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 128 * 128) return;
  int q = 0, base = 0;
  while (q + 1 < MT && base + cl_dmax(q, MT) + 1 <= tile) {
    base += cl_dmax(q, MT) + 1;
    ++q;
  }
  const int d = tile - base;
  double s = 0.0;
  for (int sl = 0; sl < S; ++sl) s += part[(static_cast<int64_t>(sl) * T + tile) * 128 * 128 + e];
  const int row = q * 128 + e / 128;
  const int col = ((q + d) % MT) * 128 + e % 128;
  if (row >= K || col >= K) return;
  if (d == 0 && col < row) return;  // diagonal tile: keep one of each pair
  G[static_cast<int64_t>(row) * K + col] = s;
  G[static_cast<int64_t>(col) * K + row] = s;
}

size_t tc_cluster_smem() {
  return static_cast<size_t>(kClVStages) * kClVStageBytes + static_cast<size_t>(kClPStages) * kClPStageBytes + 128 +
         1024;
}

struct ClPlan {
  int MT = 0, T = 0, S = 0;
  int64_t per = 0;
};

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

namespace {

// Clusters of MT CTAs that can be resident at once (queried once per MT,
// after the kernel's shared-memory limit is raised).
int max_active_clusters(int MT) {
  std::lock_guard<std::recursive_mutex> lock(init_mutex());
  static int cache[kClMaxTiles + 1] = {0, 0, 0, 0, 0};
  if (cache[MT] == 0) {
    if (cudaFuncSetAttribute(overlap_tc_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(tc_cluster_smem())) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(MT * num_sms()));
    cfg.blockDim = dim3(kClThreadsAll);
    cfg.dynamicSmemBytes = tc_cluster_smem();
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = static_cast<unsigned>(MT);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, overlap_tc_cluster_kernel, &cfg) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      n = std::max(1, num_sms() / MT / 2);
    }
    cache[MT] = n;
  }
  return cache[MT];
}

bool cl_eligible(int dtype_bytes, int64_t K) { return dtype_bytes == 4 && K <= 128 * kClMaxTiles && tc_cluster_enabled(); }

// Upper bound of the slices (clusters) of any cluster plan: no more
// clusters than SMs / MT can be resident.
ClPlan cl_plan(int64_t K, int64_t n, int clusters) {
  ClPlan pl;
  pl.MT = static_cast<int>(ceil_div(K, 128));
  pl.T = cl_tile_base(pl.MT, pl.MT);
  const int64_t nch = ceil_div(n, 64);
  const int64_t S = std::max<int64_t>(1, std::min<int64_t>(clusters, nch));
  pl.per = ceil_div(nch, S) * 64;
  pl.S = static_cast<int>(ceil_div(n, pl.per));
  return pl;
}

size_t cl_tmp_bytes(int64_t K) {
  const int MT = static_cast<int>(ceil_div(K, 128));
  const int T = cl_tile_base(MT, MT);
  const int64_t Smax = std::max(1, num_sms() / MT);
  return round_up(Smax * T * 128 * 128 * 4, 256);
}

}  // namespace

size_t overlap_tc_tmp_bytes(int64_t K, int64_t n) {
  const TcPlan pl = tc_plan(K, n);
  const size_t nc = pl.ctas.size(), ni = pl.first.size();
  const size_t items = round_up(static_cast<int64_t>(nc) * 128 * 512 * 4, 256) + round_up(nc * sizeof(TcCta), 256) +
                       round_up(2 * ni * sizeof(int), 256) + 256;
  return K <= 128 * kClMaxFactTiles ? std::max(items, cl_tmp_bytes(K)) : items;
}

static mbar_status overlap_tc_cluster(const void* v, int64_t K, int64_t n, int64_t ld, const double* a,
                                      const void* logden, const int32_t* H, double* G, unsigned* err, void* tmp,
                                      cudaStream_t st) {
  const int MT = static_cast<int>(ceil_div(K, 128));
  const int resident = max_active_clusters(MT);
  if (resident <= 0) {
    set_error("overlap_tc: cannot raise the shared-memory limit of the cluster kernel");
    return MBAR_ECUDA;
  }
  const int clusters = std::min(resident, std::max(1, num_sms() / MT));
  const ClPlan pl = cl_plan(K, n, clusters);
  CUtensorMap map;
  BUMBAR_TRY(make_tmap_2d(&map, v, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, K, n, ld, 32, 128));
  BUMBAR_CUDA(cudaMemsetAsync(G, 0, static_cast<size_t>(K) * K * sizeof(double), st));
  ClParams prm{};
  prm.K = static_cast<int>(K);
  prm.MT = pl.MT;
  prm.T = pl.T;
  prm.n = n;
  prm.per = pl.per;
  prm.a = a;
  prm.logden = static_cast<const float*>(logden);
  prm.H = H;
  prm.out = static_cast<float*>(tmp);
  prm.err = err;
  const size_t smem = tc_cluster_smem();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(pl.S * pl.MT));
  cfg.blockDim = dim3(kClThreadsAll);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = static_cast<unsigned>(pl.MT);
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  BUMBAR_CUDA(cudaLaunchKernelEx(&cfg, overlap_tc_cluster_kernel, map, prm));
  count_launches(1);
  reduce_tc_cluster<<<dim3(128 * 128 / 256, static_cast<unsigned>(pl.T)), 256, 0, st>>>(prm.out, pl.S, pl.T, pl.MT,
                                                                                       static_cast<int>(K), G);
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

mbar_status overlap_tc(const void* v, int dtype_bytes, int64_t K, int64_t n, int64_t ld, const double* a,
                       const void* logden, const int32_t* H, double* G, unsigned* err, void* tmp, size_t tmp_bytes,
                       cudaStream_t st) {
  if (tmp_bytes < overlap_tc_tmp_bytes(K, n)) {
    set_error("overlap_tc: scratch too small");
    return MBAR_EINVAL;
  }
  if (cl_eligible(dtype_bytes, K)) return overlap_tc_cluster(v, K, n, ld, a, logden, H, G, err, tmp, st);
  const TcPlan pl = tc_plan(K, n);
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
    {
      std::lock_guard<std::recursive_mutex> lock(init_mutex());
      if (!attr) {
        BUMBAR_CUDA(cudaFuncSetAttribute(overlap_tc_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem)));
        attr = true;
      }
    }
    overlap_tc_kernel<float><<<nc, kTcThreads, smem, st>>>(prm);
  } else {
    static bool attr = false;
    {
      std::lock_guard<std::recursive_mutex> lock(init_mutex());
      if (!attr) {
        BUMBAR_CUDA(cudaFuncSetAttribute(overlap_tc_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem)));
        attr = true;
      }
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

bool overlap_tc_smaj_eligible(int64_t K) { return K >= 128 && K <= 128 * kClMaxTiles && tc_cluster_enabled(); }

mbar_status overlap_tc_smaj(const float* vst, int64_t K, int64_t n, const double* a, const float* logden, double* G,
                            unsigned* err, void* tmp, size_t tmp_bytes, cudaStream_t st) {
  if (!overlap_tc_smaj_eligible(K)) {
    set_error("overlap_tc_smaj: unsupported K=%lld", static_cast<long long>(K));
    return MBAR_EUNSUPPORTED;
  }
  if (tmp_bytes < overlap_tc_tmp_bytes(K, n)) {
    set_error("overlap_tc_smaj: scratch too small");
    return MBAR_EINVAL;
  }
  const int MT = static_cast<int>(ceil_div(K, 128));
  const size_t smem = static_cast<size_t>(kSmjPStages) * kClPStageBytes + 128 + 1024;  // + barriers, TMEM slot, flag
  static int resident[kClMaxTiles + 1] = {0, 0, 0, 0, 0};
  {
    std::lock_guard<std::recursive_mutex> lock(init_mutex());
    if (resident[MT] == 0) {
      if (cudaFuncSetAttribute(overlap_tc_smaj_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(smem)) != cudaSuccess) {
        cudaGetLastError();
        set_error("overlap_tc_smaj: cannot raise the shared-memory limit");
        return MBAR_ECUDA;
      }
      cudaLaunchConfig_t q = {};
      q.gridDim = dim3(static_cast<unsigned>(MT * num_sms()));
      q.blockDim = dim3(kSmjThreadsAll);
      q.dynamicSmemBytes = smem;
      cudaLaunchAttribute qa[1];
      qa[0].id = cudaLaunchAttributeClusterDimension;
      qa[0].val.clusterDim.x = static_cast<unsigned>(MT);
      qa[0].val.clusterDim.y = 1;
      qa[0].val.clusterDim.z = 1;
      q.attrs = qa;
      q.numAttrs = 1;
      int nres = 0;
      if (cudaOccupancyMaxActiveClusters(&nres, overlap_tc_smaj_kernel, &q) != cudaSuccess || nres <= 0) {
        cudaGetLastError();
        nres = std::max(1, num_sms() / MT / 2);
      }
      resident[MT] = nres;
    }
  }
  const int clusters = std::min(resident[MT], std::max(1, num_sms() / MT));
  const ClPlan pl = cl_plan(K, n, clusters);
  BUMBAR_CUDA(cudaMemsetAsync(G, 0, static_cast<size_t>(K) * K * sizeof(double), st));
  ClParams prm{};
  prm.K = static_cast<int>(K);
  prm.MT = pl.MT;
  prm.T = pl.T;
  prm.n = n;
  prm.per = pl.per;
  prm.a = a;
  prm.logden = logden;
  prm.H = nullptr;
  prm.out = static_cast<float*>(tmp);
  prm.err = err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(pl.S * pl.MT));
  cfg.blockDim = dim3(kSmjThreadsAll);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = static_cast<unsigned>(pl.MT);
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  BUMBAR_CUDA(cudaLaunchKernelEx(&cfg, overlap_tc_smaj_kernel, vst, static_cast<int>(round_up(K, 4)), prm));
  count_launches(1);
  reduce_tc_cluster<<<dim3(128 * 128 / 256, static_cast<unsigned>(pl.T)), 256, 0, st>>>(prm.out, pl.S, pl.T, pl.MT,
                                                                                       static_cast<int>(K), G);
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

mbar_status overlap_tc_fact(const double* fa, const double* fb, const double* fphi, int64_t K, int64_t n,
                            const double* a, const double* logden, double* G, unsigned* err, void* tmp,
                            size_t tmp_bytes, cudaStream_t st) {
  if (K < 1 || K > 128 * kClMaxFactTiles) {
    set_error("overlap_tc_fact: unsupported K=%lld", static_cast<long long>(K));
    return MBAR_EUNSUPPORTED;
  }
  if (tmp_bytes < overlap_tc_tmp_bytes(K, n)) {
    set_error("overlap_tc_fact: scratch too small");
    return MBAR_EINVAL;
  }
  const int MT = static_cast<int>(ceil_div(K, 128));
  const size_t smem = static_cast<size_t>(kSmjPStages) * kClPStageBytes + 128 + 1024;
  static int resident[kClMaxFactTiles + 1] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  {
    std::lock_guard<std::recursive_mutex> lock(init_mutex());
    if (resident[MT] == 0) {
      if (cudaFuncSetAttribute(overlap_tc_fact_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(smem)) != cudaSuccess) {
        cudaGetLastError();
        set_error("overlap_tc_fact: cannot raise the shared-memory limit");
        return MBAR_ECUDA;
      }
      cudaLaunchConfig_t q = {};
      q.gridDim = dim3(static_cast<unsigned>(MT * num_sms()));
      q.blockDim = dim3(kSmjThreadsAll);
      q.dynamicSmemBytes = smem;
      cudaLaunchAttribute qa[1];
      qa[0].id = cudaLaunchAttributeClusterDimension;
      qa[0].val.clusterDim.x = static_cast<unsigned>(MT);
      qa[0].val.clusterDim.y = 1;
      qa[0].val.clusterDim.z = 1;
      q.attrs = qa;
      q.numAttrs = 1;
      int nres = 0;
      if (cudaOccupancyMaxActiveClusters(&nres, overlap_tc_fact_kernel, &q) != cudaSuccess || nres <= 0) {
        cudaGetLastError();
        nres = std::max(1, num_sms() / MT / 2);
      }
      resident[MT] = nres;
    }
  }
  const int clusters = std::min(resident[MT], std::max(1, num_sms() / MT));
  const ClPlan pl = cl_plan(K, n, clusters);
  BUMBAR_CUDA(cudaMemsetAsync(G, 0, static_cast<size_t>(K) * K * sizeof(double), st));
  ClParams prm{};
  prm.K = static_cast<int>(K);
  prm.MT = pl.MT;
  prm.T = pl.T;
  prm.n = n;
  prm.per = pl.per;
  prm.a = a;
  prm.logden = nullptr;
  prm.H = nullptr;
  prm.out = static_cast<float*>(tmp);
  prm.err = err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(pl.S * pl.MT));
  cfg.blockDim = dim3(kSmjThreadsAll);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = static_cast<unsigned>(pl.MT);
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // one launch per window of kClWindow tile distances (two at MT = 6..8);
  // every launch forms all of P~ and writes its own tiles of the partials
  for (int dlo = 0; dlo <= cl_dmax(0, MT); dlo += kClWindow) {
    prm.dlo = dlo;
    BUMBAR_CUDA(cudaLaunchKernelEx(&cfg, overlap_tc_fact_kernel, fa, fb, fphi, logden, prm));
    count_launches(1);
  }
  reduce_tc_cluster<<<dim3(128 * 128 / 256, static_cast<unsigned>(pl.T)), 256, 0, st>>>(prm.out, pl.S, pl.T, pl.MT,
                                                                                       static_cast<int>(K), G);
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

}  // namespace bumbar
