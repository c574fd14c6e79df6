// Binning step of Sec. II on the GPU: uniform bins of width w anchored at
// min(phi), nonempty bins only, integer counts H_p, and the binned reduced
// potential (mean of the members' columns).
//
// The samples are sorted by phi ONCE (stable LSD radix sort on an
// order-preserving 64-bit image of the binary64 keys). Since
// b(phi) = floor((phi - phi_lo)/w) is non-decreasing in phi for every w,
// each later histogram is a scan over contiguous runs of the sorted array:
// head flags where the bin index changes, an exclusive scan for bin
// ordinals, run starts and counts. All integer work is exact; the bin index
// uses the binary64 subtraction and division, each rounded to nearest
// (__dsub_rn/__ddiv_rn; no contraction into FMA).
#include <algorithm>
#include <cstdio>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace bumbar {

namespace {

constexpr int kSortTile = 1024;  // elements per warp tile
constexpr int kScanBlock = 1024; // elements per block in the scan (256 threads x 4)
constexpr int kMaxWidths = kWidthsPerPass;  // candidate widths per counting pass

__device__ __forceinline__ unsigned long long order_key(double x) {
  unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// floor(RN(d / w)) from a double-float FP32 pair (d_hi + d_lo ~ d to
// 2^-48 relative) and rw_hi + rw_lo ~ RN(1/w): the product is formed with an
// exact FP32 FMA error term, so q = d/w is known to ~|q| 2^-44; its integer
// part is returned when the fractional part is farther than
// 2^-20 + |q| 2^-42 from an integer, which also covers the rounding of RN(d/w)
// itself. Otherwise (about 2e-5 of random inputs) the correctly rounded FP64
// division decides. FP32 arithmetic only in the common case.
struct RecipW {
  double w;
  float hi, lo;
};

__host__ __device__ inline RecipW make_recip(double w) {
  RecipW r;
  r.w = w;
  const double rw = 1.0 / w;
  r.hi = static_cast<float>(rw);
  r.lo = static_cast<float>(rw - static_cast<double>(r.hi));
  return r;
}

__device__ __forceinline__ long long key_df(float dh, float dl, const RecipW& r, const double* d_exact) {
  const float p_hi = __fmul_rn(dh, r.hi);
  const float p_err = __fmaf_rn(dh, r.hi, -p_hi);
  const float t = __fadd_rn(__fadd_rn(__fmul_rn(dh, r.lo), __fmul_rn(dl, r.hi)), p_err);
  const float fl = floorf(p_hi);
  const float rr = __fadd_rn(__fsub_rn(p_hi, fl), t);
  const float fr = floorf(rr);
  const float frac = __fsub_rn(rr, fr);
  const float delta = 9.5367431640625e-07f + fabsf(p_hi) * 2.2737367544323206e-13f;  // 2^-20 + |q| 2^-42
  if (frac > delta && frac < 1.0f - delta) {
    if (p_hi < 16777216.0f) return static_cast<long long>(__float2int_rz(__fadd_rn(fl, fr)));  // exact below 2^24
    return static_cast<long long>(fl) + static_cast<long long>(fr);
  }
  return static_cast<long long>(floor(__ddiv_rn(*d_exact, r.w)));
}

// key_df for q = d/w < 2^22 with no conversion instructions: adding 2^23
// with rounding towards -inf leaves 2^23 + floor(p_hi) (float spacing is 1
// in [2^23, 2^24)), whose low mantissa bits are the integer part; the
// remainder (p_hi - floor(p_hi)) + t lies in (-1, 2), so its floor is one of
// -1, 0, 1. Same decisions and the same fallback as key_df.
__device__ __forceinline__ int key_small(float dh, float dl, const RecipW& r, const double* d_exact) {
  const float p_hi = __fmul_rn(dh, r.hi);
  const float p_err = __fmaf_rn(dh, r.hi, -p_hi);
  const float t = __fadd_rn(__fadd_rn(__fmul_rn(dh, r.lo), __fmul_rn(dl, r.hi)), p_err);
  const float m = __fadd_rd(p_hi, 8388608.0f);
  const float fl = __fsub_rn(m, 8388608.0f);
  const int ip = __float_as_int(m) - 0x4B000000;
  const float rr = __fadd_rn(__fsub_rn(p_hi, fl), t);
  const bool neg = rr < 0.f, big = rr >= 1.f;
  const float frac = neg ? __fadd_rn(rr, 1.f) : (big ? __fsub_rn(rr, 1.f) : rr);
  const float delta = 9.5367431640625e-07f + p_hi * 2.2737367544323206e-13f;  // 2^-20 + |q| 2^-42
  if (frac > delta && frac < 1.0f - delta) return ip + (neg ? -1 : (big ? 1 : 0));
  return static_cast<int>(floor(__ddiv_rn(*d_exact, r.w)));
}

// ---------------------------------------------------------------------------
// exclusive scan of int32 (three phases, exact)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int warp_incl_scan(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Block-wide exclusive scan of one value per thread (256 threads); returns
// the exclusive prefix and writes the block total to *total.
__device__ int block_excl_scan(int v, int* total) {
  __shared__ int wsum[kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int incl = warp_incl_scan(v);
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int x = (lane < kThreads / 32) ? wsum[lane] : 0;
    x = warp_incl_scan(x);
    if (lane < kThreads / 32) wsum[lane] = x;
  }
  __syncthreads();
  const int before = (warp > 0) ? wsum[warp - 1] : 0;
  if (total) *total = wsum[kThreads / 32 - 1];
  __syncthreads();
  return before + incl - v;
}

__global__ void scan_block_sums(const int* __restrict__ in, int64_t n, int* __restrict__ sums) {
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanBlock;
  int s = 0;
  for (int j = 0; j < 4; ++j) {
    const int64_t i = base + threadIdx.x * 4 + j;
    if (i < n) s += in[i];
  }
  int tot;
  (void)block_excl_scan(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void scan_sums_single(int* sums, int64_t nblocks, int* grand_total) {
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t b0 = 0; b0 < nblocks; b0 += kThreads) {
    const int64_t i = b0 + threadIdx.x;
    const int v = (i < nblocks) ? sums[i] : 0;
    int tot;
    const int ex = block_excl_scan(v, &tot);
    if (i < nblocks) sums[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0 && grand_total) *grand_total = carry;
}

__global__ void scan_apply(const int* __restrict__ in, int64_t n, const int* __restrict__ sums, int* __restrict__ out) {
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanBlock;
  int v[4];
  int s = 0;
  for (int j = 0; j < 4; ++j) {
    const int64_t i = base + threadIdx.x * 4 + j;
    v[j] = (i < n) ? in[i] : 0;
    s += v[j];
  }
  int ex = block_excl_scan(s, nullptr) + sums[blockIdx.x];
  for (int j = 0; j < 4; ++j) {
    const int64_t i = base + threadIdx.x * 4 + j;
    if (i < n) out[i] = ex;
    ex += v[j];
  }
}

size_t scan_tmp_bytes(int64_t n) { return (ceil_div(n, kScanBlock) + 1) * sizeof(int) + 256; }

mbar_status excl_scan(const int* in, int64_t n, int* out, int* total_dev, void* tmp, cudaStream_t st) {
  const int64_t nb = ceil_div(n, kScanBlock);
  int* sums = static_cast<int*>(tmp);
  scan_block_sums<<<static_cast<unsigned>(nb), kThreads, 0, st>>>(in, n, sums);
  count_launches(1);
  scan_sums_single<<<1, kThreads, 0, st>>>(sums, nb, total_dev);
  count_launches(1);
  scan_apply<<<static_cast<unsigned>(nb), kThreads, 0, st>>>(in, n, sums, out);
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

// ---------------------------------------------------------------------------
// radix sort (8 passes x 8 bits), warp per 1024-element tile, stable
// ---------------------------------------------------------------------------
__global__ void make_keys(const double* __restrict__ phi, int64_t N, unsigned long long* __restrict__ keys,
                          int32_t* __restrict__ idx) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < N) {
    keys[i] = order_key(phi[i]);
    idx[i] = static_cast<int32_t>(i);
  }
}

__global__ void radix_hist(const unsigned long long* __restrict__ keys, int64_t N, int shift, int64_t ntiles,
                           int* __restrict__ tile_hist) {
  __shared__ int cnt[kThreads / 32][256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t tile = static_cast<int64_t>(blockIdx.x) * (kThreads / 32) + warp;
  for (int d = lane; d < 256; d += 32) cnt[warp][d] = 0;
  __syncwarp();
  if (tile < ntiles) {
    const int64_t base = tile * kSortTile;
    for (int c = 0; c < kSortTile / 32; ++c) {
      const int64_t i = base + c * 32 + lane;
      if (i < N) atomicAdd(&cnt[warp][(keys[i] >> shift) & 0xff], 1);
    }
    __syncwarp();
    for (int d = lane; d < 256; d += 32) tile_hist[static_cast<int64_t>(d) * ntiles + tile] = cnt[warp][d];
  }
}

__global__ void radix_scatter(const unsigned long long* __restrict__ keys_in, const int32_t* __restrict__ idx_in,
                              int64_t N, int shift, int64_t ntiles, const int* __restrict__ offsets,
                              unsigned long long* __restrict__ keys_out, int32_t* __restrict__ idx_out) {
  __shared__ int cnt[kThreads / 32][257];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t tile = static_cast<int64_t>(blockIdx.x) * (kThreads / 32) + warp;
  if (tile >= ntiles) return;  // whole warp leaves together
  for (int d = lane; d < 256; d += 32) cnt[warp][d] = offsets[static_cast<int64_t>(d) * ntiles + tile];
  if (lane == 0) cnt[warp][256] = 0;
  __syncwarp();
  const unsigned lt_mask = (1u << lane) - 1u;
  const int64_t base = tile * kSortTile;
  for (int c = 0; c < kSortTile / 32; ++c) {
    const int64_t i = base + c * 32 + lane;
    const bool in = i < N;
    unsigned long long k = in ? keys_in[i] : 0ull;
    const int d = in ? static_cast<int>((k >> shift) & 0xff) : 256;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & lt_mask);
    const int b = cnt[warp][d];
    __syncwarp();
    if ((__ffs(peers) - 1) == lane) cnt[warp][d] = b + __popc(peers);
    __syncwarp();
    if (in) {
      const int dst = b + rank;
      keys_out[dst] = k;
      idx_out[dst] = idx_in[i];
    }
  }
}

__global__ void gather_phi(const double* __restrict__ phi, const int32_t* __restrict__ perm, int64_t N,
                           double* __restrict__ out) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < N) out[i] = phi[perm[i]];
}

// ---------------------------------------------------------------------------
// histogram over sorted phi
// ---------------------------------------------------------------------------
// Number of nonempty bins for up to kMaxWidths widths in one pass over
// d_i = phi_i - phi_lo (sorted). Bin indices are non-decreasing in i, so a
// thread owning 16 consecutive samples first compares the indices just before
// and at the end of its chunk: equal means no bin starts inside, a difference
// of one means exactly one does; only otherwise are all 16 indices formed.
struct WidthSet {
  RecipW r[kMaxWidths];
  int n;
};
constexpr int kCountChunk = 16;

// Up to kWidthsPerRow widths per grid row (blockIdx.y): a full pass runs as
// ceil(nw / kWidthsPerRow) times as many CTAs (several waves instead of one
// and a small remainder), each row reading the chunks again from L2.
constexpr int kWidthsPerRow = 4;
__global__ void __launch_bounds__(kThreads) count_heads_multi(const float2* __restrict__ dhl,
                                                               const double* __restrict__ d, int64_t N, WidthSet ws,
                                                               unsigned long long* __restrict__ counts) {
  __shared__ unsigned int cnt[kWidthsPerRow];
  if (threadIdx.x < kWidthsPerRow) cnt[threadIdx.x] = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t i0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) * kCountChunk;
  const int64_t i1 = (i0 + kCountChunk < N) ? i0 + kCountChunk : N;
  const int nv = i0 < N ? static_cast<int>(i1 - i0) : 0;
  // the chunk (and the sample before it) in registers, loaded once for all widths
  float2 x[kCountChunk];
#pragma unroll
  for (int j = 0; j < kCountChunk; ++j) x[j] = (j < nv) ? dhl[i0 + j] : make_float2(0.f, 0.f);
  const float2 xp = (nv > 0 && i0 > 0) ? dhl[i0 - 1] : make_float2(0.f, 0.f);
  const float2 xl = (nv > 0) ? dhl[i1 - 1] : make_float2(0.f, 0.f);
  const float dmax = N > 0 ? dhl[N - 1].x : 0.f;  // largest offset (sorted)
  // heads of one chunk under width r, keys of type Key from key_fn
  auto chunk_heads = [&](const RecipW& r, auto key_fn) -> unsigned int {
    unsigned int heads = 0;
    const auto kend = key_fn(xl, r, d + i1 - 1);
    auto kprev = kend;
    if (i0 == 0) {
      heads = 1;  // the first sample opens the first bin
      kprev = key_fn(x[0], r, d);
    } else {
      kprev = key_fn(xp, r, d + i0 - 1);
    }
    const auto diff = kend - kprev;
    if (diff == 1) {
      heads += 1;
    } else if (diff > 1) {
#pragma unroll
      for (int j = 0; j < kCountChunk; ++j) {
        if (j < nv && !(i0 == 0 && j == 0)) {
          const auto k = key_fn(x[j], r, d + i0 + j);
          heads += (k != kprev) ? 1u : 0u;
          kprev = k;
        }
      }
    }
    return heads;
  };
  const int c0 = blockIdx.y * kWidthsPerRow;
  const int c1 = (c0 + kWidthsPerRow < ws.n) ? c0 + kWidthsPerRow : ws.n;
  for (int c = c0; c < c1; ++c) {
    unsigned int heads = 0;
    if (nv > 0) {
      const RecipW r = ws.r[c];
      // every key of this width below 4e6 < 2^22 (margin for the rounding of dmax * hi)
      if (__fmul_ru(dmax, r.hi) < 4.0e6f)
        heads = chunk_heads(r, [](float2 v, const RecipW& rw, const double* de) { return key_small(v.x, v.y, rw, de); });
      else
        heads = chunk_heads(r, [](float2 v, const RecipW& rw, const double* de) { return key_df(v.x, v.y, rw, de); });
    }
    for (int o = 16; o >= 1; o >>= 1) heads += __shfl_xor_sync(0xffffffffu, heads, o);
    if (lane == 0 && heads) atomicAdd(&cnt[c - c0], heads);
  }
  __syncthreads();
  if (threadIdx.x < c1 - c0 && cnt[threadIdx.x])
    atomicAdd(&counts[c0 + threadIdx.x], static_cast<unsigned long long>(cnt[threadIdx.x]));
}

__global__ void offsets_from_lo(const double* __restrict__ phi, int64_t N, double* __restrict__ d,
                                float2* __restrict__ dhl) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < N) {
    const double x = __dsub_rn(phi[i], phi[0]);
    d[i] = x;
    const float hi = __double2float_rn(x);
    dhl[i] = make_float2(hi, __double2float_rn(__dsub_rn(x, static_cast<double>(hi))));
  }
}

__global__ void head_flags(const float2* __restrict__ dhl, const double* __restrict__ d, int64_t N, RecipW r,
                           int* __restrict__ flags) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  long long key = 0;
  if (i < N) {
    const float2 x = dhl[i];
    key = key_df(x.x, x.y, r, d + i);
  }
  long long prev = __shfl_up_sync(0xffffffffu, key, 1);
  if ((threadIdx.x & 31) == 0 && i > 0 && i < N) {
    const float2 x = dhl[i - 1];
    prev = key_df(x.x, x.y, r, d + i - 1);
  }
  if (i < N) flags[i] = (i == 0 || key != prev) ? 1 : 0;
}

__global__ void finish_histogram(const float2* __restrict__ dhl, const double* __restrict__ d, int64_t N, RecipW r,
                                 const int* __restrict__ flags,
                                 const int* __restrict__ excl, int32_t* __restrict__ seg, int32_t* __restrict__ start,
                                 int64_t* __restrict__ keys, int32_t* __restrict__ nb_dev) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int f = flags[i];
  const int e = excl[i];
  seg[i] = e + f - 1;
  if (f) {
    start[e] = static_cast<int32_t>(i);
    const float2 x = dhl[i];
    keys[e] = key_df(x.x, x.y, r, d + i);
  }
  if (i == N - 1) {
    const int nb = e + f;
    *nb_dev = nb;
    start[nb] = static_cast<int32_t>(N);
  }
}

__global__ void counts_from_starts(const int32_t* __restrict__ start, int64_t nb, int32_t* __restrict__ H) {
  const int64_t b = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (b < nb) H[b] = start[b + 1] - start[b];
}

// ---------------------------------------------------------------------------
// binned means: segmented sums over contiguous sorted columns
// ---------------------------------------------------------------------------
// Each warp owns a tile of 256 sorted columns (32 lanes x 8 consecutive
// columns) and walks a range of rows, with no block-level synchronisation.
// Per row, a lane splits its 8 values into runs of equal bin ordinal; runs
// that start and end inside the lane are written at once; the last run of
// each lane enters a warp-wide segmented inclusive scan that carries it
// across lanes. A bin whose run ends in a lane is finished there: written if
// the bin started in this tile, else its partial goes to carry0[tile] (a bin
// that began in an earlier tile). The last lane's still-open run goes to
// carry1[tile] (a bin that starts in this tile and continues) or, if it
// began before the tile, to carry0[tile]. A fix-up kernel finishes bins that
// span tiles: sum = carry1[first tile] + carry0[later tiles], in order.
constexpr int kBmCols = 8;
constexpr int kBmTile = 32 * kBmCols;  // columns per warp tile (256)
constexpr int kBmRowsPerBlock = 64;    // rows a block walks for its eight warp tiles

// Accumulation type of the segmented sums: FP32 for FP32 data (the binned
// matrix only steers Algorithm 1; the answer comes from the unbinned data,
// and FP64 arithmetic is slow on this part), FP64 for FP64 data.
template <typename T>
struct Acc;
template <>
struct Acc<float> {
  using type = float;
};
template <>
struct Acc<double> {
  using type = double;
};

// Mean of a run of `len` (1..7) columns that lies inside one lane: FP32
// division, or for FP64 the product with 1/len (as 1 / count elsewhere).
__device__ __forceinline__ float run_mean(float sum, int len) { return sum / static_cast<float>(len); }
__device__ __forceinline__ double run_mean(double sum, int len) {
  const double r = len == 1 ? 1.0 : len == 2 ? 0.5 : len == 4 ? 0.25 : 1.0 / static_cast<double>(len);
  return sum * r;
}

template <typename T, typename A>
__device__ __forceinline__ void load8(const T* src, int nvalid, A* x) {
  if constexpr (sizeof(T) == 4) {
    if (nvalid == 8) {
      const float4 a = *reinterpret_cast<const float4*>(src);
      const float4 b = *reinterpret_cast<const float4*>(src + 4);
      x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
      x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
      return;
    }
  } else {
    if (nvalid == 8) {
#pragma unroll
      for (int j = 0; j < 8; j += 2) {
        const double2 a = *reinterpret_cast<const double2*>(src + j);
        x[j] = a.x;
        x[j + 1] = a.y;
      }
      return;
    }
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = (j < nvalid) ? static_cast<A>(src[j]) : A(0);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) bin_sums_block(const T* __restrict__ v, int64_t K, int64_t N, int64_t ld,
                                                           const int32_t* __restrict__ seg,
                                                           const int32_t* __restrict__ start,
                                                           const double* __restrict__ inv_count, T* __restrict__ out,
                                                           int64_t ld_out, typename Acc<T>::type* __restrict__ carry0,
                                                           typename Acc<T>::type* __restrict__ carry1, int64_t ntiles) {
  using A = typename Acc<T>::type;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t tile = static_cast<int64_t>(blockIdx.x) * (kThreads / 32) + warp;
  if (tile >= ntiles) return;  // whole warp
  const int64_t tile0 = tile * kBmTile;
  const int64_t tile_end = (tile0 + kBmTile < N) ? tile0 + kBmTile : N;
  const int64_t c0 = tile0 + static_cast<int64_t>(lane) * kBmCols;
  const int nvalid = static_cast<int>(c0 < N ? ((N - c0) < kBmCols ? (N - c0) : kBmCols) : 0);
  const bool last_lane = nvalid > 0 && c0 + nvalid == tile_end;

  // run structure of this lane's columns (identical for every row)
  int sg[kBmCols];
#pragma unroll
  for (int j = 0; j < kBmCols; ++j) sg[j] = (j < nvalid) ? seg[c0 + j] : -1;
  const int b0 = sg[0];
  const int bl = nvalid > 0 ? sg[nvalid - 1] : -1;
  int nruns = 0;
#pragma unroll
  for (int j = 1; j < kBmCols; ++j)
    if (j < nvalid && sg[j] != sg[j - 1]) ++nruns;
  const int64_t st_b0 = nvalid > 0 ? start[b0] : 0;
  const int64_t st_bl = nvalid > 0 ? start[bl] : 0;
  const int64_t en_bl = nvalid > 0 ? start[bl + 1] : 0;
  const bool flag = nvalid <= 0 || nruns > 0 || st_bl >= c0;  // last run starts in this lane
  const bool cont = nvalid > 0 && st_b0 < c0;                 // first run continues from the left
  const bool last_ends_here = nvalid > 0 && en_bl <= c0 + nvalid;
  const A inv_b0 = nvalid > 0 ? static_cast<A>(inv_count[b0]) : A(0);
  const A inv_bl = nvalid > 0 ? static_cast<A>(inv_count[bl]) : A(0);

  const int64_t k_begin = static_cast<int64_t>(blockIdx.y) * kBmRowsPerBlock;
  const int64_t k_end = (k_begin + kBmRowsPerBlock < K) ? k_begin + kBmRowsPerBlock : K;
  A xn[kBmCols];  // next row, loaded one row ahead
  if (k_begin < k_end) load8<T, A>(v + k_begin * ld + c0, nvalid, xn);
  for (int64_t k = k_begin; k < k_end; ++k) {
    A x[kBmCols];
#pragma unroll
    for (int j = 0; j < kBmCols; ++j) x[j] = xn[j];
    if (k + 1 < k_end) load8<T, A>(v + (k + 1) * ld + c0, nvalid, xn);
    A head = A(0), run = A(0);
    int cur = b0;
    int rs = 0;  // column where the current run starts
    bool first = true;
#pragma unroll
    for (int j = 0; j < kBmCols; ++j) {
      if (j < nvalid) {
        if (sg[j] != cur) {
          if (first) {
            head = run;
            first = false;
          } else {  // interior run: the whole bin lies in this lane, its count is the run length
            out[k * ld_out + cur] = static_cast<T>(run_mean(run, j - rs));
          }
          cur = sg[j];
          rs = j;
          run = A(0);
        }
        run += x[j];
      }
    }
    // warp-wide segmented inclusive scan of the last-run sums
    A sv = nvalid > 0 ? run : A(0);
    int sf = flag ? 1 : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const A uv = __shfl_up_sync(0xffffffffu, sv, o);
      const int uf = __shfl_up_sync(0xffffffffu, sf, o);
      if (lane >= o) {
        if (!sf) sv += uv;
        sf |= uf;
      }
    }
    A prev = __shfl_up_sync(0xffffffffu, sv, 1);
    if (lane == 0) prev = A(0);
    if (nvalid > 0) {
      const A carry_in = cont ? prev : A(0);
      if (nruns > 0) {  // the first run ends inside this lane
        const A tot = carry_in + head;
        if (st_b0 >= tile0)
          out[k * ld_out + b0] = static_cast<T>(tot * inv_b0);
        else
          carry0[tile * K + k] = tot;
      }
      if (last_ends_here) {
        if (st_bl >= tile0)
          out[k * ld_out + bl] = static_cast<T>(sv * inv_bl);
        else
          carry0[tile * K + k] = sv;
      } else if (last_lane) {
        if (st_bl >= tile0)
          carry1[tile * K + k] = sv;
        else
          carry0[tile * K + k] = sv;
      }
    }
  }
}

// All levels of a schedule in one read of v: the warp-tile scheme of
// bin_sums_block, repeated per level on the same eight values of each lane.
// Bins are consecutive along the sorted columns, so a lane's runs are bins
// b0, b0 + 1, ...; per level a lane keeps only b0, a bit set of run starts
// and a few flags (row independent), and the inverse counts of its first
// and last bin.
constexpr int kMaxLevels = 8;
struct LevelOut {
  const int32_t* seg;
  const int32_t* start;
  const double* inv;
  void* out;
  int64_t ld_out;
  void* carry0;  // partial sums at tile edges, in the kernel's accumulator type
  void* carry1;
};
struct MultiLevel {
  LevelOut l[kMaxLevels];
  int L;
};

// descriptor bits: 0..7 run starts at column j (j >= 1); 8 last run starts in
// this lane; 9 first run continues from the left; 10 last run ends in this
// lane; 11 first bin starts in this tile; 12 last bin starts in this tile;
// 16..19 number of run starts
template <typename T, int NL>
__global__ void __launch_bounds__(kThreads) bin_sums_multi(const T* __restrict__ v, int64_t K, int64_t N, int64_t ld,
                                                           MultiLevel ml, int64_t ntiles) {
  using A = typename Acc<T>::type;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t tile = static_cast<int64_t>(blockIdx.x) * (kThreads / 32) + warp;
  if (tile >= ntiles) return;  // whole warp
  const int64_t tile0 = tile * kBmTile;
  const int64_t tile_end = (tile0 + kBmTile < N) ? tile0 + kBmTile : N;
  const int64_t c0 = tile0 + static_cast<int64_t>(lane) * kBmCols;
  const int nvalid = static_cast<int>(c0 < N ? ((N - c0) < kBmCols ? (N - c0) : kBmCols) : 0);
  const bool last_lane = nvalid > 0 && c0 + nvalid == tile_end;

  int b0[NL];
  unsigned bits[NL];
  A inv0[NL], invl[NL];
#pragma unroll
  for (int l = 0; l < NL; ++l) {
    b0[l] = 0;
    bits[l] = 0;
    inv0[l] = invl[l] = A(0);
    if (nvalid > 0) {
      const int32_t* seg = ml.l[l].seg;
      const int32_t* start = ml.l[l].start;
      const int first = seg[c0];
      int prev = first, nr = 0;
      unsigned b = 0;
#pragma unroll
      for (int j = 1; j < kBmCols; ++j) {
        if (j < nvalid) {
          const int sj = seg[c0 + j];
          if (sj != prev) {
            b |= 1u << j;
            ++nr;
          }
          prev = sj;
        }
      }
      const int last = prev;
      const int64_t st0 = start[first], stl = start[last], enl = start[last + 1];
      if (nr > 0 || stl >= c0) b |= 1u << 8;
      if (st0 < c0) b |= 1u << 9;
      if (enl <= c0 + nvalid) b |= 1u << 10;
      if (st0 >= tile0) b |= 1u << 11;
      if (stl >= tile0) b |= 1u << 12;
      b |= static_cast<unsigned>(nr) << 16;
      // the whole tile is one bin (row independent, uniform over the warp)
      if (seg[tile0] == seg[tile_end - 1]) b |= 1u << 13;
      b0[l] = first;
      bits[l] = b;
      inv0[l] = static_cast<A>(ml.l[l].inv[first]);
      invl[l] = static_cast<A>(ml.l[l].inv[last]);
    } else {
      bits[l] = 1u << 8;  // past the end: empty segment head
    }
  }

  // a tile one bin covers: where lane 0 puts its sum (the same on every row):
  // 0 the continuation of a bin opened in an earlier tile (carry0), 1 the
  // bin's mean (the bin lies inside the tile), 2 its opening part (carry1)
  int one_mode[NL];
#pragma unroll
  for (int l = 0; l < NL; ++l) {
    one_mode[l] = 0;
    if (lane == 0 && nvalid > 0 && (bits[l] & (1u << 13))) {
      const int64_t st = ml.l[l].start[b0[l]], en = ml.l[l].start[b0[l] + 1];
      one_mode[l] = st < tile0 ? 0 : (en <= tile_end ? 1 : 2);
    }
  }

  const int64_t k_begin = static_cast<int64_t>(blockIdx.y) * kBmRowsPerBlock;
  const int64_t k_end = (k_begin + kBmRowsPerBlock < K) ? k_begin + kBmRowsPerBlock : K;
  A xn[kBmCols];
  // row pointers advanced by their strides (no 64-bit products in the loop)
  if (k_begin < k_end) load8<T, A>(v + k_begin * ld + c0, nvalid, xn);
  for (int64_t k = k_begin; k < k_end; ++k) {
    A x[kBmCols];
#pragma unroll
    for (int j = 0; j < kBmCols; ++j) x[j] = xn[j];
    if (k + 1 < k_end) load8<T, A>(v + (k + 1) * ld + c0, nvalid, xn);
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      const unsigned b = bits[l];
      T* out = static_cast<T*>(ml.l[l].out) + k * ml.l[l].ld_out;
      if (__shfl_sync(0xffffffffu, b, 0) & (1u << 13)) {
        // one bin covers the tile: a plain warp sum, written by lane 0 as
        // the bin's mean (bin inside the tile), its opening part (carry1) or
        // a continuation (carry0)
        A t = A(0);
#pragma unroll
        for (int j = 0; j < kBmCols; ++j) t += x[j];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) {
          if (one_mode[l] == 0)
            static_cast<A*>(ml.l[l].carry0)[tile * K + k] = t;
          else if (one_mode[l] == 1)
            out[b0[l]] = static_cast<T>(t * inv0[l]);
          else
            static_cast<A*>(ml.l[l].carry1)[tile * K + k] = t;
        }
        continue;
      }
      A head = A(0), run = A(0);
      int cur = b0[l];
      int rs = 0;  // column where the current run starts
      bool first = true;
#pragma unroll
      for (int j = 0; j < kBmCols; ++j) {
        if (j < nvalid) {
          if (b & (1u << j)) {
            if (first) {
              head = run;
              first = false;
            } else {  // interior run: the whole bin lies in this lane, its count is the run length
              out[cur] = static_cast<T>(run_mean(run, j - rs));
            }
            ++cur;
            rs = j;
            run = A(0);
          }
          run += x[j];
        }
      }
      A sv = nvalid > 0 ? run : A(0);
      int sf = (b >> 8) & 1;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const A uv = __shfl_up_sync(0xffffffffu, sv, o);
        const int uf = __shfl_up_sync(0xffffffffu, sf, o);
        if (lane >= o) {
          if (!sf) sv += uv;
          sf |= uf;
        }
      }
      A prev = __shfl_up_sync(0xffffffffu, sv, 1);
      if (lane == 0) prev = A(0);
      if (nvalid > 0) {
        const int nruns = static_cast<int>((b >> 16) & 15u);
        A* carry0 = static_cast<A*>(ml.l[l].carry0) + tile * K + k;
        if (nruns > 0) {  // the first run ends inside this lane
          const A tot = (((b >> 9) & 1) ? prev : A(0)) + head;
          if ((b >> 11) & 1)
            out[b0[l]] = static_cast<T>(tot * inv0[l]);
          else
            *carry0 = tot;
        }
        const int bl = b0[l] + nruns;
        if ((b >> 10) & 1) {
          if ((b >> 12) & 1)
            out[bl] = static_cast<T>(sv * invl[l]);
          else
            *carry0 = sv;
        } else if (last_lane) {
          if ((b >> 12) & 1)
            static_cast<A*>(ml.l[l].carry1)[tile * K + k] = sv;
          else
            *carry0 = sv;
        }
      }
    }
  }
}

// Bin means of a level with small bins (a few samples each): one thread per
// bin and chunk of rows, summing the bin's columns in order; the bins of a
// warp are consecutive, so its loads of one row cover consecutive columns.
constexpr int kFineRows = 64;
constexpr double kFineMaxMean = 4.0;  // levels with at most this many samples per bin on average
template <typename T>
__global__ void __launch_bounds__(kThreads) bin_means_fine(const T* __restrict__ v, int64_t K, int64_t ld,
                                                           const int32_t* __restrict__ start, int64_t nb,
                                                           T* __restrict__ out, int64_t ld_out) {
  using A = typename Acc<T>::type;
  const int64_t b = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x;
  if (b >= nb) return;
  const int64_t s = start[b], e = start[b + 1];
  const A inv = static_cast<A>(1.0 / static_cast<double>(e - s));
  const int64_t k0 = static_cast<int64_t>(blockIdx.y) * kFineRows;
  const int64_t k1 = (k0 + kFineRows < K) ? k0 + kFineRows : K;
  int64_t k = k0;
  for (; k + 8 <= k1; k += 8) {  // eight rows at a time: their loads are in flight together
    const T* r0 = v + k * ld;
    A a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = A(0);
    for (int64_t c = s; c < e; ++c) {
      A x[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) x[i] = static_cast<A>(r0[i * ld + c]);
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] += x[i];
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) out[(k + i) * ld_out + b] = static_cast<T>(a[i] * inv);
  }
  for (; k + 4 <= k1; k += 4) {
    const T* r0 = v + k * ld;
    A a[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = A(0);
    for (int64_t c = s; c < e; ++c) {
      A x[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) x[i] = static_cast<A>(r0[i * ld + c]);
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] += x[i];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) out[(k + i) * ld_out + b] = static_cast<T>(a[i] * inv);
  }
  for (; k < k1; ++k) {
    const T* row = v + k * ld;
    A acc = A(0);
    for (int64_t c = s; c < e; ++c) acc += static_cast<A>(row[c]);
    out[k * ld_out + b] = static_cast<T>(acc * inv);
  }
}

__global__ void inverse_counts(const int32_t* __restrict__ start, int64_t nb, double* __restrict__ inv) {
  const int64_t b = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (b < nb) inv[b] = 1.0 / static_cast<double>(start[b + 1] - start[b]);
}

// Bins that span tiles. A bin crosses the first column of tile t (t >= 1)
// and began in tile t - 1 for exactly the spanning bins, each once. One warp
// per (such t, chunk of 32 rows), one row per lane: carry1[t - 1] plus the
// carry0 of every later tile the bin covers, in tile order. Carries are
// stored tile-major ([tile][K]), so each step reads 32 consecutive rows.
constexpr int kFixWarps = kThreads / 32;
template <typename T>
__global__ void bin_sums_fixup(int64_t K, const int32_t* __restrict__ seg, const int32_t* __restrict__ start,
                               const double* __restrict__ inv_count, T* __restrict__ out, int64_t ld_out,
                               const typename Acc<T>::type* __restrict__ carry0,
                               const typename Acc<T>::type* __restrict__ carry1, int64_t ntiles) {
  const int lane = threadIdx.x & 31;
  const int64_t t = static_cast<int64_t>(blockIdx.x) * kFixWarps + (threadIdx.x >> 5) + 1;
  if (t >= ntiles) return;
  const int64_t c = t * kBmTile;
  const int b = seg[c];
  const int64_t s = start[b];
  if (s >= c || s < c - kBmTile) return;
  const int64_t k = static_cast<int64_t>(blockIdx.y) * 32 + lane;
  if (k >= K) return;
  const int64_t te = (static_cast<int64_t>(start[b + 1]) - 1) / kBmTile;
  double sum = static_cast<double>(carry1[(t - 1) * K + k]);
  int64_t u = t;
  for (; u + 8 <= te + 1; u += 8) {  // eight loads in flight, added in order
    double x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = static_cast<double>(carry0[(u + j) * K + k]);
#pragma unroll
    for (int j = 0; j < 8; ++j) sum += x[j];
  }
  for (; u <= te; ++u) sum += static_cast<double>(carry0[u * K + k]);
  out[k * ld_out + b] = static_cast<T>(sum * inv_count[b]);
}

// out[k][i] = in[k][perm[i]]: each thread loads perm[i] once and moves it
// for kGatherRows rows; blocks run row-group major so the input rows being
// gathered (and the output rows being written) stay in L2 together.
constexpr int kGatherRows = 4;
template <typename T>
__global__ void gather_cols_kernel(const T* __restrict__ in, T* __restrict__ out, int64_t K, int64_t N, int64_t ld,
                                   const int32_t* __restrict__ perm) {
  const int64_t k0 = static_cast<int64_t>(blockIdx.y) * kGatherRows;
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int64_t src = perm[i];
  T vals[kGatherRows];
#pragma unroll
  for (int r = 0; r < kGatherRows; ++r)
    if (k0 + r < K) vals[r] = in[(k0 + r) * ld + src];
#pragma unroll
  for (int r = 0; r < kGatherRows; ++r)
    if (k0 + r < K) out[(k0 + r) * ld + i] = vals[r];
}

// v[k][i] = vst[perm[i]][k] (sample pitch stage_pitch(K)): sample-major
// staging -> row-major store in the new column order. A block takes one 128-byte line of output columns
// (CS = 32 FP32 / 16 FP64): it reads its CS source samples as contiguous
// K-vectors into shared memory (pitch P with P words = 1 mod 32, so both
// the row-wise fill and the column-wise read are conflict-free) and writes
// every row's CS columns as one full line.
constexpr int kGtThreads = 256;
template <typename T>
__host__ __device__ constexpr int gt_cols() {
  return 128 / static_cast<int>(sizeof(T));
}
template <typename T>
__host__ __device__ inline int64_t gt_pitch(int64_t K) {
  // in elements; P * sizeof(T) / 4 = 1 (FP32) or 2 (FP64) mod 32
  return sizeof(T) == 4 ? (K + 31) / 32 * 32 + 1 : (K + 15) / 16 * 16 + 1;
}
template <typename T>
__global__ void __launch_bounds__(kGtThreads) gather_transpose_kernel(const T* __restrict__ vst, int64_t K, int64_t N,
                                                                      const int32_t* __restrict__ perm,
                                                                      T* __restrict__ v, int64_t ld) {
  constexpr int CS = gt_cols<T>();
  extern __shared__ __align__(16) unsigned char gt_raw[];
  T* xs = reinterpret_cast<T*>(gt_raw);  // [CS][P]
  const int64_t P = gt_pitch<T>(K);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * CS;
  // two source samples per warp at a time (columns c and c + NW): up to 32
  // loads in flight per lane (two whole columns for K <= 512), which the
  // latency of these scattered 2-4 KB reads needs at three CTAs per SM
  constexpr int NW = kGtThreads / 32;
  for (int c = warp; c < CS; c += 2 * NW) {
    const int64_t ia = i0 + c, ib = i0 + c + NW;
    if (ia >= N) break;
    const bool hb = c + NW < CS && ib < N;
    const T* sa = vst + static_cast<int64_t>(perm[ia]) * stage_pitch(K);
    const T* sb = hb ? vst + static_cast<int64_t>(perm[ib]) * stage_pitch(K) : sa;
    T* da = xs + c * P;
    T* db = xs + (c + NW) * P;
    for (int64_t k0 = 0; k0 < K; k0 += 16 * 32) {
      T x[16], y[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int64_t k = k0 + lane + 32 * r;
        if (k < K) {
          x[r] = sa[k];
          if (hb) y[r] = sb[k];
        }
      }
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int64_t k = k0 + lane + 32 * r;
        if (k < K) {
          da[k] = x[r];
          if (hb) db[k] = y[r];
        }
      }
    }
  }
  __syncthreads();
  constexpr int RPW = 32 / CS;  // rows per warp instruction
  const int c = lane % CS, rs = lane / CS;
  if (i0 + c >= N) return;
  const T* col = xs + c * P;
  T* out = v + i0 + c;
  for (int64_t k = warp * RPW + rs; k < K; k += (kGtThreads / 32) * RPW) out[k * ld] = col[k];
}

}  // namespace

// ---------------------------------------------------------------------------
// host wrappers
// ---------------------------------------------------------------------------

size_t sort_tmp_bytes(int64_t N) {
  const int64_t ntiles = ceil_div(N, kSortTile);
  const int64_t L = 256 * ntiles;
  size_t b = 0;
  b += round_up(N * 8, 256) * 2;  // keys a/b
  b += round_up(N * 4, 256);      // idx b
  b += round_up(L * 4, 256) * 2;  // hist, offsets
  b += round_up(scan_tmp_bytes(L), 256);
  return b;
}

mbar_status sort_coordinate(const double* phi, int64_t N, double* phi_sorted, int32_t* perm, void* tmp,
                            size_t tmp_bytes, cudaStream_t st) {
  if (tmp_bytes < sort_tmp_bytes(N)) {
    set_error("sort_coordinate: scratch too small");
    return MBAR_EINVAL;
  }
  const int64_t ntiles = ceil_div(N, kSortTile);
  const int64_t L = 256 * ntiles;
  unsigned char* p = static_cast<unsigned char*>(tmp);
  auto* ka = reinterpret_cast<unsigned long long*>(p);
  p += round_up(N * 8, 256);
  auto* kb = reinterpret_cast<unsigned long long*>(p);
  p += round_up(N * 8, 256);
  auto* ib = reinterpret_cast<int32_t*>(p);
  p += round_up(N * 4, 256);
  int* hist = reinterpret_cast<int*>(p);
  p += round_up(L * 4, 256);
  int* offs = reinterpret_cast<int*>(p);
  p += round_up(L * 4, 256);
  void* stmp = p;

  const unsigned gN = static_cast<unsigned>(ceil_div(N, kThreads));
  int32_t* ia = perm;  // ping-pong: idx a lives in the output buffer
  make_keys<<<gN, kThreads, 0, st>>>(phi, N, ka, ia);
  count_launches(1);
  const unsigned gT = static_cast<unsigned>(ceil_div(ntiles, kThreads / 32));
  for (int pass = 0; pass < 8; ++pass) {
    const int shift = pass * 8;
    radix_hist<<<gT, kThreads, 0, st>>>(ka, N, shift, ntiles, hist);
    count_launches(1);
    BUMBAR_TRY(excl_scan(hist, L, offs, nullptr, stmp, st));
    radix_scatter<<<gT, kThreads, 0, st>>>(ka, ia, N, shift, ntiles, offs, kb, ib);
    count_launches(1);
    std::swap(ka, kb);
    std::swap(ia, ib);
  }
  // after 8 passes the sorted indices are back in `perm` (even pass count)
  gather_phi<<<gN, kThreads, 0, st>>>(phi, perm, N, phi_sorted);
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

mbar_status offsets_from_min(const double* phi_sorted, int64_t N, double* d_sorted, float2* d_pairs,
                             cudaStream_t st) {
  offsets_from_lo<<<static_cast<unsigned>(ceil_div(N, kThreads)), kThreads, 0, st>>>(phi_sorted, N, d_sorted,
                                                                                     d_pairs);
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

mbar_status count_bins(const float2* d_pairs, const double* d_sorted, int64_t N, const double* widths, int nw,
                       unsigned long long* counts_dev, cudaStream_t st) {
  if (nw < 1 || nw > kMaxWidths) {
    set_error("count_bins: 1..%d widths per pass", kMaxWidths);
    return MBAR_EINVAL;
  }
  WidthSet ws{};
  ws.n = nw;
  for (int c = 0; c < nw; ++c) ws.r[c] = make_recip(widths[c]);
  BUMBAR_CUDA(cudaMemsetAsync(counts_dev, 0, kMaxWidths * sizeof(unsigned long long), st));
  const dim3 grid(static_cast<unsigned>(ceil_div(N, static_cast<int64_t>(kThreads) * kCountChunk)),
                  static_cast<unsigned>(ceil_div(nw, kWidthsPerRow)));
  count_heads_multi<<<grid, kThreads, 0, st>>>(d_pairs, d_sorted, N, ws, counts_dev);
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

size_t hist_tmp_bytes(int64_t N) { return round_up(N * 4, 256) * 2 + round_up(scan_tmp_bytes(N), 256); }

mbar_status build_histogram(const float2* d_pairs, const double* d_sorted, int64_t N, double w, int32_t* seg,
                            int32_t* start, int32_t* H, int64_t* keys, int32_t* nb_dev, void* tmp, size_t tmp_bytes,
                            cudaStream_t st) {
  if (tmp_bytes < hist_tmp_bytes(N)) {
    set_error("build_histogram: scratch too small");
    return MBAR_EINVAL;
  }
  unsigned char* p = static_cast<unsigned char*>(tmp);
  int* flags = reinterpret_cast<int*>(p);
  p += round_up(N * 4, 256);
  int* excl = reinterpret_cast<int*>(p);
  p += round_up(N * 4, 256);
  const unsigned gN = static_cast<unsigned>(ceil_div(N, kThreads));
  const RecipW rw = make_recip(w);
  head_flags<<<gN, kThreads, 0, st>>>(d_pairs, d_sorted, N, rw, flags);
  count_launches(1);
  BUMBAR_TRY(excl_scan(flags, N, excl, nullptr, p, st));
  finish_histogram<<<gN, kThreads, 0, st>>>(d_pairs, d_sorted, N, rw, flags, excl, seg, start, keys, nb_dev);
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  int32_t nb = 0;
  BUMBAR_CUDA(cudaMemcpyAsync(&nb, nb_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  BUMBAR_CUDA(cudaStreamSynchronize(st));
  counts_from_starts<<<static_cast<unsigned>(ceil_div(nb, kThreads)), kThreads, 0, st>>>(start, nb, H);
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

size_t bin_means_multi_tmp_bytes(int64_t K, int64_t N, int L, const int64_t* nb) {
  const int64_t ntiles = ceil_div(N, kBmTile);
  size_t b = 0;
  for (int l = 0; l < L; ++l) b += round_up(K * ntiles * 8, 256) * 2 + round_up(nb[l] * 8, 256);
  return b;
}

mbar_status bin_means_multi(const void* v, int dtype_bytes, int64_t K, int64_t N, int64_t ld, int L,
                            const int32_t* const* seg, const int32_t* const* start, const int64_t* nb,
                            void* const* out, const int64_t* ld_out, void* tmp, size_t tmp_bytes, cudaStream_t st) {
  if (L < 1 || L > kMaxLevels) {
    set_error("bin_means_multi: 1..%d levels", kMaxLevels);
    return MBAR_EINVAL;
  }
  if (tmp_bytes < bin_means_multi_tmp_bytes(K, N, L, nb)) {
    set_error("bin_means_multi: scratch too small");
    return MBAR_EINVAL;
  }
  const int64_t ntiles = ceil_div(N, kBmTile);
  // levels with small bins go to bin_means_fine (its own read of v); the
  // others share one bin_sums_multi pass
  std::vector<int> coarse;
  for (int l = 0; l < L; ++l) {
    if (static_cast<double>(N) / static_cast<double>(std::max<int64_t>(nb[l], 1)) <= kFineMaxMean) {
      const dim3 gf(static_cast<unsigned>(ceil_div(nb[l], kThreads)), static_cast<unsigned>(ceil_div(K, kFineRows)));
      if (dtype_bytes == 4)
        bin_means_fine<float><<<gf, kThreads, 0, st>>>(static_cast<const float*>(v), K, ld, start[l], nb[l],
                                                       static_cast<float*>(out[l]), ld_out[l]);
      else
        bin_means_fine<double><<<gf, kThreads, 0, st>>>(static_cast<const double*>(v), K, ld, start[l], nb[l],
                                                        static_cast<double*>(out[l]), ld_out[l]);
      count_launches(1);
    } else {
      coarse.push_back(l);
    }
  }
  if (coarse.empty()) {
    BUMBAR_CUDA(cudaGetLastError());
    return MBAR_OK;
  }
  MultiLevel ml{};
  ml.L = static_cast<int>(coarse.size());
  unsigned char* q = static_cast<unsigned char*>(tmp);
  for (int i = 0; i < ml.L; ++i) {
    const int l = coarse[i];
    LevelOut& o = ml.l[i];
    o.seg = seg[l];
    o.start = start[l];
    o.out = out[l];
    o.ld_out = ld_out[l];
    o.carry0 = q;  // sized for FP64 accumulators; FP32 data uses half
    q += round_up(K * ntiles * 8, 256);
    o.carry1 = q;
    q += round_up(K * ntiles * 8, 256);
    double* inv = reinterpret_cast<double*>(q);
    q += round_up(nb[l] * 8, 256);
    o.inv = inv;
    inverse_counts<<<static_cast<unsigned>(ceil_div(nb[l], kThreads)), kThreads, 0, st>>>(start[l], nb[l], inv);
    count_launches(1);
  }
  const dim3 g1(static_cast<unsigned>(ceil_div(ntiles, kThreads / 32)),
                static_cast<unsigned>(ceil_div(K, kBmRowsPerBlock)));
  const dim3 g2(static_cast<unsigned>(std::max<int64_t>(1, ceil_div(ntiles - 1, kFixWarps))),
                static_cast<unsigned>(ceil_div(K, 32)));
  auto launch = [&](auto tag) {
    using T = decltype(tag);
    const T* vv = static_cast<const T*>(v);
    switch (ml.L) {
      case 1: bin_sums_multi<T, 1><<<g1, kThreads, 0, st>>>(vv, K, N, ld, ml, ntiles); break;
      case 2: bin_sums_multi<T, 2><<<g1, kThreads, 0, st>>>(vv, K, N, ld, ml, ntiles); break;
      case 3: bin_sums_multi<T, 3><<<g1, kThreads, 0, st>>>(vv, K, N, ld, ml, ntiles); break;
      case 4: bin_sums_multi<T, 4><<<g1, kThreads, 0, st>>>(vv, K, N, ld, ml, ntiles); break;
      case 5: bin_sums_multi<T, 5><<<g1, kThreads, 0, st>>>(vv, K, N, ld, ml, ntiles); break;
      case 6: bin_sums_multi<T, 6><<<g1, kThreads, 0, st>>>(vv, K, N, ld, ml, ntiles); break;
      case 7: bin_sums_multi<T, 7><<<g1, kThreads, 0, st>>>(vv, K, N, ld, ml, ntiles); break;
      default: bin_sums_multi<T, 8><<<g1, kThreads, 0, st>>>(vv, K, N, ld, ml, ntiles); break;
    }
  };
  if (dtype_bytes == 4)
    launch(float{});
  else
    launch(double{});
  count_launches(1);
  for (int l = 0; l < ml.L; ++l) {
    const LevelOut& o = ml.l[l];
    if (dtype_bytes == 4)
      bin_sums_fixup<float><<<g2, kThreads, 0, st>>>(K, o.seg, o.start, o.inv, static_cast<float*>(o.out), o.ld_out,
                                                     static_cast<const float*>(o.carry0),
                                                     static_cast<const float*>(o.carry1), ntiles);
    else
      bin_sums_fixup<double><<<g2, kThreads, 0, st>>>(K, o.seg, o.start, o.inv, static_cast<double*>(o.out),
                                                      o.ld_out, static_cast<const double*>(o.carry0),
                                                      static_cast<const double*>(o.carry1), ntiles);
    count_launches(1);
  }
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

size_t bin_means_tmp_bytes(int64_t K, int64_t N) {
  const int64_t ntiles = ceil_div(N, kBmTile);
  return round_up(K * ntiles * 8, 256) * 2 + round_up(N * 8, 256);
}

mbar_status bin_means(const void* v, int dtype_bytes, int64_t K, int64_t N, int64_t ld, const int32_t* seg,
                      const int32_t* start, int64_t nb, void* out, int64_t ld_out, void* tmp, size_t tmp_bytes,
                      cudaStream_t st) {
  if (tmp_bytes < bin_means_tmp_bytes(K, N)) {
    set_error("bin_means: scratch too small");
    return MBAR_EINVAL;
  }
  const int64_t ntiles = ceil_div(N, kBmTile);
  double* carry0 = static_cast<double*>(tmp);
  double* carry1 = carry0 + round_up(K * ntiles, 32);
  double* inv = carry1 + round_up(K * ntiles, 32);
  inverse_counts<<<static_cast<unsigned>(ceil_div(nb, kThreads)), kThreads, 0, st>>>(start, nb, inv);
  count_launches(1);
  const dim3 g1(static_cast<unsigned>(ceil_div(ntiles, kThreads / 32)), static_cast<unsigned>(ceil_div(K, kBmRowsPerBlock)));
  const dim3 g2(static_cast<unsigned>(std::max<int64_t>(1, ceil_div(ntiles - 1, kFixWarps))),
                static_cast<unsigned>(ceil_div(K, 32)));
  if (dtype_bytes == 4) {
    float* c0f = reinterpret_cast<float*>(carry0);  // FP32 accumulators (the buffers fit FP64 ones)
    float* c1f = reinterpret_cast<float*>(carry1);
    bin_sums_block<float><<<g1, kThreads, 0, st>>>(static_cast<const float*>(v), K, N, ld, seg, start, inv,
                                                   static_cast<float*>(out), ld_out, c0f, c1f, ntiles);
    count_launches(1);
    bin_sums_fixup<float><<<g2, kThreads, 0, st>>>(K, seg, start, inv, static_cast<float*>(out), ld_out, c0f, c1f,
                                                   ntiles);
    count_launches(1);
  } else {
    bin_sums_block<double><<<g1, kThreads, 0, st>>>(static_cast<const double*>(v), K, N, ld, seg, start, inv,
                                                    static_cast<double*>(out), ld_out, carry0, carry1, ntiles);
    count_launches(1);
    bin_sums_fixup<double><<<g2, kThreads, 0, st>>>(K, seg, start, inv, static_cast<double*>(out), ld_out, carry0,
                                                    carry1, ntiles);
    count_launches(1);
  }
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

mbar_status gather_transpose(const void* vst, int dtype_bytes, int64_t K, int64_t N, const int32_t* perm, void* v,
                             int64_t ld, cudaStream_t st) {
  {
    std::lock_guard<std::recursive_mutex> lock(init_mutex());
    static bool init = false;
    if (!init) {
      int dev = 0, optin = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      cudaFuncSetAttribute(gather_transpose_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
      cudaFuncSetAttribute(gather_transpose_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
      init = true;
    }
  }
  if (dtype_bytes == 4) {
    const size_t smem = static_cast<size_t>(gt_cols<float>()) * gt_pitch<float>(K) * 4;
    gather_transpose_kernel<float><<<static_cast<unsigned>(ceil_div(N, gt_cols<float>())), kGtThreads, smem, st>>>(
        static_cast<const float*>(vst), K, N, perm, static_cast<float*>(v), ld);
  } else {
    const size_t smem = static_cast<size_t>(gt_cols<double>()) * gt_pitch<double>(K) * 8;
    gather_transpose_kernel<double><<<static_cast<unsigned>(ceil_div(N, gt_cols<double>())), kGtThreads, smem, st>>>(
        static_cast<const double*>(vst), K, N, perm, static_cast<double*>(v), ld);
  }
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

mbar_status gather_columns(const void* in, void* out, int dtype_bytes, int64_t K, int64_t N, int64_t ld,
                           const int32_t* perm, cudaStream_t st) {
  const dim3 g(static_cast<unsigned>(ceil_div(N, kThreads)), static_cast<unsigned>(ceil_div(K, kGatherRows)));
  if (dtype_bytes == 4) {
    gather_cols_kernel<float><<<g, kThreads, 0, st>>>(static_cast<const float*>(in), static_cast<float*>(out), K, N,
                                                      ld, perm);
    count_launches(1);
  } else {
    gather_cols_kernel<double><<<g, kThreads, 0, st>>>(static_cast<const double*>(in), static_cast<double*>(out), K,
                                                       N, ld, perm);
    count_launches(1);
  }
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

}  // namespace bumbar
