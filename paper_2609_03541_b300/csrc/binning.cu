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
#include <cstdio>

#include "common.cuh"
#include "kernels.cuh"

namespace bumbar {

namespace {

constexpr int kSortTile = 1024;  // elements per warp tile
constexpr int kScanBlock = 1024; // elements per block in the scan (256 threads x 4)
constexpr int kMaxWidths = 15;   // candidate widths per counting pass

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
  if (frac > delta && frac < 1.0f - delta) return static_cast<long long>(fl) + static_cast<long long>(fr);
  return static_cast<long long>(floor(__ddiv_rn(*d_exact, r.w)));
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

__global__ void count_heads_multi(const float2* __restrict__ dhl, const double* __restrict__ d, int64_t N,
                                  WidthSet ws, unsigned long long* __restrict__ counts) {
  __shared__ unsigned int cnt[kMaxWidths];
  if (threadIdx.x < kMaxWidths) cnt[threadIdx.x] = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t i0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) * kCountChunk;
  const int64_t i1 = (i0 + kCountChunk < N) ? i0 + kCountChunk : N;
  for (int c = 0; c < ws.n; ++c) {
    unsigned int heads = 0;
    if (i0 < N) {
      const RecipW r = ws.r[c];
      const float2 e = dhl[i1 - 1];
      const long long kend = key_df(e.x, e.y, r, d + i1 - 1);
      long long kprev;
      if (i0 == 0) {
        heads = 1;  // the first sample opens the first bin
        const float2 s0 = dhl[0];
        kprev = key_df(s0.x, s0.y, r, d);
      } else {
        const float2 sp = dhl[i0 - 1];
        kprev = key_df(sp.x, sp.y, r, d + i0 - 1);
      }
      const long long diff = kend - kprev;
      if (diff == 1) {
        heads += 1;
      } else if (diff > 1) {
        for (int64_t i = (i0 == 0 ? 1 : i0); i < i1; ++i) {
          const float2 x = dhl[i];
          const long long k = key_df(x.x, x.y, r, d + i);
          heads += (k != kprev) ? 1u : 0u;
          kprev = k;
        }
      }
    }
    for (int o = 16; o >= 1; o >>= 1) heads += __shfl_xor_sync(0xffffffffu, heads, o);
    if (lane == 0 && heads) atomicAdd(&cnt[c], heads);
  }
  __syncthreads();
  if (threadIdx.x < ws.n && cnt[threadIdx.x]) atomicAdd(&counts[threadIdx.x], static_cast<unsigned long long>(cnt[threadIdx.x]));
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
// A block owns a tile of 2048 sorted columns (256 threads x 8 consecutive
// columns) for kRowsPerBlock rows. Per row, each thread splits its 8 values
// into runs of equal bin ordinal; runs that start and end inside the thread
// are written at once; the last run of each thread enters a block-wide
// segmented inclusive scan (FP64) that carries it across thread boundaries.
// A bin whose run ends in a thread is finished there: written if the bin
// started in this tile, else its partial goes to carry0[tile] (a bin that
// began in an earlier tile). The last thread's still-open run goes to
// carry1[tile] (a bin that starts in this tile and continues) or, if it
// began before the tile, to carry0[tile]. A fix-up kernel finishes bins that
// span tiles: sum = carry1[first tile] + carry0[later tiles], in order.
constexpr int kBmCols = 8;
constexpr int kBmTile = kThreads * kBmCols;  // 2048
constexpr int kRowsPerBlock = 4;

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
                                                           int64_t ld_out, double* __restrict__ carry0,
                                                           double* __restrict__ carry1, int64_t ntiles) {
  using A = typename Acc<T>::type;
  __shared__ A wv[kThreads / 32];
  __shared__ int wf[kThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t tile = blockIdx.x;
  const int64_t tile0 = tile * kBmTile;
  const int64_t tile_end = (tile0 + kBmTile < N) ? tile0 + kBmTile : N;
  const int64_t c0 = tile0 + static_cast<int64_t>(tid) * kBmCols;
  const int nvalid = static_cast<int>(c0 < N ? ((N - c0) < kBmCols ? (N - c0) : kBmCols) : 0);
  const bool last_thread = nvalid > 0 && c0 + nvalid == tile_end;

  // run structure of this thread's columns (identical for every row)
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
  const bool flag = nvalid <= 0 || nruns > 0 || st_bl >= c0;  // last run starts in this thread
  const bool cont = nvalid > 0 && st_b0 < c0;                 // first run continues from the left
  const bool last_ends_here = nvalid > 0 && en_bl <= c0 + nvalid;
  const A inv_b0 = nvalid > 0 ? static_cast<A>(inv_count[b0]) : A(0);
  const A inv_bl = nvalid > 0 ? static_cast<A>(inv_count[bl]) : A(0);

  const int64_t k_begin = static_cast<int64_t>(blockIdx.y) * kRowsPerBlock;
  for (int64_t k = k_begin; k < K && k < k_begin + kRowsPerBlock; ++k) {
    A x[kBmCols];
    load8<T, A>(v + k * ld + c0, nvalid, x);
    // local runs
    A head = A(0), run = A(0);
    int cur = b0;
    bool first = true;
#pragma unroll
    for (int j = 0; j < kBmCols; ++j) {
      if (j < nvalid) {
        if (sg[j] != cur) {
          if (first) {
            head = run;
            first = false;
          } else {  // interior run: starts and ends inside this thread
            out[k * ld_out + cur] = static_cast<T>(run * static_cast<A>(inv_count[cur]));
          }
          cur = sg[j];
          run = A(0);
        }
        run += x[j];
      }
    }
    // block-wide segmented inclusive scan of the last-run sums
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
    if (lane == 31) {
      wv[warp] = sv;
      wf[warp] = sf;
    }
    __syncthreads();
    A pv = A(0);  // segmented prefix of all earlier warps
    for (int w = 0; w < warp; ++w) pv = wf[w] ? wv[w] : pv + wv[w];
    if (!sf) sv += pv;
    A prev = __shfl_up_sync(0xffffffffu, sv, 1);
    if (lane == 0) prev = pv;
    if (tid == 0) prev = A(0);
    __syncthreads();
    if (nvalid > 0) {
      const A carry_in = cont ? prev : A(0);
      if (nruns > 0) {  // the first run ends inside this thread
        const A tot = carry_in + head;
        if (st_b0 >= tile0)
          out[k * ld_out + b0] = static_cast<T>(tot * inv_b0);
        else
          carry0[k * ntiles + tile] = static_cast<double>(tot);
      }
      if (last_ends_here) {
        if (st_bl >= tile0)
          out[k * ld_out + bl] = static_cast<T>(sv * inv_bl);
        else
          carry0[k * ntiles + tile] = static_cast<double>(sv);
      } else if (last_thread) {
        if (st_bl >= tile0)
          carry1[k * ntiles + tile] = static_cast<double>(sv);
        else
          carry0[k * ntiles + tile] = static_cast<double>(sv);
      }
    }
  }
}

__global__ void inverse_counts(const int32_t* __restrict__ start, int64_t nb, double* __restrict__ inv) {
  const int64_t b = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (b < nb) inv[b] = 1.0 / static_cast<double>(start[b + 1] - start[b]);
}

template <typename T>
__global__ void bin_sums_fixup(int64_t K, int64_t nb, const int32_t* __restrict__ start,
                               const double* __restrict__ inv_count, T* __restrict__ out, int64_t ld_out,
                               const double* __restrict__ carry0, const double* __restrict__ carry1, int64_t ntiles) {
  const int64_t b = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t k = blockIdx.y;
  if (b >= nb) return;
  const int64_t s = start[b], e = start[b + 1];
  const int64_t ts = s / kBmTile, te = (e - 1) / kBmTile;
  if (ts == te) return;  // finished inside one tile
  double sum = carry1[k * ntiles + ts];
  for (int64_t t = ts + 1; t <= te; ++t) sum += carry0[k * ntiles + t];
  out[k * ld_out + b] = static_cast<T>(sum * inv_count[b]);
}

// out[k][i] = in[k][perm[i]]: each thread loads perm[i] once and moves it
// for 8 rows; blocks run row-group major so the 8 input rows being gathered
// stay in L2.
constexpr int kGatherRows = 8;
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
  count_heads_multi<<<static_cast<unsigned>(ceil_div(N, static_cast<int64_t>(kThreads) * kCountChunk)), kThreads, 0,
                      st>>>(d_pairs, d_sorted, N, ws, counts_dev);
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
  const dim3 g1(static_cast<unsigned>(ntiles), static_cast<unsigned>(ceil_div(K, kRowsPerBlock)));
  const dim3 g2(static_cast<unsigned>(ceil_div(nb, kThreads)), static_cast<unsigned>(K));
  if (dtype_bytes == 4) {
    bin_sums_block<float><<<g1, kThreads, 0, st>>>(static_cast<const float*>(v), K, N, ld, seg, start, inv,
                                                   static_cast<float*>(out), ld_out, carry0, carry1, ntiles);
    count_launches(1);
    bin_sums_fixup<float><<<g2, kThreads, 0, st>>>(K, nb, start, inv, static_cast<float*>(out), ld_out, carry0,
                                                   carry1, ntiles);
    count_launches(1);
  } else {
    bin_sums_block<double><<<g1, kThreads, 0, st>>>(static_cast<const double*>(v), K, N, ld, seg, start, inv,
                                                    static_cast<double*>(out), ld_out, carry0, carry1, ntiles);
    count_launches(1);
    bin_sums_fixup<double><<<g2, kThreads, 0, st>>>(K, nb, start, inv, static_cast<double*>(out), ld_out, carry0,
                                                    carry1, ntiles);
    count_launches(1);
  }
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
