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

__device__ __forceinline__ unsigned long long order_key(double x) {
  unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ long long bin_index(double phi, double lo, double w) {
  const double q = __ddiv_rn(__dsub_rn(phi, lo), w);
  return static_cast<long long>(floor(q));
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
__global__ void count_heads(const double* __restrict__ phi, int64_t N, double w,
                            unsigned long long* __restrict__ count) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const double lo = phi[0];
  long long key = 0;
  if (i < N) key = bin_index(phi[i], lo, w);
  long long prev = __shfl_up_sync(0xffffffffu, key, 1);
  if ((threadIdx.x & 31) == 0 && i > 0 && i < N) prev = bin_index(phi[i - 1], lo, w);
  const int head = (i < N) && (i == 0 || key != prev);
  const int n = __syncthreads_count(head);
  if (threadIdx.x == 0 && n) atomicAdd(count, static_cast<unsigned long long>(n));
}

__global__ void head_flags(const double* __restrict__ phi, int64_t N, double w, int* __restrict__ flags) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const double lo = phi[0];
  long long key = 0;
  if (i < N) key = bin_index(phi[i], lo, w);
  long long prev = __shfl_up_sync(0xffffffffu, key, 1);
  if ((threadIdx.x & 31) == 0 && i > 0 && i < N) prev = bin_index(phi[i - 1], lo, w);
  if (i < N) flags[i] = (i == 0 || key != prev) ? 1 : 0;
}

__global__ void finish_histogram(const double* __restrict__ phi, int64_t N, double w, const int* __restrict__ flags,
                                 const int* __restrict__ excl, int32_t* __restrict__ seg, int32_t* __restrict__ start,
                                 int64_t* __restrict__ keys, int32_t* __restrict__ nb_dev) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int f = flags[i];
  const int e = excl[i];
  seg[i] = e + f - 1;
  if (f) {
    start[e] = static_cast<int32_t>(i);
    keys[e] = bin_index(phi[i], phi[0], w);
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
// binned means: each thread walks one (row, tile of TW sorted columns)
// ---------------------------------------------------------------------------
template <typename T, int TW>
__global__ void bin_means_tiles(const T* __restrict__ v, int64_t K, int64_t N, int64_t ld,
                                const int32_t* __restrict__ seg, const int32_t* __restrict__ start,
                                T* __restrict__ out, int64_t ld_out, double* __restrict__ part0,
                                double* __restrict__ part1, int64_t ntiles) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t k = blockIdx.y;
  if (t >= ntiles) return;
  const int64_t c0 = t * TW;
  const int64_t c1 = (c0 + TW < N) ? c0 + TW : N;
  const T* row = v + k * ld;
  int cur = seg[c0];
  double sum = 0.0;
  bool first_run = true;
  double p0 = 0.0, p1 = 0.0;
  for (int64_t c = c0; c < c1; ++c) {
    const int s = seg[c];
    if (s != cur) {
      // run of bin `cur` ends at column c-1 inside this tile
      const bool starts_here = start[cur] >= c0;
      if (starts_here) {
        out[k * ld_out + cur] = static_cast<T>(sum / static_cast<double>(start[cur + 1] - start[cur]));
      } else {
        p0 = sum;  // first run, bin began in an earlier tile
      }
      first_run = false;
      cur = s;
      sum = 0.0;
    }
    sum += static_cast<double>(row[c]);
  }
  // last run of the tile
  const bool starts_here = start[cur] >= c0;
  const bool ends_here = start[cur + 1] <= c1;
  if (starts_here && ends_here) {
    out[k * ld_out + cur] = static_cast<T>(sum / static_cast<double>(start[cur + 1] - start[cur]));
  } else if (first_run) {
    p0 = sum;  // the only run of the tile, cut on at least one side
  } else {
    p1 = sum;  // last run, continues into the next tile
  }
  part0[k * ntiles + t] = p0;
  part1[k * ntiles + t] = p1;
}

template <typename T, int TW>
__global__ void bin_means_fixup(int64_t K, int64_t nb, const int32_t* __restrict__ start, T* __restrict__ out,
                                int64_t ld_out, const double* __restrict__ part0, const double* __restrict__ part1,
                                int64_t ntiles) {
  const int64_t b = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t k = blockIdx.y;
  if (b >= nb) return;
  const int64_t s = start[b], e = start[b + 1];
  const int64_t ts = s / TW, te = (e - 1) / TW;
  if (ts == te) return;  // complete inside one tile, written by the tile pass
  const double* p0 = part0 + k * ntiles;
  const double* p1 = part1 + k * ntiles;
  double sum = (s == ts * TW) ? p0[ts] : p1[ts];
  for (int64_t t = ts + 1; t <= te; ++t) sum += p0[t];
  out[k * ld_out + b] = static_cast<T>(sum / static_cast<double>(e - s));
}

template <typename T>
__global__ void gather_cols_kernel(const T* __restrict__ in, T* __restrict__ out, int64_t N, int64_t ld,
                                   const int32_t* __restrict__ perm) {
  const int64_t k = blockIdx.y;
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < N) out[k * ld + i] = in[k * ld + perm[i]];
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

mbar_status count_bins(const double* phi_sorted, int64_t N, double w, unsigned long long* count_dev,
                       cudaStream_t st) {
  BUMBAR_CUDA(cudaMemsetAsync(count_dev, 0, sizeof(unsigned long long), st));
  count_heads<<<static_cast<unsigned>(ceil_div(N, kThreads)), kThreads, 0, st>>>(phi_sorted, N, w, count_dev);
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

size_t hist_tmp_bytes(int64_t N) { return round_up(N * 4, 256) * 2 + round_up(scan_tmp_bytes(N), 256); }

mbar_status build_histogram(const double* phi_sorted, int64_t N, double w, int32_t* seg, int32_t* start, int32_t* H,
                            int64_t* keys, int32_t* nb_dev, void* tmp, size_t tmp_bytes, cudaStream_t st) {
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
  head_flags<<<gN, kThreads, 0, st>>>(phi_sorted, N, w, flags);
  count_launches(1);
  BUMBAR_TRY(excl_scan(flags, N, excl, nullptr, p, st));
  finish_histogram<<<gN, kThreads, 0, st>>>(phi_sorted, N, w, flags, excl, seg, start, keys, nb_dev);
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

static constexpr int kTileF32 = 64;
static constexpr int kTileF64 = 32;

size_t bin_means_tmp_bytes(int64_t K, int64_t N) {
  const int64_t ntiles = ceil_div(N, kTileF64);  // the larger tile count of the two
  return round_up(K * ntiles * 8, 256) * 2;
}

mbar_status bin_means(const void* v, int dtype_bytes, int64_t K, int64_t N, int64_t ld, const int32_t* seg,
                      const int32_t* start, int64_t nb, void* out, int64_t ld_out, void* tmp, size_t tmp_bytes,
                      cudaStream_t st) {
  if (tmp_bytes < bin_means_tmp_bytes(K, N)) {
    set_error("bin_means: scratch too small");
    return MBAR_EINVAL;
  }
  const int TW = dtype_bytes == 4 ? kTileF32 : kTileF64;
  const int64_t ntiles = ceil_div(N, TW);
  double* part0 = static_cast<double*>(tmp);
  double* part1 = part0 + round_up(K * ntiles, 32);
  const dim3 g1(static_cast<unsigned>(ceil_div(ntiles, kThreads)), static_cast<unsigned>(K));
  const dim3 g2(static_cast<unsigned>(ceil_div(nb, kThreads)), static_cast<unsigned>(K));
  if (dtype_bytes == 4) {
    bin_means_tiles<float, kTileF32><<<g1, kThreads, 0, st>>>(static_cast<const float*>(v), K, N, ld, seg, start,
                                                              static_cast<float*>(out), ld_out, part0, part1, ntiles);
    count_launches(1);
    bin_means_fixup<float, kTileF32><<<g2, kThreads, 0, st>>>(K, nb, start, static_cast<float*>(out), ld_out, part0,
                                                              part1, ntiles);
    count_launches(1);
  } else {
    bin_means_tiles<double, kTileF64><<<g1, kThreads, 0, st>>>(static_cast<const double*>(v), K, N, ld, seg, start,
                                                               static_cast<double*>(out), ld_out, part0, part1,
                                                               ntiles);
    count_launches(1);
    bin_means_fixup<double, kTileF64><<<g2, kThreads, 0, st>>>(K, nb, start, static_cast<double*>(out), ld_out, part0,
                                                               part1, ntiles);
    count_launches(1);
  }
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

mbar_status gather_columns(const void* in, void* out, int dtype_bytes, int64_t K, int64_t N, int64_t ld,
                           const int32_t* perm, cudaStream_t st) {
  const dim3 g(static_cast<unsigned>(ceil_div(N, kThreads)), static_cast<unsigned>(K));
  if (dtype_bytes == 4) {
    gather_cols_kernel<float><<<g, kThreads, 0, st>>>(static_cast<const float*>(in), static_cast<float*>(out), N, ld,
                                                      perm);
    count_launches(1);
  } else {
    gather_cols_kernel<double><<<g, kThreads, 0, st>>>(static_cast<const double*>(in), static_cast<double*>(out), N,
                                                       ld, perm);
    count_launches(1);
  }
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

}  // namespace bumbar
