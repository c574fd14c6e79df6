// Newton Hessian of the MBAR objective on the current columns (samples or
// bins with counts H_p):
//     H_ij = delta_ij sum_p H_p P_ip - sum_p H_p P_ip P_jp,
//     P_ip = N_i W_ip = exp(f_i + log N_i - v_ip - logden_p).
// Because sum_j P_jp = 1 for every column, the row sums of the overlap
// matrix G_ij = sum_p H_p P_ip P_jp equal the diagonal term, so
//     H = L(G):  H_ij = -G_ij (i != j),  H_ii = sum_{j != i} G_ij,
// which avoids the cancellation of diag(Q) - G on the diagonal and keeps the
// gauge null vector exact. G is the contraction; this file holds the
// CUDA-core path (used for small K) and the shared reduction/assembly; the
// tensor-core path for larger K lives in hessian_tc.cu.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "kernels.cuh"

namespace bumbar {

namespace {

constexpr int kTile = 64;   // output tile edge
constexpr int kChunk = 32;  // columns per shared-memory chunk

__host__ __device__ inline void pair_of(int idx, int nt, int* ti, int* tj) {
  // idx enumerates (ti <= tj) row-major over ti
  int t = 0;
  while (idx >= nt - t) {
    idx -= nt - t;
    ++t;
  }
  *ti = t;
  *tj = t + idx;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) overlap_simt(const T* __restrict__ v, int64_t K, int64_t n, int64_t ld,
                                                         const double* __restrict__ f, const double* __restrict__ logN,
                                                         const T* __restrict__ logden, const int32_t* __restrict__ H,
                                                         int nt, int64_t cols_per_slice, float* __restrict__ out) {
  __shared__ __align__(16) float Pi[kChunk][kTile];
  __shared__ __align__(16) float Pj[kChunk][kTile];
  __shared__ double a_s[2 * kTile];
  int ti, tj;
  pair_of(blockIdx.x, nt, &ti, &tj);
  const int tid = threadIdx.x;
  const int i0 = ti * kTile, j0 = tj * kTile;
  for (int r = tid; r < 2 * kTile; r += kThreads) {
    const int64_t k = (r < kTile) ? i0 + r : j0 + (r - kTile);
    a_s[r] = (k < K) ? f[k] + logN[k] : 0.0;
  }
  __syncthreads();
  const int64_t c_begin = static_cast<int64_t>(blockIdx.y) * cols_per_slice;
  const int64_t c_end = (c_begin + cols_per_slice < n) ? c_begin + cols_per_slice : n;
  const int ty = tid / 16, tx = tid % 16;
  float acc[4][4] = {};
  for (int64_t c0 = c_begin; c0 < c_end; c0 += kChunk) {
    // build P for rows of both tiles, 32 columns
    for (int e = tid; e < 2 * kTile * kChunk; e += kThreads) {
      const int r = e / kChunk, c = e % kChunk;
      const int64_t col = c0 + c;
      const int64_t k = (r < kTile) ? i0 + r : j0 + (r - kTile);
      float pv = 0.f;
      if (col < c_end && k < K) {
        if constexpr (sizeof(T) == 4) {
          const float x = static_cast<float>(a_s[r]) - v[k * ld + col] - logden[col];
          const float h = H ? static_cast<float>(H[col]) : 1.f;
          pv = ex2_approx(x * kLog2e) * sqrtf(h);
        } else {
          const double x = a_s[r] - v[k * ld + col] - logden[col];
          const double h = H ? static_cast<double>(H[col]) : 1.0;
          pv = static_cast<float>(exp(x) * sqrt(h));
        }
      }
      if (r < kTile)
        Pi[c][r] = pv;
      else
        Pj[c][r - kTile] = pv;
    }
    __syncthreads();
#pragma unroll 8
    for (int c = 0; c < kChunk; ++c) {
      const float4 a = *reinterpret_cast<const float4*>(&Pi[c][ty * 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Pj[c][tx * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w};
      const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(av[x], bv[y], acc[x][y]);
    }
    __syncthreads();
  }
  float* o = out + (static_cast<int64_t>(blockIdx.y) * gridDim.x + blockIdx.x) * kTile * kTile;
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) o[(ty * 4 + x) * kTile + tx * 4 + y] = acc[x][y];
}

// Sum the per-slice tiles (fixed order, FP64) into the symmetric G.
__global__ void reduce_tiles(const float* __restrict__ part, int nslices, int npairs, int nt, int64_t K,
                             double* __restrict__ G) {
  int ti, tj;
  pair_of(blockIdx.x, nt, &ti, &tj);
  for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
    double s = 0.0;
    for (int sl = 0; sl < nslices; ++sl) s += part[(static_cast<int64_t>(sl) * npairs + blockIdx.x) * kTile * kTile + e];
    const int64_t i = ti * kTile + e / kTile, j = tj * kTile + e % kTile;
    if (i < K && j < K) {
      G[i * K + j] = s;
      G[j * K + i] = s;
    }
  }
}

}  // namespace

// H = L(G): off-diagonal -G, diagonal = sum of the row's off-diagonal G.
__global__ void laplacian_from_overlap(const double* __restrict__ G, int64_t K, double* __restrict__ hess) {
  const int64_t i = blockIdx.x;
  __shared__ double red[kThreads / 32];
  double s = 0.0;
  for (int64_t j = threadIdx.x; j < K; j += blockDim.x) {
    const double g = G[i * K + j];
    if (j != i) {
      s += g;
      hess[i * K + j] = -g;
    }
  }
  for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    hess[i * K + i] = t;
  }
}

// a_k = f_k + log N_k for the tensor-core path
__global__ void add_vectors(const double* __restrict__ x, const double* __restrict__ y, double* __restrict__ out,
                            int64_t K) {
  const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k < K) out[k] = x[k] + y[k];
}

static int g_hessian_path = 0;
void set_hessian_path(int path) { g_hessian_path = path; }
// Automatic choice: tensor cores from K = 64 for FP64 data (below that the
// CUDA-core kernel's FP32 products keep Newton quadratic to f_tol = 1e-10),
// from K = 16 for FP32 data (MIXED, f_tol 1e-5; on the parallel-tempering
// shape, K = 50 and N = 1e7, the CUDA-core overlap took 8.8 ms per Hessian)
int hessian_path_for(int64_t K, int dtype_bytes) {
  if (g_hessian_path == 1 || g_hessian_path == 2) return g_hessian_path;
  if (g_hessian_path == 3) return 2;
  return K >= (dtype_bytes == 4 ? 16 : 64) ? 2 : 1;
}
bool tc_cluster_enabled() { return g_hessian_path != 3; }

struct SimtPlan {
  int nt, npairs, nslices;
  int64_t cols_per_slice;
};

static SimtPlan simt_plan(int64_t K, int64_t n) {
  SimtPlan p;
  p.nt = static_cast<int>(ceil_div(K, kTile));
  p.npairs = p.nt * (p.nt + 1) / 2;
  const int64_t target = 2 * static_cast<int64_t>(num_sms());
  int64_t s = std::max<int64_t>(1, ceil_div(target, p.npairs));
  s = std::min<int64_t>(s, std::max<int64_t>(1, ceil_div(n, 4 * kChunk)));
  p.cols_per_slice = round_up(ceil_div(n, s), kChunk);
  p.nslices = static_cast<int>(ceil_div(n, p.cols_per_slice));
  return p;
}

size_t hessian_tmp_bytes(int64_t K, int64_t n) {
  const SimtPlan p = simt_plan(K, n);
  const size_t simt = round_up(static_cast<int64_t>(p.nslices) * p.npairs * kTile * kTile * 4, 256);
  const size_t tc = overlap_tc_tmp_bytes(K, n) + round_up(K * 8, 256);
  return std::max(simt, tc) + round_up(K * K * 8, 256);
}

bool hessian_smaj_eligible(int64_t K) { return hessian_path_for(K, 4) == 2 && overlap_tc_smaj_eligible(K); }

mbar_status hessian_smaj(const float* vst, int64_t K, int64_t n, const double* f, const double* logN,
                         const float* logden, double* hess, unsigned* err, void* tmp, size_t tmp_bytes,
                         cudaStream_t st) {
  if (tmp_bytes < hessian_tmp_bytes(K, n)) {
    set_error("hessian: scratch too small");
    return MBAR_EINVAL;
  }
  const SimtPlan p = simt_plan(K, n);
  const size_t simt = round_up(static_cast<int64_t>(p.nslices) * p.npairs * kTile * kTile * 4, 256);
  const size_t tc = overlap_tc_tmp_bytes(K, n) + round_up(K * 8, 256);
  double* G = reinterpret_cast<double*>(static_cast<unsigned char*>(tmp) + std::max(simt, tc));
  double* a = static_cast<double*>(tmp);
  unsigned char* rest = static_cast<unsigned char*>(tmp) + round_up(K * 8, 256);
  add_vectors<<<static_cast<unsigned>(ceil_div(K, 256)), 256, 0, st>>>(f, logN, a, K);
  count_launches(1);
  BUMBAR_TRY(overlap_tc_smaj(vst, K, n, a, logden, G, err, rest, overlap_tc_tmp_bytes(K, n), st));
  laplacian_from_overlap<<<static_cast<unsigned>(K), kThreads, 0, st>>>(G, K, hess);
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

mbar_status hessian_fact(const double* fa, const double* fb, const double* fphi, int64_t K, int64_t n,
                         const double* f, const double* logN, const double* logden, double* hess, unsigned* err,
                         void* tmp, size_t tmp_bytes, cudaStream_t st) {
  if (tmp_bytes < hessian_tmp_bytes(K, n)) {
    set_error("hessian: scratch too small");
    return MBAR_EINVAL;
  }
  const SimtPlan p = simt_plan(K, n);
  const size_t simt = round_up(static_cast<int64_t>(p.nslices) * p.npairs * kTile * kTile * 4, 256);
  const size_t tc = overlap_tc_tmp_bytes(K, n) + round_up(K * 8, 256);
  double* G = reinterpret_cast<double*>(static_cast<unsigned char*>(tmp) + std::max(simt, tc));
  double* a = static_cast<double*>(tmp);
  unsigned char* rest = static_cast<unsigned char*>(tmp) + round_up(K * 8, 256);
  add_vectors<<<static_cast<unsigned>(ceil_div(K, 256)), 256, 0, st>>>(f, logN, a, K);
  count_launches(1);
  BUMBAR_TRY(overlap_tc_fact(fa, fb, fphi, K, n, a, logden, G, err, rest, overlap_tc_tmp_bytes(K, n), st));
  laplacian_from_overlap<<<static_cast<unsigned>(K), kThreads, 0, st>>>(G, K, hess);
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

mbar_status hessian(const void* v, int dtype_bytes, int64_t K, int64_t n, int64_t ld, const double* f,
                    const double* logN, const void* logden, const int32_t* H, double* hess, unsigned* err,
                    void* tmp, size_t tmp_bytes, cudaStream_t st) {
  if (tmp_bytes < hessian_tmp_bytes(K, n)) {
    set_error("hessian: scratch too small");
    return MBAR_EINVAL;
  }
  const SimtPlan p = simt_plan(K, n);
  const size_t simt = round_up(static_cast<int64_t>(p.nslices) * p.npairs * kTile * kTile * 4, 256);
  const size_t tc = overlap_tc_tmp_bytes(K, n) + round_up(K * 8, 256);
  double* G = reinterpret_cast<double*>(static_cast<unsigned char*>(tmp) + std::max(simt, tc));
  if (hessian_path_for(K, dtype_bytes) == 2) {
    double* a = static_cast<double*>(tmp);
    unsigned char* rest = static_cast<unsigned char*>(tmp) + round_up(K * 8, 256);
    add_vectors<<<static_cast<unsigned>(ceil_div(K, 256)), 256, 0, st>>>(f, logN, a, K);
    count_launches(1);
    BUMBAR_TRY(overlap_tc(v, dtype_bytes, K, n, ld, a, logden, H, G, err, rest, overlap_tc_tmp_bytes(K, n), st));
    laplacian_from_overlap<<<static_cast<unsigned>(K), kThreads, 0, st>>>(G, K, hess);
    count_launches(1);
    BUMBAR_CUDA(cudaGetLastError());
    return MBAR_OK;
  }
  float* part = static_cast<float*>(tmp);
  const dim3 grid(p.npairs, p.nslices);
  if (dtype_bytes == 4) {
    overlap_simt<float><<<grid, kThreads, 0, st>>>(static_cast<const float*>(v), K, n, ld, f, logN,
                                                   static_cast<const float*>(logden), H, p.nt, p.cols_per_slice, part);
    count_launches(1);
  } else {
    overlap_simt<double><<<grid, kThreads, 0, st>>>(static_cast<const double*>(v), K, n, ld, f, logN,
                                                    static_cast<const double*>(logden), H, p.nt, p.cols_per_slice,
                                                    part);
    count_launches(1);
  }
  reduce_tiles<<<p.npairs, kThreads, 0, st>>>(part, p.nslices, p.npairs, p.nt, K, G);
  count_launches(1);
  laplacian_from_overlap<<<static_cast<unsigned>(K), kThreads, 0, st>>>(G, K, hess);
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

}  // namespace bumbar
