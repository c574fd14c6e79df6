// Gauge-fixed Newton solve in FP64 on the device: the Hessian annihilates
// the all-ones vector (f is defined up to a constant), so state 0 is held
// fixed (delta_0 = 0) and the remaining (K-1) x (K-1) block, symmetric
// positive definite for connected data, is factored by a blocked
// right-looking Cholesky (32-wide panels: diagonal block in shared memory,
// panel triangular solve, trailing symmetric update) followed by forward
// and backward substitution. The same factor gives the asymptotic
// covariance of f (its inverse, column by column, minus the sample terms).
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "kernels.cuh"

namespace bumbar {

namespace {

constexpr int NB = 32;

__global__ void copy_reduced(const double* __restrict__ hess, int64_t K, const double* __restrict__ g,
                             double* __restrict__ A, double* __restrict__ b) {
  const int64_t m = K - 1;
  const int64_t i = blockIdx.x;
  for (int64_t j = threadIdx.x; j < m; j += blockDim.x) A[i * m + j] = hess[(i + 1) * K + (j + 1)];
  if (threadIdx.x == 0) b[i] = -g[i + 1];
}

__global__ void potrf_block(double* __restrict__ A, int64_t m, int64_t kb, int nb, int* info) {
  __shared__ double L[NB][NB + 1];
  const int t = threadIdx.x;
  const int r = t / NB, c = t % NB;
  if (r < nb && c < nb) L[r][c] = A[(kb + r) * m + kb + c];
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (t == 0) {
      const double d = L[j][j];
      if (!(d > 0.0) || !isfinite(d)) {
        atomicOr(info, 1);
        L[j][j] = 1.0;
      } else {
        L[j][j] = sqrt(d);
      }
    }
    __syncthreads();
    if (t > j && t < nb) L[t][j] /= L[j][j];
    __syncthreads();
    if (r > j && r < nb && c > j && c <= r) L[r][c] -= L[r][j] * L[c][j];
    __syncthreads();
  }
  if (r < nb && c < nb && c <= r) A[(kb + r) * m + kb + c] = L[r][c];
}

__global__ void trsm_panel(double* __restrict__ A, int64_t m, int64_t kb, int nb) {
  __shared__ double L[NB][NB + 1];
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    L[r][c] = (r < nb && c < nb && c <= r) ? A[(kb + r) * m + kb + c] : 0.0;
  }
  __syncthreads();
  const int64_t i = kb + nb + static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  __shared__ double rdiag[NB];
  if (threadIdx.x < NB) rdiag[threadIdx.x] = threadIdx.x < nb ? 1.0 / L[threadIdx.x][threadIdx.x] : 0.0;
  __syncthreads();
  if (i >= m) return;
  double y[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) y[j] = j < nb ? A[i * m + kb + j] : 0.0;  // independent loads first
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    if (j < nb) {
      double s = y[j];
      for (int l = 0; l < j; ++l) s -= y[l] * L[j][l];
      y[j] = s * rdiag[j];
    }
  }
#pragma unroll
  for (int j = 0; j < NB; ++j)
    if (j < nb) A[i * m + kb + j] = y[j];
}

__global__ void syrk_update(double* __restrict__ A, int64_t m, int64_t kb, int nb) {
  const int64_t base = kb + nb;
  const int ti = blockIdx.y, tj = blockIdx.x;
  if (tj > ti) return;
  __shared__ double Pi[NB][NB + 1];
  __shared__ double Pj[NB][NB + 1];
  const int r = threadIdx.x / NB, c = threadIdx.x % NB;  // 1024 threads
  const int64_t i = base + ti * NB + r, jr = base + tj * NB + r;
  Pi[r][c] = (i < m && c < nb) ? A[i * m + kb + c] : 0.0;
  Pj[r][c] = (jr < m && c < nb) ? A[jr * m + kb + c] : 0.0;
  __syncthreads();
  const int64_t j = base + tj * NB + c;
  if (i < m && j < m && j <= i) {
    double s = 0.0;
    for (int l = 0; l < nb; ++l) s += Pi[r][l] * Pj[c][l];
    A[i * m + j] -= s;
  }
}

// Single-block forward then backward substitution with the lower factor L,
// by 32-row panels: warp 0 solves the 32 x 32 triangle of a panel in
// registers (one row per lane, shuffles), then all threads apply the panel
// to the remaining right-hand side (a matrix-vector product).
__global__ void __launch_bounds__(1024) chol_solve(const double* __restrict__ A, int64_t m, double* __restrict__ b,
                                                   double* __restrict__ delta) {
  __shared__ double xs[NB];
  __shared__ double D[NB][NB + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // forward: L y = b
  for (int64_t j0 = 0; j0 < m; j0 += NB) {
    const int nb = static_cast<int>(m - j0 < NB ? m - j0 : NB);
    __syncthreads();
    // the diagonal block, loaded by all threads (no load latency in the
    // recurrence below)
    for (int e = tid; e < NB * NB; e += blockDim.x) {
      const int r = e / NB, cc = e % NB;
      D[r][cc] = (r < nb && cc < nb) ? A[(j0 + r) * m + j0 + cc] : 0.0;
    }
    __syncthreads();
    if (warp == 0) {
      double rhs = lane < nb ? b[j0 + lane] : 0.0;
      double y = 0.0;
      const double rd = lane < nb ? 1.0 / D[lane][lane] : 0.0;
      for (int j = 0; j < nb; ++j) {
        const double yj = __shfl_sync(0xffffffffu, rhs * rd, j);
        if (lane == j) y = yj;
        if (lane > j && lane < nb) rhs -= D[lane][j] * yj;
      }
      if (lane < nb) {
        xs[lane] = y;
        b[j0 + lane] = y;
      }
    }
    __syncthreads();
    for (int64_t i = j0 + nb + tid; i < m; i += blockDim.x) {
      double s = 0.0;
      for (int j = 0; j < nb; ++j) s += A[i * m + j0 + j] * xs[j];
      b[i] -= s;
    }
  }
  // backward: L^T x = y
  for (int64_t j1 = m; j1 > 0; j1 -= NB) {
    const int64_t j0 = j1 - NB > 0 ? j1 - NB : 0;
    const int nb = static_cast<int>(j1 - j0);
    __syncthreads();
    for (int e = tid; e < NB * NB; e += blockDim.x) {
      const int r = e / NB, cc = e % NB;
      D[r][cc] = (r < nb && cc < nb) ? A[(j0 + r) * m + j0 + cc] : 0.0;
    }
    __syncthreads();
    if (warp == 0) {
      double rhs = lane < nb ? b[j0 + lane] : 0.0;
      double x = 0.0;
      const double rd = lane < nb ? 1.0 / D[lane][lane] : 0.0;
      for (int j = nb - 1; j >= 0; --j) {
        const double xj = __shfl_sync(0xffffffffu, rhs * rd, j);
        if (lane == j) x = xj;
        if (lane < j) rhs -= D[j][lane] * xj;
      }
      if (lane < nb) {
        xs[lane] = x;
        b[j0 + lane] = x;
      }
    }
    __syncthreads();
    for (int64_t i = tid; i < j0; i += blockDim.x) {
      double s = 0.0;
      for (int j = 0; j < nb; ++j) s += A[(j0 + j) * m + i] * xs[j];
      b[i] -= s;
    }
  }
  __syncthreads();
  for (int64_t i = tid; i < m; i += blockDim.x) delta[i + 1] = b[i];
  if (tid == 0) delta[0] = 0.0;
}

// Columns of the inverse of A = L L^T (L: lower factor in the lower triangle
// of the m x m row-major `A`), one CTA per column j: forward substitution of
// e_j (column-oriented: each step scales y_i and updates the rows below it),
// then backward substitution with L^T (row-oriented: row i of L is column i
// of L^T). X[:, j] = A^{-1} e_j.
constexpr int kInvThreads = 256;
__global__ void __launch_bounds__(kInvThreads) chol_inverse_cols(const double* __restrict__ A, int64_t m,
                                                                 double* __restrict__ X) {
  __shared__ double y[1024];
  const int64_t j = blockIdx.x;
  const int tid = threadIdx.x;
  for (int64_t i = tid; i < m; i += kInvThreads) y[i] = (i == j) ? 1.0 : 0.0;
  __syncthreads();
  // L y = e_j (y_i = 0 for i < j)
  for (int64_t i = j; i < m; ++i) {
    const double yi = y[i] / A[i * m + i];
    __syncthreads();  // every thread has read y[i]
    if (tid == 0) y[i] = yi;
    for (int64_t r = i + 1 + tid; r < m; r += kInvThreads) y[r] -= A[r * m + i] * yi;
    __syncthreads();
  }
  // L^T x = y
  for (int64_t i = m - 1; i >= 0; --i) {
    const double xi = y[i] / A[i * m + i];
    __syncthreads();
    if (tid == 0) y[i] = xi;
    for (int64_t r = tid; r < i; r += kInvThreads) y[r] -= A[i * m + r] * xi;
    __syncthreads();
  }
  for (int64_t i = tid; i < m; i += kInvThreads) X[i * m + j] = y[i];
}

// cov(f_i - f_0, f_j - f_0) = [H_red^-1]_(i-1)(j-1) - delta_ij / N_i - 1 / N_0
// for i, j >= 1; row and column 0 are 0 (the gauge).
__global__ void covariance_from_inverse(const double* __restrict__ X, int64_t K, const double* __restrict__ Nk,
                                        double* __restrict__ cov) {
  const int64_t i = blockIdx.x;
  const int64_t m = K - 1;
  for (int64_t j = threadIdx.x; j < K; j += blockDim.x) {
    double v = 0.0;
    if (i > 0 && j > 0) v = X[(i - 1) * m + (j - 1)] - (i == j ? 1.0 / Nk[i] : 0.0) - 1.0 / Nk[0];
    cov[i * K + j] = v;
  }
}

// Blocked right-looking Cholesky of the m x m row-major A in place.
void factor_blocked(double* A, int64_t m, int* info, cudaStream_t st) {
  for (int64_t kb = 0; kb < m; kb += NB) {
    const int nb = static_cast<int>(std::min<int64_t>(NB, m - kb));
    potrf_block<<<1, NB * NB, 0, st>>>(A, m, kb, nb, info);
    count_launches(1);
    const int64_t rest = m - kb - nb;
    if (rest > 0) {
      trsm_panel<<<static_cast<unsigned>(ceil_div(rest, 128)), 128, 0, st>>>(A, m, kb, nb);
      count_launches(1);
      const unsigned nt = static_cast<unsigned>(ceil_div(rest, NB));
      syrk_update<<<dim3(nt, nt), NB * NB, 0, st>>>(A, m, kb, nb);
      count_launches(1);
    }
  }
}

}  // namespace

size_t covariance_tmp_bytes(int64_t K) {
  const int64_t m = std::max<int64_t>(K - 1, 1);
  return 2 * round_up(m * m * 8, 256) + round_up(K * 8, 256) + 256;
}

mbar_status covariance(const double* hess, int64_t K, const double* Nk, double* cov, int* info, void* tmp,
                       size_t tmp_bytes, cudaStream_t st) {
  if (K == 1) {
    BUMBAR_CUDA(cudaMemsetAsync(cov, 0, sizeof(double), st));
    return MBAR_OK;
  }
  if (K > 1024 || tmp_bytes < covariance_tmp_bytes(K)) {
    set_error("covariance: K > 1024 or scratch too small");
    return MBAR_EINVAL;
  }
  const int64_t m = K - 1;
  double* A = static_cast<double*>(tmp);
  double* X = reinterpret_cast<double*>(static_cast<unsigned char*>(tmp) + round_up(m * m * 8, 256));
  double* b = reinterpret_cast<double*>(static_cast<unsigned char*>(tmp) + 2 * round_up(m * m * 8, 256));
  // copy_reduced's right-hand side is not needed here (b gets -hess[1..K-1]
  // and is ignored)
  copy_reduced<<<static_cast<unsigned>(m), kThreads, 0, st>>>(hess, K, hess, A, b);
  count_launches(1);
  factor_blocked(A, m, info, st);
  chol_inverse_cols<<<static_cast<unsigned>(m), kInvThreads, 0, st>>>(A, m, X);
  covariance_from_inverse<<<static_cast<unsigned>(K), kThreads, 0, st>>>(X, K, Nk, cov);
  count_launches(2);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

size_t newton_tmp_bytes(int64_t K) { return round_up((K - 1) * (K - 1) * 8, 256) + round_up(K * 8, 256) + 256; }

mbar_status newton_solve(double* hess, int64_t K, const double* g, double* delta, int* info, void* tmp,
                         size_t tmp_bytes, cudaStream_t st) {
  if (K == 1) {
    BUMBAR_CUDA(cudaMemsetAsync(delta, 0, sizeof(double), st));
    return MBAR_OK;
  }
  if (tmp_bytes < newton_tmp_bytes(K)) {
    set_error("newton_solve: scratch too small");
    return MBAR_EINVAL;
  }
  const int64_t m = K - 1;
  double* A = static_cast<double*>(tmp);
  double* b = reinterpret_cast<double*>(static_cast<unsigned char*>(tmp) + round_up(m * m * 8, 256));
  copy_reduced<<<static_cast<unsigned>(m), kThreads, 0, st>>>(hess, K, g, A, b);
  count_launches(1);
  factor_blocked(A, m, info, st);
  chol_solve<<<1, 1024, 0, st>>>(A, m, b, delta);
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

}  // namespace bumbar
