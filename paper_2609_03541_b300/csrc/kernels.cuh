// Internal kernel interfaces of the BU-MBAR library (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace bumbar {

// Device control block of the iteration driver (one per context).
struct Ctrl {
  int done;       // first loop of Algorithm 1: set when s < eps
  int nonfinite;  // an update produced a non-finite f
  int iters;      // SCI steps executed by the guarded kernels
  int underflow;  // an SCI step found Q_k below 1e-20 N_k (its linear-domain sum lost the state): f kept
  double last_s;  // relative step (Eq. 2) of the last SCI step
};

constexpr int kLseModePass = 0;  // Q (and logden) only
constexpr int kLseModeSci = 1;   // + Eq. 1 update, gauge, gradient, Eq. 2

struct LseParams {
  int K, n;
  int num_strips, box_rows, nbox, stages;  // filled by lse_launch from the plan
  const double* f;                         // [K] current f
  const double* logN;                      // [K]
  const int32_t* H;                        // [n] counts or nullptr (all ones)
  double* partials;                        // [grid x K] scratch
  double* epi;                             // scratch after the partials: new f [K], then per-CTA (s, d, finite)
  int nparts;                              // CTAs of the pass (rows of partials); set by lse_launch
  unsigned* counter;                       // scratch: completion counter of the epilogue (zero between passes)
  unsigned* err;                           // scratch: timeout count
  double* Q;                               // [K] out
  void* logden;                            // [n] out (dtype of v) or nullptr
  int mode;
  // SCI epilogue
  const double* Nk;  // [K] sample counts as doubles
  double* f_out;     // [K]
  double* g_out;     // [K] or nullptr
  double* s_out;     // scalar or nullptr
  double* d_out;     // scalar or nullptr: max_k |f_out_k - (f_k - f_0)|
  Ctrl* ctrl;        // or nullptr
  double eps;        // > 0: set ctrl->done when s < eps
  double noise;      // > 0: set ctrl->done when max|f_out - f| < noise
  int skip_if_done;  // return at once if ctrl->done
  int skip_if_underflow;  // return at once if ctrl->underflow (SCI steps after an underflowed one)
  int exact_max;          // sample-major FP32 pass: split each sample's largest weight into an exact
                          // count and its remainder (the gradient's bias on poorly overlapping states)
};

// The guard every LSE pass kernel and its epilogue apply first.
__device__ __forceinline__ bool lse_skip(const LseParams& p) {
  return p.ctrl != nullptr && ((p.skip_if_done && p.ctrl->done) || (p.skip_if_underflow && p.ctrl->underflow));
}

struct LsePlan {
  int C, num_strips, box_rows, nbox, stages, grid, threads;
  int variant;  // 0 = tiled (lse.cu), 1 = register-resident (lse_regs.cu)
  int J;        // rows per thread of the register-resident variant
  int H;        // row halves of the register-resident variant (1 or 2)
  size_t smem;
  bool ok;  // fits the device's shared-memory limit
};

LsePlan lse_plan(int64_t K, int64_t n, int dtype_bytes);
bool lse_regs_supported(int64_t K, int dtype_bytes);
// Sample-major FP32 variant (lse_smaj.cu): v given as vst[n * Kp + k],
// Kp = K rounded up to 4 (entries k >= K zero), n = prm.n samples; logden
// (if requested) in the same sample order. Launches the pass and the
// epilogue.
// Repeated SCI steps on one small binned FP32 level in a single launch
// (sci_loop.cu); vT is the level sample-major (n x stage_pitch(K), zero
// padded). f is read at the start and written back at the end (gauge
// f_0 = 0); ctrl->iters counts the applied steps, ctrl->done is set when the
// last one met s < eps or max|df| < noise, ctrl->underflow when a step was
// not applied (some Q_k < 1e-20 N_k; redo it exactly), ctrl->nonfinite as in
// the LSE epilogue. s_out / d_out (nullable) get the last step's s and
// max|df|.
struct SciLoopParams {
  int K, n;
  const int32_t* H;    // [n] counts
  double* f;           // [K] in/out
  const double* logN;  // [K]
  const double* Nk;    // [K]
  Ctrl* ctrl;
  double* s_out;
  double* d_out;
  unsigned* err;  // timeouts of bounded waits
  double eps, noise;
  int64_t max_steps;
};
// K within the kernel's shapes and the level (n x stage_pitch(K) floats) at
// most max_bytes.
bool sci_loop_supported(int64_t K, int64_t n, double max_bytes);
size_t sci_loop_level_bytes(int64_t K, int64_t n);
mbar_status sci_loop_launch(const float* vT, const SciLoopParams& prm, cudaStream_t st);
// The same loop over the whole GPU (one cooperative launch, one CTA per SM,
// the level resident in shared memory): for one solve alone on the device.
// scratch: sci_grid_scratch_bytes(K) bytes, 256-byte aligned.
bool sci_grid_supported(int64_t K, int64_t n);
size_t sci_grid_scratch_bytes(int64_t K);
mbar_status sci_grid_launch(const float* vT, const SciLoopParams& prm, void* scratch, cudaStream_t st);
// Algorithm 1's first loop for many problems in one persistent launch
// (batch_loop.cu): a device queue of descriptors, one CTA per problem with its
// level in shared memory; K <= 256.
struct BatchLoopItem {
  const float* vT;  // the level sample-major (n x Kp, zero padded)
  int K, n, Kp, pad;
  const int32_t* H;
  double* f;  // [K] in/out
  const double* logN;
  const double* Nk;
  Ctrl* ctrl;
  double* s_out;
  double eps, noise;
  int64_t max_steps;
};
bool first_loop_batch_supported(int64_t K, int64_t n);
// level_floats: the largest n x Kp of the items
mbar_status first_loop_batch_launch(const BatchLoopItem* items_dev, int count, int* next_dev, size_t level_floats,
                                    cudaStream_t st);
// Continuous batching of the first loops of concurrent solves (batch_loop.cu):
// run() queues one item and blocks until the launch that took it has ended.
struct FirstLoopBatcher;
FirstLoopBatcher* first_loop_batcher_create();
void first_loop_batcher_destroy(FirstLoopBatcher* b);
mbar_status first_loop_batcher_run(FirstLoopBatcher* b, const BatchLoopItem& item);
void first_loop_batcher_stats(FirstLoopBatcher* b, int64_t* launches, int64_t* items);
// out[p * stage_pitch(K) + k] = v[k * ld + p] for p < n (entries k >= K zero).
mbar_status level_to_samples(const float* v, int64_t K, int64_t n, int64_t ld, float* out, cudaStream_t st);
LsePlan lse_smaj_plan(int64_t K, int64_t n);
LsePlan lse_smaj_plan_rule(int64_t K, int64_t n);  // the built-in shape rule (no tuned table)
LsePlan lse_smaj_plan_for(int64_t K, int64_t n, int lps, int nk, int nt, int stage_bytes);
bool lse_smaj_preferred(int64_t K);
mbar_status lse_smaj_launch(const float* vst, const LsePlan& pl, LseParams prm, cudaStream_t st);
// The SCI epilogue over the partials of a pass (lse.cu).
mbar_status lse_epilogue_launch(const LseParams& prm, cudaStream_t stream);
// Factorised u_kp = a_k + b_k phi_p (lse_fact.cu): a, b device FP64[K],
// phi device FP64[n]; logden (if set) device FP64[n].
// u_kn = a_k + b_k phi_n into a K x N FP64 buffer (prep.cu)
mbar_status factorised_u(const double* a, const double* b, const double* phi, int64_t K, int64_t N, double* u,
                         cudaStream_t st);
// Reference-state table of a factorised pass: the state of the largest
// exponent at kRefGrid points spread evenly over [min phi, max phi]; a
// sample's state is state[rint((phi - lo) * inv_step)] (clamped). `relative`
// is set where the exponents can exceed 2^12 in magnitude (one FP32 ulp
// 2.4e-4 or more): only then does the pass form them relative to that state.
constexpr int kRefGrid = 4096;
struct FactRef {
  float lo, inv_step;
  int relative;  // exponents relative to the reference state (else absolute)
  int pad;
  int16_t state[kRefGrid];
};
// Device bytes of a pass's table plus the partial (min, max) of phi that a
// pass without a known range computes first.
size_t lse_fact_ref_bytes();
LsePlan lse_fact_plan(int64_t K, int64_t n);
LsePlan lse_fact_plan_rule(int64_t K, int64_t n);  // the built-in shape rule (no tuned table)
LsePlan lse_fact_plan_for(int64_t K, int64_t n, int lps, int nk);
int fact_threads(int nk);
// LSE-pass autotuning (autotune.cu): the tuned shape of a (family, K, n), if
// tuning is enabled and the table has the key.
constexpr int kTuneSamples = MBAR_TUNE_SAMPLES;
constexpr int kTuneFactorised = MBAR_TUNE_FACTORISED;
bool tuned_shape(int family, int64_t K, int64_t n, int* lps, int* nk, int* nt, int* stage_bytes);
// phi_min / phi_max: device pointers to `nparts` partial minima / maxima of
// phi (a sorted copy's first and last element, nparts = 1), or nullptr: the
// range is then reduced from phi into `ref_buf` first. ref_buf: device,
// lse_fact_ref_bytes(), 16-byte aligned.
mbar_status lse_fact_launch(const double* a, const double* b, const double* phi, const LsePlan& pl, LseParams prm,
                            const double* phi_min, const double* phi_max, int nparts, void* ref_buf,
                            cudaStream_t st);
LsePlan lse_regs_plan(int64_t K, int64_t n);
mbar_status lse_regs_launch(const CUtensorMap& tmap, const LsePlan& pl, const LseParams& prm, cudaStream_t st);
size_t lse_scratch_bytes(int64_t K, int64_t n, int dtype_bytes);
// Exact log-domain SCI step (lse.cu) for steps whose linear-domain row sums
// underflowed: logQ_k = log sum_p H_p exp(a_k - v_kp - logden_p) from the
// pass's logden, then the Eq. 1 update, gauge, Eq. 2 and loop control like
// the epilogue. K x n work in FP32 with running maxima, FP64 combination.
size_t log_sci_tmp_bytes(int64_t K, int64_t n);
mbar_status log_sci_finish(const void* v, int dtype_bytes, int64_t K, int64_t n, int64_t ld, const LseParams& p,
                           void* tmp, size_t tmp_bytes, cudaStream_t st);
// Scratch of a pass whose plan has `grid` CTAs: 256 bytes (counter, error
// word), grid x K FP64 partials, then the epilogue's new f and per-CTA slots.
size_t lse_scratch_for_grid(int64_t K, int grid);
mbar_status lse_launch(const CUtensorMap& tmap, const LsePlan& pl, LseParams prm, int dtype_bytes,
                       cudaStream_t stream);

// ---- binning (binning.cu) ----
// Stable LSD radix sort of phi (binary64, order-preserving key transform);
// writes phi_sorted[N] and perm[N] (sorted position -> original sample).
mbar_status sort_coordinate(const double* phi, int64_t N, double* phi_sorted, int32_t* perm, void* tmp,
                            size_t tmp_bytes, cudaStream_t stream);
size_t sort_tmp_bytes(int64_t N);

// d_sorted[i] = phi_sorted[i] - phi_sorted[0] (binary64, rounded to nearest):
// the offsets every bin index is computed from.
// d_pairs[i] = (hi, lo) FP32 split of d_sorted[i] for the FP32 bin-index path.
mbar_status offsets_from_min(const double* phi_sorted, int64_t N, double* d_sorted, float2* d_pairs,
                             cudaStream_t stream);

// Counts of nonempty bins g(w) over the sorted offsets for nw <= 15 widths
// in one pass; counts_dev holds 15 entries.
constexpr int kWidthsPerPass = 15;  // candidate widths per counting pass
mbar_status count_bins(const float2* d_pairs, const double* d_sorted, int64_t N, const double* widths, int nw,
                       unsigned long long* counts_dev, cudaStream_t stream);

// Histogram at width w over the sorted offsets: per sorted sample its bin ordinal
// seg[N] (0..nb-1), bin start offsets start[nb+1], counts H[nb] (int32),
// keys[nb] (int64). nb is returned through *nb_dev. tmp sized by
// hist_tmp_bytes.
mbar_status build_histogram(const float2* d_pairs, const double* d_sorted, int64_t N, double w, int32_t* seg,
                            int32_t* start,
                            int32_t* H, int64_t* keys, int32_t* nb_dev, void* tmp, size_t tmp_bytes,
                            cudaStream_t stream);
size_t hist_tmp_bytes(int64_t N);

// Binned matrix: out[k][b] = mean over the bin's members of v[k][i]
// (members are the contiguous sorted columns start[b]..start[b+1]-1).
mbar_status bin_means(const void* v, int dtype_bytes, int64_t K, int64_t N, int64_t ld, const int32_t* seg,
                      const int32_t* start, int64_t nb, void* out, int64_t ld_out, void* tmp, size_t tmp_bytes,
                      cudaStream_t stream);
size_t bin_means_tmp_bytes(int64_t K, int64_t N);
// The bin means of up to 8 histograms of the same sorted data in one read of
// v (level l: segment ids seg[l], bin starts start[l], nb[l] bins, output
// out[l] with row pitch ld_out[l]).
constexpr int kMaxBinLevels = 8;
mbar_status bin_means_multi(const void* v, int dtype_bytes, int64_t K, int64_t N, int64_t ld, int L,
                            const int32_t* const* seg, const int32_t* const* start, const int64_t* nb,
                            void* const* out, const int64_t* ld_out, void* tmp, size_t tmp_bytes, cudaStream_t st);
size_t bin_means_multi_tmp_bytes(int64_t K, int64_t N, int L, const int64_t* nb);

// Column gather: out[k][i] = in[k][perm[i]] (row pitch ld for both).
mbar_status gather_columns(const void* in, void* out, int dtype_bytes, int64_t K, int64_t N, int64_t ld,
                           const int32_t* perm, cudaStream_t stream);

// ---- data preparation (prep.cu) ----
// Sample pitch of the staging: K rounded up to 4 (16-byte aligned samples).
__host__ __device__ inline int64_t stage_pitch(int64_t K) { return (K + 3) / 4 * 4; }
// u_kn (K x N FP64, row pitch ldu) -> sample-major staging
// vst[n * stage_pitch(K) + k] (entries k >= K set to 0): fl32(u - c_n) with
// c_n = min_k u_kn written to c (dtype_bytes 4), or the FP64 values
// (dtype_bytes 8; c unused); *bad |= 1 if any entry is not finite; *err
// counts bounded waits that gave up.
mbar_status stage_samples(const double* u, int64_t K, int64_t N, int64_t ldu, double* c, void* vst, int dtype_bytes,
                          int* bad, unsigned* err, cudaStream_t st);
// v[k * ld + i] = vst[perm[i] * stage_pitch(K) + k] for i < N (the row-major
// store in the column order perm).
mbar_status gather_transpose(const void* vst, int dtype_bytes, int64_t K, int64_t N, const int32_t* perm, void* v,
                             int64_t ld, cudaStream_t st);
// Adds o_p = max_k (f_k + log N_k - v_kp) to column p of an FP32 K x n
// matrix (row pitch ld), p < n; K <= 1024.
mbar_status recenter_columns(float* v, int64_t K, int64_t n, int64_t ld, const double* f, const double* logN,
                             cudaStream_t st);
mbar_status check_finite(const double* x, int64_t n, int* bad, cudaStream_t stream);
// FP32 store (K x ld, row-major) of a factorised context's binned level with
// nb bins of coordinate means phibar: v_kb = a_k + b_k phibar_b - c_b, c_b =
// min_k of it (prep.cu); tmp of fact_level_tmp_bytes(K, nb).
size_t fact_level_tmp_bytes(int64_t K, int64_t nb);
mbar_status fact_level_store(const double* a, const double* b, const double* phibar, int64_t K, int64_t nb,
                             float* out, int64_t ld, void* tmp, cudaStream_t st);

// ---- Hessian (hessian.cu) ----
// G = sum_p H_p P_ip P_jp with P_ip = exp(a_i - v_ip - logden_p) (a = f + log N);
// writes the FP64 Hessian hess[K x K] = Laplacian of G (off-diagonal -G_ij,
// diagonal sum_{j != i} G_ij).
mbar_status hessian(const void* v, int dtype_bytes, int64_t K, int64_t n, int64_t ld, const double* f,
                    const double* logN, const void* logden, const int32_t* H, double* hess, unsigned* err,
                    void* tmp, size_t tmp_bytes, cudaStream_t stream);
size_t hessian_tmp_bytes(int64_t K, int64_t n);
// The same Hessian of unbinned FP32 data read from the sample-major copy
// vst[n][round_up(K, 4)] (logden in that sample order); false from
// hessian_smaj_eligible when the tensor-core cluster kernel does not take
// this K (the caller then uses hessian on the row-major store).
bool hessian_smaj_eligible(int64_t K);
// The Hessian of a factorised context's unbinned data (K <= 1024).
mbar_status hessian_fact(const double* fa, const double* fb, const double* fphi, int64_t K, int64_t n,
                         const double* f, const double* logN, const double* logden, double* hess, unsigned* err,
                         void* tmp, size_t tmp_bytes, cudaStream_t stream);
mbar_status hessian_smaj(const float* vst, int64_t K, int64_t n, const double* f, const double* logN,
                         const float* logden, double* hess, unsigned* err, void* tmp, size_t tmp_bytes,
                         cudaStream_t stream);

// Tensor-core overlap matrix (hessian_tc.cu): G[K x K] (FP64, symmetric) =
// sum_p H_p P_ip P_jp with FP16 operands and FP32 accumulation in TMEM.
// a = f + log N (device, K). err counts bounded waits that gave up.
mbar_status overlap_tc(const void* v, int dtype_bytes, int64_t K, int64_t n, int64_t ld, const double* a,
                       const void* logden, const int32_t* H, double* G, unsigned* err, void* tmp, size_t tmp_bytes,
                       cudaStream_t st);
size_t overlap_tc_tmp_bytes(int64_t K, int64_t n);
bool overlap_tc_smaj_eligible(int64_t K);
// Factorised data (u_ip = a_i + b_i phi_p; phi and logden FP64, original
// sample order), K <= 1024: clusters of ceil(K / 128) CTAs, one launch per
// window of three tile distances (two launches above K = 640).
mbar_status overlap_tc_fact(const double* fa, const double* fb, const double* fphi, int64_t K, int64_t n,
                            const double* a, const double* logden, double* G, unsigned* err, void* tmp,
                            size_t tmp_bytes, cudaStream_t st);
mbar_status overlap_tc_smaj(const float* vst, int64_t K, int64_t n, const double* a, const float* logden, double* G,
                            unsigned* err, void* tmp, size_t tmp_bytes, cudaStream_t st);

// Which contraction hessian() uses: 0 = by size (tensor cores for K >= 64),
// 1 = CUDA cores, 2 = tensor cores.
void set_hessian_path(int path);
int hessian_path_for(int64_t K, int dtype_bytes);
bool tc_cluster_enabled();
// Direct launches instead of captured CUDA graphs for a context's binned
// loops (server workers: a stream capture in one thread would make another
// thread's device-wide synchronisation fail).
void ctx_set_graphs(mbar_ctx* c, bool on);
// A context whose first loop (MIXED, a level that fits the batched kernel)
// goes through the batcher (nullptr: its own launches).
void ctx_set_batcher(mbar_ctx* c, FirstLoopBatcher* b);

// Eqs. 5-6 (reweight.cu): p (original sample order) and log C from the
// target potential u0 (original order), the LSE pass's logden (stored order,
// dtype of the data) and the per-sample shift (nullable).
size_t reweight_tmp_bytes(int64_t N);
mbar_status reweight_weights(const double* u0, const int32_t* perm, const void* logden, int dtype_bytes,
                             const double* shift, int64_t N, double* p, double* log_c, void* tmp, size_t tmp_bytes,
                             cudaStream_t st);
mbar_status weighted_hist2d(const double* x, const double* y, const double* p, int64_t N, double x0, double dx,
                            int64_t nx, double y0, double dy, int64_t ny, double* out, cudaStream_t st);  // false: tensor-core path without the cluster variant

// ---- dense FP64 (cholesky.cu) ----
// Asymptotic covariance of f in the gauge f_0 = 0 from the MBAR Hessian
// (K x K, the Laplacian of the overlap matrix at the solution): cov[i][j] =
// [H_red^-1]_(i-1)(j-1) - delta_ij / N_i - 1 / N_0 for i, j >= 1, row and
// column 0 zero; *info |= 1 if H_red is not positive definite.
size_t covariance_tmp_bytes(int64_t K);
mbar_status covariance(const double* hess, int64_t K, const double* Nk, double* cov, int* info, void* tmp,
                       size_t tmp_bytes, cudaStream_t st);
// Solves A x = b for the (m x m) symmetric positive definite block
// A = hess[1:,1:] (row pitch K) and b = -g[1:]; x written to delta[1:],
// delta[0] = 0. Sets *info != 0 if a pivot is not positive.
mbar_status newton_solve(double* hess, int64_t K, const double* g, double* delta, int* info, void* tmp,
                         size_t tmp_bytes, cudaStream_t stream);
size_t newton_tmp_bytes(int64_t K);

// small helpers (prep.cu)
// out = f + t d in the gauge out_0 = 0
mbar_status vec_add_gauge(const double* f, const double* d, double* out, int64_t K, cudaStream_t stream,
                          double t = 1.0);

}  // namespace bumbar
