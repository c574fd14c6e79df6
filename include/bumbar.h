/*
 * bumbar.h -- C ABI of the B300-native BU-MBAR hot path.
 *
 * BU-MBAR (binned-to-unbinned MBAR; Mueller, Alesiani, Christiansen) solves
 * the MBAR / UWHAM equations for K thermodynamic states and N samples by
 * iterating the WHAM self-consistent update (Eq. 1) on histograms with a
 * growing number of nonempty bins (Algorithm 1, heuristic Eq. 3), and ends
 * with derivative-based (Newton) iterations on the unbinned data (Sec. II,
 * Sec. III). The data are the reduced potentials
 *
 *     u_kn  =  reduced potential of sample n evaluated in state k
 *              (the paper's beta_i E_p; row-major, K rows of N samples),
 *     N_k   =  number of samples drawn from state k, sum_k N_k = N,
 *
 * and the result is the dimensionless free-energy vector f (gauge f_0 = 0).
 *
 * Conventions of every entry point:
 *   - return an mbar_status; nothing aborts, throws or exits;
 *   - pointers documented "host" are read or written synchronously before
 *     the call returns; "device" pointers must be CUDA device memory of the
 *     current device; the library never keeps a caller pointer after a call;
 *   - a context owns all device memory it allocates; mbar_destroy frees it;
 *   - calls on one context are not thread safe; distinct contexts on
 *     distinct streams are independent;
 *   - on error, mbar_last_error() returns a message for the calling thread.
 */
#ifndef BUMBAR_H
#define BUMBAR_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define BUMBAR_API __attribute__((visibility("default")))
#else
#define BUMBAR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mbar_ctx mbar_ctx; /* opaque, owned by the library */

typedef enum {
  MBAR_OK = 0,
  MBAR_EINVAL = 1,      /* bad argument: K < 1, N_k sum != N, non-finite u, ... */
  MBAR_ENOMEM = 2,      /* device or host allocation failed */
  MBAR_ECUDA = 3,       /* a CUDA runtime/driver call failed */
  MBAR_ENOTCONV = 4,    /* iteration limit reached; the current f is readable */
  MBAR_ESTATE = 5,      /* call not valid in the context's current state */
  MBAR_ETIMEOUT = 6,    /* a bounded device-side wait gave up */
  MBAR_EUNSUPPORTED = 7 /* size or option outside what the library supports */
} mbar_status;

typedef enum {
  MBAR_FP64 = 0,  /* u_kn stored in FP64, exp/LSE/accumulation in FP64 */
  MBAR_MIXED = 1  /* u_kn shifted per sample and stored in FP32, exp/LSE in
                     FP32, row sums accumulated in FP64, FP64 Newton solve */
} mbar_precision;

/* Options. mbar_opts_default fills the paper's hyperparameters (Sec. II,
 * after Algorithm 1): n0 = 100, eps = 1e-3, inc = 10, n_intermediate = 20. */
typedef struct {
  int32_t precision;      /* mbar_precision */
  int32_t n0;             /* initial number of nonempty bins */
  double eps;             /* first-loop threshold on the relative step (Eq. 2) */
  int32_t inc;            /* bin-count increase factor */
  int32_t n_intermediate; /* SCI steps between checks of Eq. 3 */
  double h0;              /* > 0: explicit width schedule h0, h0/inc, ...
                             instead of the width rule w*(n) of Sec. II */
  int32_t use_binning;    /* 0: skip Algorithm 1 (plain MBAR: unbinned SCI
                             warm-up, then Newton) */
  double f_tol;           /* Newton stops when max|delta f| < f_tol; Newton
                             steps below 10 f_tol are always accepted */
  double warm_tol;        /* plain-MBAR warm-up: SCI until max_k|g_k|/N_k < warm_tol */
  int32_t max_newton;     /* Newton iteration limit */
  int32_t max_sci;        /* limit on SCI steps per loop of Algorithm 1 */
  double noise_floor;     /* > 0: an SCI step with max_k |delta f_k| below this
                             many kT is under the rounding floor of the
                             evaluation; Algorithm 1 then treats the level as
                             converged (first loop: stop; second loop: raise
                             n). 0 = Eqs. 2-3 exactly as printed. */
} mbar_opts;

typedef struct {
  int64_t iters_first_loop;  /* SCI steps of Algorithm 1's first loop */
  int64_t iters_second_loop; /* SCI steps (including probes) of its second loop */
  int64_t iters_newton;      /* Newton iterations on unbinned data */
  int64_t newton_fallbacks;  /* Newton steps replaced by an SCI step */
  int64_t n_rebins;          /* histograms built */
  int64_t final_bins;        /* nonempty bins of the last binned level */
  double max_abs_grad;       /* max_k |g_k| at the returned f */
  double last_step;          /* max |delta f| of the last Newton step */
  double seconds_width;      /* host wall time in the width search w*(n) */
  double seconds_levels;     /* ... building histograms and binned matrices */
  double seconds_sci;        /* ... in the SCI loops of Algorithm 1 */
  double seconds_newton;     /* ... in the unbinned Newton phase */
} mbar_report;

/* Fills *opts with the defaults above (f_tol 1e-10 for MBAR_FP64, 1e-5 for
 * MBAR_MIXED, chosen by `precision`; warm_tol 1e-3; max_newton 50;
 * max_sci 200000; use_binning 1; h0 0; noise_floor 1e-11 kT for MBAR_FP64
 * and 2e-6 kT for MBAR_MIXED: rounding alone moves f by ~1e-13 kT per FP64
 * step and ~1e-7..1e-6 kT per FP32 step). */
BUMBAR_API mbar_status mbar_opts_default(mbar_opts* opts, int32_t precision);

/* Creates a context for one problem (the paper's input list of Algorithm 1:
 * per-state sample counts and energies, generalised to u_kn).
 *   K, N         number of states (1 <= K <= 1024) and samples (N >= 1);
 *   N_k          host[K], positive, sum == N;
 *   u_kn         K x N row-major FP64, host or device (u_on_device != 0);
 *                every entry must be finite;
 *   opts         NULL for defaults of MBAR_MIXED;
 *   cuda_stream  cudaStream_t to run on (NULL = legacy default stream).
 * The library copies u_kn into its own device buffer (FP64, or FP32 after
 * subtracting c_n = min_k u_kn from each column in mixed precision) and
 * sets the bin coordinate to row 0 of u_kn. Freed stream-ordered allocations
 * stay cached in the device's default memory pool (rebins reuse them).
 * Errors: EINVAL (sizes, counts, non-finite u), ENOMEM, ECUDA, EUNSUPPORTED. */
BUMBAR_API mbar_status mbar_create(mbar_ctx** out, int64_t K, int64_t N, const int64_t* N_k, const double* u_kn,
                        int32_t u_on_device, const mbar_opts* opts, void* cuda_stream);

/* Creates a context from factorised reduced potentials
 *     u_kn = a_k + b_k phi_n
 * (Sec. II: the paper's u = beta_k E_n is a = 0, b = beta, phi = E): only
 * the 2 K + N numbers cross the host link, and phi is the bin coordinate.
 * a, b: FP64[K]; phi: FP64[N]; all three on the host (on_device = 0) or all
 * in device memory (on_device = 1). N_k, opts, cuda_stream and the errors as
 * for mbar_create.
 *   MBAR_MIXED with binning (the default options): the context keeps a, b
 *   and phi (FP64, O(K + N) bytes) and no K x N store. A binned level's
 *   entries are a_k + b_k mean_b(phi) (the bin means of u, exactly so for a
 *   factorised u); the unbinned passes and the Hessian form u from a, b and
 *   phi inside their kernels. mbar_set_coordinate returns EUNSUPPORTED.
 *   Otherwise: u is generated on the device, with the product and the sum
 *   each rounded to nearest in binary64, exactly as a host evaluating
 *   a + b * phi gets it, and stored like mbar_create stores a given u; the
 *   call holds a temporary K x N FP64 buffer (ENOMEM if it cannot be
 *   allocated).
 * The call returns once the context's device data are complete. */
BUMBAR_API mbar_status mbar_create_factorised(mbar_ctx** out, int64_t K, int64_t N, const int64_t* N_k,
                                              const double* a, const double* b, const double* phi,
                                              int32_t on_device, const mbar_opts* opts, void* cuda_stream);

/* Sets the 1-D bin coordinate phi_n (Sec. II bins the energies E_p; here any
 * per-sample coordinate). phi: N finite FP64 values, host or device.
 * Sorts the samples by phi once (stable LSD radix sort) and reorders the
 * stored columns, so every later histogram is a scan over contiguous runs. */
BUMBAR_API mbar_status mbar_set_coordinate(mbar_ctx* ctx, const double* phi, int32_t phi_on_device);

/* Builds the histogram of nonempty bins of uniform width h anchored at
 * min(phi) (Sec. II): bin index floor((phi_n - min phi)/h) with the
 * subtraction and division each rounded to nearest in binary64, counts
 * H_p >= 1, and the binned reduced potential u_kp = mean of u_kn over the
 * bin's members. h == 0 selects the unbinned data. The histogram becomes the
 * context's current level for mbar_sci_step / mbar_hessian.
 * n_bins_out (host, nullable) receives the number of nonempty bins.
 * EINVAL if h < 0 or (max phi - min phi)/h > 2^52. */
BUMBAR_API mbar_status mbar_bin(mbar_ctx* ctx, double h, int64_t* n_bins_out);

/* Width rule of Sec. II, w*(n) = max{w : n <= g(w)}, by the deterministic
 * search: R = range of phi; w_hi = 2R, w_lo = R/n; halve w_lo (w_hi takes
 * its old value) until g(w_lo) >= n, giving up once R/w_lo > 2^52; then up
 * to 64 geometric bisections mid = sqrt(w_lo*w_hi) (each operation rounded
 * to nearest), keeping w_lo with g(w_lo) >= n. On success bins at w* like
 * mbar_bin and returns w* in *w_out; if n cannot be reached, selects the
 * unbinned data and returns *w_out = 0. n <= 1 or R == 0 gives one bin. */
BUMBAR_API mbar_status mbar_bin_count(mbar_ctx* ctx, int64_t n, double* w_out, int64_t* n_bins_out);

/* Reads the current histogram back. keys (host int64[n_bins], nullable):
 * bin indices in increasing order; H (host int64[n_bins], nullable): counts;
 * u_kp (host FP64 K x n_bins row-major, nullable): binned reduced potential
 * as stored -- in MBAR_MIXED column p is lowered by the constant
 * mean_{n in p} c_n of its members (differences between states are exact
 * up to FP32 storage). ESTATE if the current level is unbinned. */
BUMBAR_API mbar_status mbar_get_bins(mbar_ctx* ctx, int64_t* keys, int64_t* H, double* u_kp);

/* One self-consistent step, Eq. 1, on the current level (bins with counts
 * H_p, or the unbinned samples with H = 1), from f_in (host[K]):
 *   logden_p = log sum_j N_j exp(f_j - u_jp)           (paired LSE, part 1)
 *   Q_i      = sum_p H_p N_i exp(f_i - u_ip - logden_p) (paired LSE, part 2)
 *   f_out_i  = f_i - log(Q_i / N_i), then gauge f_out_0 = 0
 *   grad_i   = Q_i - N_i (gradient of the convex MBAR objective)
 *   s        = max over i with f_in_i != 0 of |f_out_i/f_in_i - 1| (Eq. 2),
 *              +inf if f_in is all zero.
 * f_out, grad (host[K]), s_out (host scalar), logden (host FP64[n_cols] in
 * the caller's original sample order when unbinned, bin order otherwise)
 * are all nullable. */
BUMBAR_API mbar_status mbar_sci_step(mbar_ctx* ctx, const double* f_in, double* f_out, double* grad, double* s_out,
                          double* logden);

/* Hessian of the MBAR objective on the current level at f_in (host[K]):
 *   H_ij = delta_ij sum_p H_p P_ip - sum_p H_p P_ip P_jp,  P_ip = N_i W_ip,
 * evaluated as the overlap matrix G_ij = sum_p H_p P_ip P_jp (off-diagonal,
 * tensor cores, FP16 operands / FP32 accumulation) with the diagonal taken
 * from the zero row sums, H_ii = sum_{j != i} G_ij.
 * hess (host FP64 K x K row-major). */
BUMBAR_API mbar_status mbar_hessian(mbar_ctx* ctx, const double* f_in, double* hess);

/* One gauge-fixed Newton step from f_in on the current level: gradient,
 * Hessian, FP64 Cholesky of the (K-1)x(K-1) block without state 0, and
 * f_out = f_in + delta (delta_0 = 0). step_max_abs (nullable) = max|delta|.
 * ENOTCONV if the reduced Hessian is not numerically positive definite. */
BUMBAR_API mbar_status mbar_newton_step(mbar_ctx* ctx, const double* f_in, double* f_out, double* step_max_abs);

/* Full solve: Algorithm 1 on the binned data (unless opts.use_binning == 0)
 * followed by Newton iterations on the unbinned data until
 * max|delta f| < f_tol. f_init (host[K], nullable => 0) warm-starts; with a
 * warm start the first loop of Algorithm 1 runs from f_init.
 * report (host, nullable). ENOTCONV: limit reached, f still readable. */
BUMBAR_API mbar_status mbar_solve(mbar_ctx* ctx, const double* f_init, mbar_report* report);

/* Eqs. 5-6: statistical weight of every sample at a target state whose
 * reduced potential is u0_n (beta_0 E_n in the paper), at the context's
 * current free energies, over the unbinned samples:
 *   p_n = (1/C) exp(-u0_n) / sum_m N_m exp(f_m - u_mn),
 *   C   = sum_n exp(-u0_n) / sum_m N_m exp(f_m - u_mn).
 * u0 (N finite FP64, host or device per u0_on_device) and p_out (host
 * FP64[N], nullable) are in the caller's original sample order; log_C
 * (nullable) receives log C. The weights stay on the device for
 * mbar_weighted_histogram2d. EINVAL for non-finite u0. */
BUMBAR_API mbar_status mbar_reweight(mbar_ctx* ctx, const double* u0, int32_t u0_on_device, double* p_out,
                                     double* log_C);

/* Histogram of the last mbar_reweight weights over per-sample coordinates
 * (x_n, y_n) (original order, host or device per on_device): bin
 * (floor((x - x0)/dx), floor((y - y0)/dy)), each subtraction and division
 * rounded to nearest in binary64, kept when inside nx x ny; out (host FP64
 * nx*ny, row-major by x bin) receives the summed weights (the paper's Fig. 1
 * plots -log of this over two dihedral angles). ESTATE before any
 * mbar_reweight; EINVAL for dx, dy <= 0 or nx, ny < 1. */
BUMBAR_API mbar_status mbar_weighted_histogram2d(mbar_ctx* ctx, const double* x, const double* y, int32_t on_device,
                                                 double x0, double dx, int64_t nx, double y0, double dy, int64_t ny,
                                                 double* out);

/* Copies the current free energies (gauge f_0 = 0) to f_out (host[K]). */
BUMBAR_API mbar_status mbar_free_energies(mbar_ctx* ctx, double* f_out);

/* Frees everything the context owns. mbar_destroy(NULL) is MBAR_OK. */
BUMBAR_API mbar_status mbar_destroy(mbar_ctx* ctx);

/* Static description of a status code. */
BUMBAR_API const char* mbar_status_string(mbar_status status);

/* Whether the context may assume the GPU to itself (1, the default) or
 * shares it with solves running concurrently on other streams (0). With 1
 * the binned loops of Algorithm 1 are captured into CUDA graphs, and the
 * SCI steps of binned FP32 levels that fit in the shared memory of all SMs
 * (up to ~25 MB) run in one cooperative launch over every SM with the level
 * resident in shared memory. With 0 no graphs are captured and such levels
 * run on one cluster of 8 SMs (or as separate launches), leaving the other
 * SMs to the concurrent solves; a cooperative launch of every SM would wait
 * for them. Results agree within the tolerance of the mixed precision
 * (the per-state sums are grouped differently). EINVAL for a null context. */
BUMBAR_API mbar_status mbar_set_exclusive(mbar_ctx* ctx, int32_t exclusive);

/* Message of the last failed call on this thread ("" if none). */
BUMBAR_API const char* mbar_last_error(void);

/* Opt-in timing of the context's large launches with CUDA events on its
 * stream (for profiling; adds two event records per timed launch).
 * mbar_set_timing(ctx, 1) clears earlier records and starts recording,
 * 0 stops. mbar_get_timing sums the records of one kind:
 *   0 = unbinned fused LSE passes, 1 = Hessian (in the Newton phase and in
 *       mbar_hessian), 2 = FP64 Newton solve,
 *   3 = unbinned passes that only confirm a Newton step below f_tol (FP32
 *       data: plain FP32 sums instead of the exact split of each sample's
 *       largest weight that kind 0 uses),
 *   4 = rounds of Algorithm 1's second loop (N_intermediate + 1 passes over
 *       the current binned level and one over the next; bytes = the data
 *       those passes read),
 *   5 = one-launch runs of the first loop on a small FP32 level (bytes =
 *       steps taken x the level's data);
 * launches, total_ms (device time) and bytes (K x n x element size of the
 * data each launch streams; K x K x 8 for the solve) are all nullable. */
BUMBAR_API mbar_status mbar_set_timing(mbar_ctx* ctx, int32_t enable);
BUMBAR_API mbar_status mbar_get_timing(mbar_ctx* ctx, int32_t kind, int64_t* launches, double* total_ms,
                                       double* bytes);

/* Trace of the last mbar_solve, one row of 4 doubles per event:
 *   (1, n, s, iterations)      end of Algorithm 1's first loop at n bins;
 *   (2, n, s_n, s_next)        one check of Eq. 3 in the second loop;
 *   (3, iteration, |delta f|max, max|g|)  accepted Newton step;
 *   (5, iteration, |t delta f|max, max|g|)  rejected full Newton step, the
 *                              step t = 2^-h accepted instead (backtracking
 *                              on ||g||^2 while |delta f|max >= 100 f_tol);
 *   (4, iteration, |delta f|max, max|g|)  rejected Newton step (SCI instead).
 * *rows receives the number of rows; out (host, nullable) receives up to
 * `capacity` rows. */
BUMBAR_API mbar_status mbar_get_trace(mbar_ctx* ctx, int64_t* rows, double* out, int64_t capacity);

/* Process-wide choice of the Hessian contraction: 0 = by size (tensor
 * cores, FP16 operands / FP32 accumulation, for K >= 64; CUDA cores, FP32,
 * below), 1 = always CUDA cores, 2 = always tensor cores, 3 = tensor cores
 * without the thread-block-cluster kernel (which otherwise serves FP32 data
 * with K <= 512). For testing and tuning; EINVAL for other values. */
BUMBAR_API mbar_status mbar_set_hessian_path(int32_t path);

/* ---- Autotuning of the LSE passes' launch shapes ----------------------
 * Not part of the method: a measurement-driven choice among the compiled
 * launch shapes of the two streaming passes that have several, the
 * sample-major FP32 pass (every MIXED unbinned pass; MBAR_TUNE_SAMPLES) and
 * the factorised pass (MBAR_TUNE_FACTORISED). A key is (device name, family,
 * K rounded up to a power of two >= 4, floor(log2 n)). The candidates are
 * the compiled shapes (lanes per sample, chunks of 4 states per lane) that
 * cover the key's K with the fewest chunks, and for the sample-major pass
 * stage sizes of 24-96 KB; each is timed on synthetic device data of the
 * given size (capped at 1 GB) with CUDA events: the median of three rounds
 * of the exact-split pass plus the plain pass. While tuning is enabled,
 * every plan of those passes whose key is in the table takes its shape (the
 * FP32 partial sums then add in another order: results move at their
 * rounding level); otherwise the built-in shape rules apply. */
enum { MBAR_TUNE_SAMPLES = 0, MBAR_TUNE_FACTORISED = 1 };

typedef struct {
  int32_t family;            /* MBAR_TUNE_* */
  int32_t lanes_per_sample;  /* the chosen shape */
  int32_t chunks_per_lane;
  int32_t threads;
  int32_t stage_bytes;       /* sample-major pass only (0 otherwise) */
  int32_t candidates;        /* shapes timed */
  double ms;                 /* chosen shape: one exact-split + one plain pass */
  double heuristic_ms;       /* the built-in rule's shape, the same way */
  int32_t cached;            /* 1: taken from the table, nothing was timed */
  int32_t pad;
} mbar_tune_result;

/* Searches the shape of (family, K, n)'s key, unless the table already has
 * it, and records it (and appends it to the cache file, if one is set).
 * Allocates and frees its own device buffers (up to ~1 GB) on the current
 * device and synchronises its own stream. EINVAL for a bad family or sizes,
 * EUNSUPPORTED for K > 1024, ENOMEM, ECUDA. */
BUMBAR_API mbar_status mbar_autotune_lse(int32_t family, int64_t K, int64_t n, mbar_tune_result* out);
/* Plans consult the tuned table (on != 0) or the built-in rules (0, the
 * default). Process-wide. */
BUMBAR_API mbar_status mbar_autotune_enable(int32_t on);
/* Sets the text file the table is appended to, and loads its lines now
 * (NULL or "": none). A missing file is not an error. */
BUMBAR_API mbar_status mbar_autotune_cache(const char* path);
/* Empties the in-memory table (the file is left as it is). */
BUMBAR_API mbar_status mbar_autotune_clear(void);

/* Number of CUDA kernels this library has launched in this process. */
BUMBAR_API mbar_status mbar_kernel_launches(int64_t* count);

/* Asymptotic covariance of the free energies at the context's current f
 * (call after mbar_solve). Not in the paper; the standard large-sample
 * result for the MBAR estimator: with H the Hessian of the MBAR objective at
 * the solution (the Laplacian of the overlap matrix, as used by the Newton
 * phase) and H_red its block without state 0,
 *   cov_out[i*K + j] = cov(f_i - f_0, f_j - f_0)
 *                    = [H_red^-1]_(i-1)(j-1) - delta_ij / N_i - 1 / N_0,
 * i, j >= 1; row and column 0 are zero (the gauge f_0 = 0).
 * cov_out: host FP64[K*K]. H comes from the same kernels as mbar_hessian
 * (FP16 tensor-core products for K >= 64: relative error ~1e-3).
 * ENOTCONV if H_red is not positive definite (states without overlap). */
BUMBAR_API mbar_status mbar_covariance(mbar_ctx* ctx, double* cov_out);

/* Bytes of device memory the context currently holds. */
BUMBAR_API mbar_status mbar_device_bytes(mbar_ctx* ctx, int64_t* bytes);

/* ---------------------------------------------------------------------
 * Stateless device-level entry point: one fused paired-LSE pass.
 *
 * The Eq. 1 evaluation over a K x n matrix that is already resident in
 * device memory. v: device, K rows of n columns, row pitch ld elements
 * (ld >= n, ld * elem_bytes a multiple of 16, v 16-byte aligned);
 * dtype_bytes 4 (FP32) or 8 (FP64). Columns may carry any per-column
 * shift (f does not depend on it).
 *   f (device FP64[K]) current free energies; log_N (device FP64[K]);
 *   H (device int32[n], nullable => all ones) column counts;
 *   Q (device FP64[K], out) Q_i = sum_p H_p exp(f_i + log N_i - v_ip - logden_p);
 *   logden (device, nullable, same dtype as v, [n], out)
 *          logden_p = log sum_j exp(f_j + log N_j - v_jp);
 *   scratch (device) of at least mbar_lse_scratch_bytes(K, n, dtype_bytes)
 *          bytes, 16-byte aligned, owned by the caller; it holds per-CTA
 *          partial row sums and a completion counter, which must be zero
 *          before the first call (the pass leaves it zero again).
 * Runs asynchronously on `stream`. EINVAL on bad sizes or alignment,
 * EUNSUPPORTED for K > 1024.
 * ------------------------------------------------------------------- */
BUMBAR_API size_t mbar_lse_scratch_bytes(int64_t K, int64_t n, int32_t dtype_bytes);
BUMBAR_API mbar_status mbar_lse_pass(const void* v, int32_t dtype_bytes, int64_t K, int64_t n, int64_t ld,
                          const double* f, const double* log_N, const int32_t* H, double* Q, void* logden,
                          void* scratch, size_t scratch_bytes, void* stream);

/* The same pass over FP32 data stored sample-major, the layout of MIXED's
 * unbinned passes: v_nk (device FP32, 16-byte aligned) holds sample p's
 * K values contiguously at v_nk[p * Kp + k], Kp = K rounded up to a
 * multiple of 4; the Kp - K padding entries of each sample must be finite
 * (they get weight 0). Each stage of the pass is then one contiguous run
 * of samples, fetched by a single bulk copy. f, log_N, H, Q as above;
 * logden (device FP32[n], nullable) per sample. scratch of at least
 * mbar_lse_samples_scratch_bytes(K, n) bytes, same rules as above.
 * EINVAL on bad sizes or alignment, EUNSUPPORTED for K > 1024. */
BUMBAR_API size_t mbar_lse_samples_scratch_bytes(int64_t K, int64_t n);
BUMBAR_API mbar_status mbar_lse_pass_samples(const float* v_nk, int64_t K, int64_t n, const double* f,
                                             const double* log_N, const int32_t* H, double* Q, float* logden,
                                             void* scratch, size_t scratch_bytes, void* stream);

/* The same pass over factorised reduced potentials u_kp = a_k + b_k phi_p
 * (Sec. II: the paper's energies u_kp = beta_k E_p are the case a = 0,
 * b = beta, phi = E), generated on the device from the 2 K + n inputs
 * instead of read from a K x n store. The exponents are formed from
 * unevaluated FP32 pairs of the FP64 inputs and rounded once where
 * f_k + log N_k - a_k and b_k phi_p cancel, so potentials of thousands of
 * kT keep about FP32 resolution of the exponent itself; the sums are FP32
 * per sample and FP64 across samples.
 *   a, b (device FP64[K]); phi (device FP64[n], finite);
 *   f, log_N, H, Q as for mbar_lse_pass;
 *   logden (device FP64[n], nullable, out): logden_p as above;
 *   scratch of at least mbar_lse_factorised_scratch_bytes(K, n) bytes,
 *   16-byte aligned, zero before the first call (left zero again).
 * Runs asynchronously on `stream`. EINVAL on null pointers, bad sizes or
 * a short or misaligned scratch; EUNSUPPORTED for K > 1024. */
BUMBAR_API size_t mbar_lse_factorised_scratch_bytes(int64_t K, int64_t n);
BUMBAR_API mbar_status mbar_lse_pass_factorised(const double* a, const double* b, const double* phi, int64_t K,
                                                int64_t n, const double* f, const double* log_N, const int32_t* H,
                                                double* Q, double* logden, void* scratch, size_t scratch_bytes,
                                                void* stream);

/* ---------------------------------------------------------------------
 * Allocation-free variant of mbar_lse_pass (no counterpart in the paper;
 * an interface for callers that cannot allocate device memory: for example
 * a host framework whose caching allocator already owns nearly all of the
 * GPU's memory, or a latency-critical loop where cudaMalloc's implicit
 * device synchronisation is not acceptable).
 *
 * Same arguments, layout and results as mbar_lse_pass, minus the scratch
 * buffer: the pass uses a fixed, 256-byte-aligned array of
 * mbar_lse_static_scratch_bytes() bytes (1 MiB) compiled into this library,
 * which every GPU that loads the library holds until the process exits.
 * The call allocates nothing (no cudaMalloc/cudaFree, no allocating library
 * routine); it zeroes the array's counter on `stream` before launching.
 *   - Every call looks up the array's device address on the current device
 *     (cudaGetSymbolAddress; it allocates nothing); the first call on a
 *     device also loads the library's module there, so make it before any
 *     stream capture.
 *   - All calls share the one array, which keeps the last call's contents:
 *     calls that overlap on the GPU (concurrent streams, several host
 *     threads) race and give wrong results; order them.
 *   - Sizes whose scratch need (mbar_lse_scratch_bytes) exceeds the array
 *     are rejected with MBAR_EUNSUPPORTED and a message naming both sizes;
 *     use mbar_lse_pass with a caller buffer for those.
 * ------------------------------------------------------------------- */
BUMBAR_API size_t mbar_lse_static_scratch_bytes(void);
BUMBAR_API mbar_status mbar_lse_pass_static(const void* v, int32_t dtype_bytes, int64_t K, int64_t n, int64_t ld,
                                            const double* f, const double* log_N, const int32_t* H, double* Q,
                                            void* logden, void* stream);

/* ---------------------------------------------------------------------
 * Serving and batching. These layer on mbar_ctx: every request is solved by
 * its own context (mbar_create, mbar_set_coordinate, mbar_solve,
 * mbar_free_energies, mbar_destroy) on one of the server's worker threads,
 * each with its own CUDA stream, so requests that are admitted together
 * run concurrently on the GPU. A request's kernels, launch shapes and
 * reduction orders depend only on its own K, N and options: its result is
 * the same alone and in any mix.
 *
 * Admission (continuous batching): queued requests are admitted in arrival
 * order while a worker is free and the request's device footprint
 * (mbar_footprint_bytes) fits in what the admitted requests leave of
 * hbm_budget_bytes; a request that does not fit yet is passed over by later
 * ones, at most 4 x workers times, after which admission waits for it.
 * ------------------------------------------------------------------- */
typedef struct mbar_server mbar_server;

enum { MBAR_BATCH_PERSISTENT = 1 };

typedef struct {
  int32_t workers;           /* concurrent solves, 1..256 */
  int32_t flags;             /* MBAR_BATCH_PERSISTENT: first loops batched (mbar_batch_solve) */
  uint64_t hbm_budget_bytes; /* device memory the admitted requests may hold together */
  mbar_opts opts;            /* options of every solve */
} mbar_server_config;

/* Estimated peak device memory of one solve from host u (creation with an
 * FP64 staging copy of u, the stored data, Algorithm 1's binned levels,
 * reorder buffer, per-sample vectors and the Hessian). 0 for K < 1 or N < 1.
 * The server charges requests whose u is in device memory without the
 * staging copy. */
BUMBAR_API uint64_t mbar_footprint_bytes(int64_t K, int64_t N, int32_t precision, int32_t use_binning);

/* The same estimate for a solve from the factorised form (as
 * mbar_create_factorised): with MBAR_MIXED and binning, Algorithm 1's binned
 * levels, the FP64 a, b, phi and per-sample vectors and the Hessian's
 * scratch, no K x N store; otherwise a K x N FP64 buffer of u plus the
 * footprint of a context made from device u. 0 for K < 1 or N < 1. */
BUMBAR_API uint64_t mbar_footprint_factorised_bytes(int64_t K, int64_t N, int32_t precision, int32_t use_binning);

/* Starts `cfg->workers` worker threads on the current device. With
 * MBAR_BATCH_PERSISTENT in cfg->flags (MBAR_MIXED and binning) the server
 * also runs a first-loop batcher: the first loops of the solves it runs go
 * into shared persistent launches (see mbar_batch_solve), and results agree
 * with the solves alone to rounding instead of bit for bit.
 * EINVAL for a bad configuration, ENOMEM if the threads cannot start. */
BUMBAR_API mbar_status mbar_server_create(mbar_server** out, const mbar_server_config* cfg);

/* Queues one solve (arguments as mbar_create / mbar_set_coordinate; phi
 * nullable => row 0 of u). N_k is copied now; u_kn and phi (host or
 * device) are read when the request is admitted and must stay valid until
 * mbar_server_wait has returned for it. *id receives the request id.
 * EUNSUPPORTED if the footprint exceeds the whole budget (it could never be
 * admitted) or K > 1024; ESTATE while the server shuts down. */
BUMBAR_API mbar_status mbar_server_submit(mbar_server* server, int64_t K, int64_t N, const int64_t* N_k,
                                          const double* u_kn, int32_t u_on_device, const double* phi,
                                          int32_t phi_on_device, int64_t* id);

/* Queues one solve from the factorised form u_kn = a_k + b_k phi_n
 * (arguments as mbar_create_factorised: a, b FP64[K], phi FP64[N], all on
 * the host or all on the device; phi is the bin coordinate). N_k is copied
 * now; a, b and phi are read when the request is admitted and must stay
 * valid until mbar_server_wait has returned for it. The request is charged
 * mbar_footprint_factorised_bytes. Results, errors and waiting as for
 * mbar_server_submit. */
BUMBAR_API mbar_status mbar_server_submit_factorised(mbar_server* server, int64_t K, int64_t N, const int64_t* N_k,
                                                     const double* a, const double* b, const double* phi,
                                                     int32_t on_device, int64_t* id);

/* Non-blocking state of a request: 0 queued, 1 admitted/running, 2 done. */
BUMBAR_API mbar_status mbar_server_poll(mbar_server* server, int64_t id, int32_t* state);

/* Blocks until request `id` is done and releases its record. f_out
 * (host[K], nullable) receives the free energies (f_0 = 0), report
 * (nullable) the solve's report, latency_s (nullable) the seconds from
 * submit to completion, run_s (nullable) from admission to completion.
 * Returns the request's own status (e.g. ENOTCONV, with f still copied). */
BUMBAR_API mbar_status mbar_server_wait(mbar_server* server, int64_t id, double* f_out, mbar_report* report,
                                        double* latency_s, double* run_s);

/* Counters since creation: completed requests, the largest number of
 * requests admitted at once, and the largest sum of their footprints. */
BUMBAR_API mbar_status mbar_server_stats(mbar_server* server, int64_t* completed, int32_t* peak_running,
                                         uint64_t* peak_bytes);

/* Stops the server: running requests finish, queued ones are dropped (their
 * waiters get ESTATE). mbar_server_destroy(NULL) is MBAR_OK. */
BUMBAR_API mbar_status mbar_server_destroy(mbar_server* server);

/* P independent solves with configuration cfg: problem p has K[p] states,
 * N[p] samples, counts N_k[p], energies u_kn[p] (all host, or all device
 * with u_on_device) and coordinate phi[p] (phi nullable, or entries
 * nullable). f_out[p] (host[K[p]]) receives its free energies, reports[p] /
 * statuses[p] (nullable arrays) its report and status. Returns the first
 * failing status, MBAR_OK if all succeeded.
 * The problems run through a temporary server (cfg->workers threads,
 * admission within the budget). Without MBAR_BATCH_PERSISTENT in cfg->flags
 * results are bit for bit those of each problem solved alone. With it
 * (MBAR_MIXED and binning), every first loop of Algorithm 1 whose level fits
 * a CTA's shared memory (K <= 256) is queued to a batcher thread, which runs
 * all queued first loops in one persistent launch (a device queue of the
 * problems, one CTA each; loops that arrive meanwhile go into the next
 * launch); those loops sum in another order, so results agree with the
 * solve alone to rounding, not bit for bit. */
BUMBAR_API mbar_status mbar_batch_solve(int32_t P, const int64_t* K, const int64_t* N, const int64_t* const* N_k,
                                        const double* const* u_kn, int32_t u_on_device, const double* const* phi,
                                        int32_t phi_on_device, const mbar_server_config* cfg, double* const* f_out,
                                        mbar_report* reports, mbar_status* statuses);

/* Self-test of the device-side failure path (diagnostics; no counterpart
 * in the paper): one kernel waits on an mbarrier that nothing completes,
 * gives up after limit_us (1 us .. 2 s), records the timeout and returns.
 * Returns MBAR_ETIMEOUT (the expected outcome) with *waited_s (nullable)
 * the time the wait ran; the device stays usable. Every wait in this
 * library's kernels is bounded the same way and reports MBAR_ETIMEOUT. */
BUMBAR_API mbar_status mbar_selftest_wait_timeout(int64_t limit_us, double* waited_s);

#ifdef __cplusplus
}
#endif

#endif /* BUMBAR_H */
