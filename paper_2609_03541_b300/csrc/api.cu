// C ABI and the solver driver: Algorithm 1 (binned-to-unbinned SCI with the
// bin-refinement heuristic of Eq. 3) followed by Newton iterations on the
// unbinned data. All arithmetic runs in the kernels of this library; the
// host only sequences launches and takes the scalar decisions of
// Algorithm 1 (s < eps, 2 s_next > inc s_n, the break rule) and of the
// Newton safeguard from values the kernels leave in device memory.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <numeric>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace bumbar {
const char* last_error();
}

using namespace bumbar;

namespace {

constexpr double kMaxIndex = 4503599627370496.0;  // 2^52

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
constexpr int kPhase1Batch = 16;                  // guarded SCI launches per host check

// Scalars the kernels leave for the host, contiguous so one pinned copy
// brings them all back.
struct DevStatus {
  Ctrl ctrl;
  double s, s2, d;  // relative steps (Eq. 2) of the last probes, max |delta f|
  unsigned err;     // bounded waits that gave up
  unsigned pad;
};

struct Level {
  bool binned = false;
  int64_t n = 0;         // columns
  int64_t ld = 0;        // row pitch (elements)
  void* v = nullptr;     // K x ld, owned if binned
  int32_t* H = nullptr;  // counts (binned)
  int64_t* keys = nullptr;
  double w = 0.0;
  int64_t n_sched = 0;  // n used by Algorithm 1's break rule
  bool fact = false;    // unbinned data of a factorised context: generated from (a, b, phi), no store
  CUtensorMap tmap;
  const float* vT = nullptr;  // binned FP32: a sample-major copy (n x stage_pitch(K)), not owned
};

}  // namespace

struct mbar_ctx {
  int64_t K = 0, N = 0;
  int dtype = 4;
  mbar_opts opts{};
  cudaStream_t st = nullptr;
  std::vector<double> Nk_h;
  double* Nk_d = nullptr;
  double* logN_d = nullptr;
  // unbinned data in the current column order (allocated when first needed)
  void* v = nullptr;
  // sample-major copy of the data (vst[n * stage_pitch(K) + k], original
  // sample order): from creation until v is formed, and for MIXED for good
  // (the unbinned LSE passes stream it)
  void* vst = nullptr;
  float* logden_orig = nullptr;  // MIXED: logden of those passes, original order
  bool smaj = false;             // unbinned passes on the sample-major copy
  // the next unbinned pass only confirms a Newton step already below f_tol:
  // the plain FP32 sums suffice (every other unbinned pass splits each
  // sample's largest weight into an exact count and its remainder)
  bool confirm_only = false;
  // factorised context (u_kn = a_k + b_k phi_n, MIXED): no K x N store; the
  // binned levels are generated from a, b and the bin means of phi, the
  // unbinned passes and the Hessian read phi (original sample order)
  bool fact = false;
  double *fa = nullptr, *fb = nullptr, *fphi = nullptr;
  double* logden64 = nullptr;  // logden of the factorised unbinned passes (FP64, original order)
  void* fref = nullptr;        // reference-state table of the factorised unbinned passes
  int64_t ld = 0;
  double* cshift = nullptr;  // mixed: per-column shift (current order)
  int32_t* perm = nullptr;   // current column -> original sample
  double* phi0 = nullptr;    // default bin coordinate (row 0 of u, original order)
  double* phi_sorted = nullptr;
  double* d_sorted = nullptr;  // phi_sorted - min(phi)
  float2* d_pairs = nullptr;   // FP32 (hi, lo) split of d_sorted
  bool sorted = false;
  double phi_lo = 0.0, phi_hi = 0.0;
  Level full;  // unbinned level view (not owning)
  Level cur;   // level selected through mbar_bin / mbar_bin_count
  // iteration state
  double *f = nullptr, *fs = nullptr, *ft = nullptr, *fts = nullptr;
  double *g = nullptr, *gt = nullptr, *Q = nullptr, *s = nullptr, *s2 = nullptr, *d = nullptr;
  double *hess = nullptr, *delta = nullptr;
  int* info = nullptr;
  int* bad = nullptr;
  Ctrl* ctrl = nullptr;
  DevStatus* stat = nullptr;   // device
  DevStatus* hstat = nullptr;  // pinned host mirror
  void* logden = nullptr;  // N entries, dtype
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  int32_t* seg = nullptr;  // N, bin ordinal of each sorted sample
  int32_t* start = nullptr;
  unsigned long long* count = nullptr;
  int32_t* nb_dev = nullptr;
  std::vector<double> f_h;
  std::unordered_map<void*, size_t> live;  // device allocations -> bytes
  int64_t bytes = 0;
  // opt-in kernel timing (CUDA events on the context's stream)
  struct Rec {
    cudaEvent_t a, b;
    int kind;
    double bytes;
  };
  bool timing = false;
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  // solver trace: (phase, n, a, b) rows, see mbar_get_trace
  std::vector<double> trace;
  double t_width = 0.0, t_levels = 0.0;  // host seconds, accumulated during a solve
  cudaStream_t ust = nullptr;            // the caller's stream
  bool graphs = true;                    // capture the binned loops into CUDA graphs
  FirstLoopBatcher* batcher = nullptr;   // first loops through a shared persistent launch
  double* weights = nullptr;             // last mbar_reweight weights (original sample order)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
};

namespace {

mbar_status dalloc(mbar_ctx* c, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMallocAsync(p, bytes, c->st);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_status(e, "cudaMallocAsync");
  }
  c->bytes += static_cast<int64_t>(bytes);
  c->live[*p] = bytes;
  return MBAR_OK;
}

template <typename T>
mbar_status dalloc_t(mbar_ctx* c, T** p, size_t count) {
  void* q = nullptr;
  BUMBAR_TRY(dalloc(c, &q, count * sizeof(T)));
  *p = static_cast<T*>(q);
  return MBAR_OK;
}

void dfree(mbar_ctx* c, void* p) {
  if (!p) return;
  auto it = c->live.find(p);
  if (it != c->live.end()) {
    c->bytes -= static_cast<int64_t>(it->second);
    c->live.erase(it);
  }
  cudaFreeAsync(p, c->st);
}

void level_free(mbar_ctx* c, Level* L) {
  if (L->binned) {
    dfree(c, L->v);
    dfree(c, L->H);
    dfree(c, L->keys);
  }
  *L = Level{};
}

mbar_status level_tmap(mbar_ctx* c, Level* L) {
  const int C = 128 / c->dtype;
  const int box_rows = static_cast<int>(std::min<int64_t>(256, round_up(c->K, 8)));
  return make_tmap_2d(&L->tmap, L->v, c->dtype == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                      c->dtype, c->K, L->n, L->ld, C, box_rows);
}

cudaEvent_t take_event(mbar_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets one timed launch: call with begin=true before and false after.
void time_mark(mbar_ctx* c, bool begin, int kind, double bytes) {
  if (!c->timing) return;
  if (begin) {
    mbar_ctx::Rec r{take_event(c), take_event(c), kind, bytes};
    cudaEventRecord(r.a, c->st);
    c->recs.push_back(r);
  } else {
    // the most recent record of this kind (brackets of other kinds may nest
    // inside, e.g. an unbinned pass inside a second-loop round)
    for (auto it = c->recs.rbegin(); it != c->recs.rend(); ++it)
      if (it->kind == kind) {
        cudaEventRecord(it->b, c->st);
        break;
      }
  }
}

void trace_row(mbar_ctx* c, double phase, double n, double a, double b) {
  c->trace.insert(c->trace.end(), {phase, n, a, b});
}

// One pass of the fused LSE kernel over a level.
mbar_status run_lse(mbar_ctx* c, const Level& L, const double* f_in, int mode, double* f_out, double* g_out,
                    double* s_out, double eps, int skip_if_done, void* logden_out, double* d_out = nullptr,
                    double noise = 0.0) {
  const LsePlan pl = lse_plan(c->K, L.n, c->dtype);
  LseParams p{};
  p.K = static_cast<int>(c->K);
  p.n = static_cast<int>(L.n);
  p.f = f_in;
  p.logN = c->logN_d;
  p.H = L.H;
  unsigned char* sc = static_cast<unsigned char*>(c->scratch);
  p.counter = reinterpret_cast<unsigned*>(sc);
  p.err = &c->stat->err;
  p.partials = reinterpret_cast<double*>(sc + 256);
  p.Q = c->Q;
  p.logden = logden_out;
  p.mode = mode;
  p.Nk = c->Nk_d;
  p.f_out = f_out;
  p.g_out = g_out;
  p.s_out = s_out;
  p.ctrl = c->ctrl;
  p.eps = eps;
  p.noise = noise;
  p.d_out = d_out;
  p.skip_if_done = skip_if_done;
  p.skip_if_underflow = mode == kLseModeSci ? 1 : 0;
  const bool timed = !L.binned;
  const int tkind = (c->confirm_only && ((c->smaj && c->vst) || c->fact)) ? 3 : 0;
  // bytes the pass reads: the level's data, or phi for factorised data
  if (timed) time_mark(c, true, tkind, c->fact ? 8.0 * L.n : static_cast<double>(c->K) * L.n * c->dtype);
  mbar_status s = MBAR_OK;
  if (!L.binned && c->fact) {
    // factorised context: u generated from (a, b, phi) in registers; logden
    // in FP64 and the original sample order
    p.H = nullptr;
    p.logden = logden_out ? c->logden64 : nullptr;
    p.exact_max = c->confirm_only ? 0 : 1;
    // phi's range from the sorted copy: its first and last element
    s = lse_fact_launch(c->fa, c->fb, c->fphi, lse_fact_plan(c->K, L.n), p, c->phi_sorted, c->phi_sorted + c->N - 1,
                        1, c->fref, c->st);
  } else if (L.binned && L.vT && !logden_out) {
    // a large binned FP32 level with a sample-major copy (the second loop's
    // current level): the sample-major pass streams whole contiguous bins
    p.exact_max = 0;
    s = lse_smaj_launch(L.vT, lse_smaj_plan(c->K, L.n), p, c->st);
  } else if (!L.binned && c->smaj && c->vst) {
    // unbinned MIXED pass over the sample-major copy (original sample order);
    // logden comes back to the store's column order through perm
    p.logden = logden_out ? c->logden_orig : nullptr;
    p.exact_max = c->confirm_only ? 0 : 1;
    s = lse_smaj_launch(static_cast<const float*>(c->vst), lse_smaj_plan(c->K, L.n), p, c->st);
    if (s == MBAR_OK && logden_out) s = gather_columns(c->logden_orig, logden_out, 4, 1, L.n, L.n, c->perm, c->st);
  } else {
    s = lse_launch(L.tmap, pl, p, c->dtype, c->st);
  }
  if (timed) time_mark(c, false, tkind, 0);
  return s;
}

unsigned* err_word(mbar_ctx* c) { return &c->stat->err; }

// One pinned copy of the status block, one sync; then the error checks.
mbar_status read_status(mbar_ctx* c) {
  BUMBAR_CUDA(cudaMemcpyAsync(c->hstat, c->stat, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->st));
  BUMBAR_CUDA(cudaStreamSynchronize(c->st));
  if (c->hstat->err) {
    set_error("a bounded device-side wait gave up (%u CTAs)", c->hstat->err);
    BUMBAR_CUDA(cudaMemsetAsync(&c->stat->err, 0, sizeof(unsigned), c->st));
    return MBAR_ETIMEOUT;
  }
  if (c->hstat->ctrl.nonfinite) {
    set_error("non-finite free energies (a state lost all weight)");
    BUMBAR_CUDA(cudaMemsetAsync(&c->ctrl->nonfinite, 0, sizeof(int), c->st));
    return MBAR_ENOTCONV;
  }
  return MBAR_OK;
}

mbar_status check_device_errors(mbar_ctx* c) { return read_status(c); }

// True (and the device flag cleared) when the last SCI step(s) read by
// read_status stopped on an underflowed state.
bool take_underflow(mbar_ctx* c) {
  if (!c->hstat->ctrl.underflow) return false;
  c->hstat->ctrl.underflow = 0;
  cudaMemsetAsync(&c->ctrl->underflow, 0, sizeof(int), c->st);
  return true;
}

// The SCI step of run_lse redone exactly in the log domain: logden by a
// pass over the level, then log Q_k = LSE_p(log H_p + a_k - v_kp - logden_p).
mbar_status log_sci_step(mbar_ctx* c, const Level& L, const double* f_in, double* f_out, double* g_out,
                         double* s_out, double eps, double* d_out, double noise) {
  if (!L.binned && c->fact) {
    set_error("a step on the unbinned factorised data underflowed (a state lost all weight); the log-domain redo "
              "needs a stored level");
    return MBAR_ENOTCONV;
  }
  BUMBAR_TRY(run_lse(c, L, f_in, kLseModePass, nullptr, nullptr, nullptr, 0.0, 0, c->logden));
  LseParams p{};
  p.K = static_cast<int>(c->K);
  p.n = static_cast<int>(L.n);
  p.f = f_in;
  p.logN = c->logN_d;
  p.H = L.H;
  p.logden = c->logden;
  p.Q = c->Q;
  p.mode = kLseModeSci;
  p.Nk = c->Nk_d;
  p.f_out = f_out;
  p.g_out = g_out;
  p.s_out = s_out;
  p.d_out = d_out;
  p.ctrl = c->ctrl;
  p.eps = eps;
  p.noise = noise;
  void* tmp = nullptr;
  const size_t bytes = log_sci_tmp_bytes(c->K, L.n);
  BUMBAR_TRY(dalloc(c, &tmp, bytes));
  const mbar_status s = log_sci_finish(L.v, c->dtype, c->K, L.n, L.ld, p, tmp, bytes, c->st);
  dfree(c, tmp);
  return s;
}

// One SCI step with its status read back; a step that underflowed is redone
// in the log domain.
mbar_status sci_step_exact(mbar_ctx* c, const Level& L, const double* f_in, double* f_out, double* g_out,
                           double* s_out, void* logden_out, double* d_out = nullptr) {
  BUMBAR_TRY(run_lse(c, L, f_in, kLseModeSci, f_out, g_out, s_out, 0.0, 0, logden_out, d_out));
  BUMBAR_TRY(read_status(c));
  if (take_underflow(c)) {
    BUMBAR_TRY(log_sci_step(c, L, f_in, f_out, g_out, s_out, 0.0, d_out, 0.0));
    BUMBAR_TRY(read_status(c));
  }
  return MBAR_OK;
}

// The Hessian at f on level L, with logden at f from the last pass over L.
// Unbinned MIXED data with a tensor-core K read the sample-major copy
// (contiguous 64-sample runs for the kernel's TMA boxes; logden in that
// order); everything else the level's row-major store.
mbar_status level_hessian(mbar_ctx* c, const Level& L, const double* f, void* tmp, size_t htmp) {
  if (!L.binned && c->fact)
    return hessian_fact(c->fa, c->fb, c->fphi, c->K, L.n, f, c->logN_d, c->logden64, c->hess, err_word(c), tmp, htmp,
                        c->st);
  if (!L.binned && c->smaj && c->vst && c->dtype == 4 && hessian_smaj_eligible(c->K))
    return hessian_smaj(static_cast<const float*>(c->vst), c->K, L.n, f, c->logN_d,
                        static_cast<const float*>(c->logden_orig), c->hess, err_word(c), tmp, htmp, c->st);
  return hessian(L.v, c->dtype, c->K, L.n, L.ld, f, c->logN_d, c->logden, L.binned ? L.H : nullptr, c->hess,
                 err_word(c), tmp, htmp, c->st);
}

mbar_status ensure_sorted(mbar_ctx* c);

// Histogram at width w over the sorted coordinate -> a binned level.
mbar_status make_level_w_impl(mbar_ctx* c, double w, Level* L);
mbar_status fill_level_stores(mbar_ctx* c, int L, const int32_t* const* seg, const int32_t* const* start,
                              const int64_t* nb, void* const* out, const int64_t* ld);

mbar_status make_level_w(mbar_ctx* c, double w, Level* L) {
  const double t0 = now_s();
  const mbar_status s = make_level_w_impl(c, w, L);
  c->t_levels += now_s() - t0;
  return s;
}

mbar_status make_level_w_impl(mbar_ctx* c, double w, Level* L) {
  *L = Level{};
  BUMBAR_TRY(ensure_sorted(c));
  const size_t htmp = hist_tmp_bytes(c->N);
  const size_t mtmp = bin_means_tmp_bytes(c->K, c->N);
  void* tmp = nullptr;
  BUMBAR_TRY(dalloc(c, &tmp, std::max(htmp, mtmp)));
  int64_t* keys_full = nullptr;
  int32_t* H_full = nullptr;
  mbar_status s = dalloc_t(c, &keys_full, c->N);
  if (s == MBAR_OK) s = dalloc_t(c, &H_full, c->N);
  if (s == MBAR_OK)
    s = build_histogram(c->d_pairs, c->d_sorted, c->N, w, c->seg, c->start, H_full, keys_full, c->nb_dev, tmp, htmp,
                        c->st);
  int32_t nb = 0;
  if (s == MBAR_OK) {
    cudaError_t e = cudaMemcpyAsync(&nb, c->nb_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) s = cuda_status(e, "histogram size");
  }
  if (s == MBAR_OK) {
    L->binned = true;
    L->n = nb;
    L->ld = round_up(nb, 32);
    L->w = w;
    L->n_sched = nb;
    s = dalloc(c, &L->v, static_cast<size_t>(c->K) * L->ld * c->dtype);
  }
  if (s == MBAR_OK) s = dalloc_t(c, &L->H, nb);
  if (s == MBAR_OK) s = dalloc_t(c, &L->keys, nb);
  if (s == MBAR_OK) {
    cudaError_t e = cudaMemcpyAsync(L->H, H_full, nb * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(L->keys, keys_full, nb * sizeof(int64_t), cudaMemcpyDeviceToDevice, c->st);
    if (e != cudaSuccess) s = cuda_status(e, "histogram copy");
  }
  if (s == MBAR_OK) {
    if (c->fact) {
      const int32_t* sg1 = c->seg;
      const int32_t* st1 = c->start;
      const int64_t nb1 = nb;
      void* out1 = L->v;
      const int64_t ld1 = L->ld;
      s = fill_level_stores(c, 1, &sg1, &st1, &nb1, &out1, &ld1);
    } else {
      s = bin_means(c->v, c->dtype, c->K, c->N, c->ld, c->seg, c->start, nb, L->v, L->ld, tmp, mtmp, c->st);
    }
  }
  if (s == MBAR_OK) s = level_tmap(c, L);
  dfree(c, tmp);
  dfree(c, keys_full);
  dfree(c, H_full);
  if (s != MBAR_OK) level_free(c, L);
  return s;
}

mbar_status count_at(mbar_ctx* c, const double* ws, int nw, int64_t* g) {
  BUMBAR_TRY(count_bins(c->d_pairs, c->d_sorted, c->N, ws, nw, c->count, c->st));
  unsigned long long h[kWidthsPerPass];
  BUMBAR_CUDA(cudaMemcpyAsync(h, c->count, nw * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->st));
  BUMBAR_CUDA(cudaStreamSynchronize(c->st));
  for (int i = 0; i < nw; ++i) g[i] = static_cast<int64_t>(h[i]);
  return MBAR_OK;
}

mbar_status width_search_multi(mbar_ctx* c, const int64_t* n, int count, double* w_out, bool* found);

// Width rule w*(n) by the deterministic search (width_search_multi with one
// target); *found = false when n cannot be reached (the caller then uses the
// unbinned data).
mbar_status width_search(mbar_ctx* c, int64_t n, double* w_out, bool* found) {
  return width_search_multi(c, &n, 1, w_out, found);
}

// Forms the row-major store v from the sample-major staging, columns in the
// order perm (absolute: column i holds original sample perm[i]); FP64
// releases the staging.
mbar_status form_store(mbar_ctx* c, const int32_t* perm) {
  void* v = nullptr;
  BUMBAR_TRY(dalloc(c, &v, static_cast<size_t>(c->K) * c->ld * c->dtype));
  mbar_status s = gather_transpose(c->vst, c->dtype, c->K, c->N, perm, v, c->ld, c->st);
  if (s != MBAR_OK) {
    dfree(c, v);
    return s;
  }
  if (!c->smaj) {  // the sample-major copy stays only where the LSE passes stream it
    dfree(c, c->vst);
    c->vst = nullptr;
  }
  c->v = v;
  c->full.v = v;
  BUMBAR_TRY(level_tmap(c, &c->full));
  if (!c->cur.binned) c->cur = c->full;
  return MBAR_OK;
}

// The unbinned store in the current column order (the identity until a
// coordinate is set).
mbar_status ensure_store(mbar_ctx* c) {
  if (c->v || c->fact) return MBAR_OK;
  return form_store(c, c->perm);
}

mbar_status set_coordinate_dev(mbar_ctx* c, const double* phi_orig) {
  // phi in the caller's original order -> current column order
  const int64_t N = c->N;
  double* phi_cur = nullptr;
  int32_t* perm_rel = nullptr;
  void* tmp = nullptr;
  const size_t stmp = sort_tmp_bytes(N);
  // while the data is still staged the current order is the original one
  // (perm = identity) and the store is formed directly in the sorted order
  const bool staged = c->v == nullptr;
  const size_t vbytes = staged ? 0 : static_cast<size_t>(c->K) * c->ld * c->dtype;
  BUMBAR_TRY(dalloc_t(c, &phi_cur, N));
  mbar_status s = dalloc_t(c, &perm_rel, N);
  if (s == MBAR_OK) s = dalloc(c, &tmp, std::max<size_t>(stmp, vbytes));
  // phi_cur[i] = phi[perm[i]]
  if (s == MBAR_OK) s = gather_columns(phi_orig, phi_cur, 8, 1, N, N, c->perm, c->st);
  if (s == MBAR_OK) s = sort_coordinate(phi_cur, N, c->phi_sorted, perm_rel, tmp, stmp, c->st);
  if (s == MBAR_OK) s = offsets_from_min(c->phi_sorted, N, c->d_sorted, c->d_pairs, c->st);
  // reorder the data columns and the bookkeeping by perm_rel
  if (staged) {
    if (s == MBAR_OK) s = form_store(c, perm_rel);
  } else {
    if (s == MBAR_OK) s = gather_columns(c->v, tmp, c->dtype, c->K, N, c->ld, perm_rel, c->st);
    if (s == MBAR_OK) {
      std::swap(c->v, tmp);
      c->full.v = c->v;
    }
    if (s == MBAR_OK) s = level_tmap(c, &c->full);
  }
  if (s == MBAR_OK && c->cshift) {
    s = gather_columns(c->cshift, phi_cur, 8, 1, N, N, perm_rel, c->st);  // phi_cur reused as scratch
    if (s == MBAR_OK) {
      cudaError_t e = cudaMemcpyAsync(c->cshift, phi_cur, N * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
      if (e != cudaSuccess) s = cuda_status(e, "shift reorder");
    }
  }
  if (s == MBAR_OK) {
    // perm_new[i] = perm[perm_rel[i]]
    int32_t* pn = reinterpret_cast<int32_t*>(phi_cur);
    s = gather_columns(c->perm, pn, 4, 1, N, N, perm_rel, c->st);
    if (s == MBAR_OK) {
      cudaError_t e = cudaMemcpyAsync(c->perm, pn, N * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->st);
      if (e != cudaSuccess) s = cuda_status(e, "perm update");
    }
  }
  if (s == MBAR_OK) {
    cudaError_t e = cudaMemcpyAsync(&c->phi_lo, c->phi_sorted, sizeof(double), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&c->phi_hi, c->phi_sorted + N - 1, sizeof(double), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) s = cuda_status(e, "coordinate range");
  }
  dfree(c, tmp);
  dfree(c, phi_cur);
  dfree(c, perm_rel);
  if (s == MBAR_OK) {
    c->sorted = true;
    level_free(c, &c->cur);
    c->cur = c->full;
  }
  return s;
}

mbar_status ensure_sorted(mbar_ctx* c) {
  if (c->sorted) return MBAR_OK;
  return set_coordinate_dev(c, c->phi0);
}

mbar_status h2d(mbar_ctx* c, double* dst, const double* src, int64_t n) {
  BUMBAR_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyHostToDevice, c->st));
  return MBAR_OK;
}

mbar_status d2h(mbar_ctx* c, double* dst, const double* src, int64_t n) {
  BUMBAR_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  return MBAR_OK;
}

double max_abs(const std::vector<double>& x) {
  double m = 0.0;
  for (double v : x) m = std::max(m, std::fabs(v));
  return m;
}

// step halvings of a rejected Newton step before the SCI fallback
constexpr int kMaxHalvings = 12;

mbar_status newton_phase(mbar_ctx* c, mbar_report* rep) {
  const int64_t K = c->K;
  const Level& L = c->full;
  std::vector<double> gh(K), dh(K);
  // evaluate at f: SCI step (fs), gradient (g), logden
  BUMBAR_TRY(sci_step_exact(c, L, c->f, c->fs, c->g, c->s, c->logden));
  BUMBAR_TRY(d2h(c, gh.data(), c->g, K));
  BUMBAR_CUDA(cudaStreamSynchronize(c->st));
  double gmax = max_abs(gh);
  const size_t htmp = hessian_tmp_bytes(K, L.n);
  const size_t ntmp = newton_tmp_bytes(K);
  void* tmp = nullptr;
  BUMBAR_TRY(dalloc(c, &tmp, std::max(htmp, ntmp)));
  mbar_status st = MBAR_ENOTCONV;
  int rejects = 0;
  double prev_step = INFINITY;
  // the rounding floor of a gradient evaluation: below it max|g| says
  // nothing about whether a step helped (FP32 data and exponentials, with
  // each sample's largest weight split into an exact count and its small
  // remainder, give ~1e-9 of N_k; FP64 ~1e-13)
  double nk_max = 0.0;
  for (int64_t k = 0; k < K; ++k) nk_max = std::max(nk_max, c->Nk_h[k]);
  const double g_floor = (c->dtype == 4 ? 1e-8 : 1e-13) * nk_max;
  for (int it = 0; it < c->opts.max_newton; ++it) {
    if (gmax == 0.0 || K == 1) {
      st = MBAR_OK;
      break;
    }
    rep->iters_newton++;
    time_mark(c, true, 1, static_cast<double>(K) * L.n * c->dtype);
    mbar_status s = level_hessian(c, L, c->f, tmp, htmp);
    time_mark(c, false, 1, 0);
    if (s == MBAR_OK) s = cudaMemsetAsync(c->info, 0, sizeof(int), c->st) == cudaSuccess ? MBAR_OK : MBAR_ECUDA;
    time_mark(c, true, 2, static_cast<double>(K) * K * 8);
    if (s == MBAR_OK) s = newton_solve(c->hess, K, c->g, c->delta, c->info, tmp, ntmp, c->st);
    time_mark(c, false, 2, 0);
    int info = 0;
    if (s == MBAR_OK) {
      cudaError_t e = cudaMemcpyAsync(&info, c->info, sizeof(int), cudaMemcpyDeviceToHost, c->st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(dh.data(), c->delta, K * sizeof(double), cudaMemcpyDeviceToHost, c->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
      if (e != cudaSuccess) s = cuda_status(e, "newton readback");
    }
    if (s != MBAR_OK) {
      dfree(c, tmp);
      return s;
    }
    const double step = max_abs(dh);
    double g2 = 0.0;  // ||g||^2 at f
    for (double x : gh) g2 += x * x;
    bool accepted = false;
    if (info == 0 && std::isfinite(step)) {
      s = vec_add_gauge(c->f, c->delta, c->ft, K, c->st);
      // a step below f_tol is accepted and ends the phase whatever the
      // gradient at its end: that evaluation only confirms it
      c->confirm_only = step < c->opts.f_tol;
      if (s == MBAR_OK) s = sci_step_exact(c, L, c->ft, c->fts, c->gt, c->s2, c->logden);
      c->confirm_only = false;
      if (s == MBAR_OK) s = d2h(c, gh.data(), c->gt, K);
      if (s == MBAR_OK && cudaStreamSynchronize(c->st) != cudaSuccess) s = MBAR_ECUDA;
      if (s != MBAR_OK && s != MBAR_ENOTCONV) {
        dfree(c, tmp);
        return s;
      }
      const double gmax_t = (s == MBAR_OK) ? max_abs(gh) : INFINITY;
      if (std::isfinite(gmax_t) && (gmax_t <= gmax || step <= 10.0 * c->opts.f_tol || gmax_t <= g_floor)) {
        std::swap(c->f, c->ft);
        std::swap(c->fs, c->fts);
        std::swap(c->g, c->gt);
        gmax = gmax_t;
        accepted = true;
        rejects = 0;
        rep->last_step = step;
        trace_row(c, 3, it, step, gmax);
        if (step < c->opts.f_tol) {
          st = MBAR_OK;
          break;
        }
        // Newton contracts quadratically; accepted steps that stop shrinking
        // while already small are moving on the rounding noise of the gradient
        if (step > 0.5 * prev_step && step < 1e2 * c->opts.f_tol) {
          st = MBAR_OK;
          break;
        }
        prev_step = step;
      }
      // A rejected full step well above the gradient's rounding noise (f far
      // from the root, e.g. after coarse levels on a long replica ladder):
      // backtrack along the Newton direction. It is the direction of
      // Newton's method for g(f) = 0, whose Jacobian is the Hessian, so a
      // short enough step lowers ||g||^2 (Armijo test on ||g||^2 / 2).
      for (int h = 1; !accepted && step >= 1e2 * c->opts.f_tol && h <= kMaxHalvings; ++h) {
        const double t = std::ldexp(1.0, -h);
        s = vec_add_gauge(c->f, c->delta, c->ft, K, c->st, t);
        if (s == MBAR_OK) s = sci_step_exact(c, L, c->ft, c->fts, c->gt, c->s2, c->logden);
        if (s == MBAR_OK) s = d2h(c, gh.data(), c->gt, K);
        if (s == MBAR_OK && cudaStreamSynchronize(c->st) != cudaSuccess) s = MBAR_ECUDA;
        if (s != MBAR_OK && s != MBAR_ENOTCONV) {
          dfree(c, tmp);
          return s;
        }
        if (s != MBAR_OK) continue;  // the trial underflowed: shorter still
        double g2t = 0.0;
        for (double x : gh) g2t += x * x;
        if (!std::isfinite(g2t) || g2t > (1.0 - 2e-4 * t) * g2) continue;
        std::swap(c->f, c->ft);
        std::swap(c->fs, c->fts);
        std::swap(c->g, c->gt);
        gmax = max_abs(gh);
        accepted = true;
        rejects = 0;
        rep->last_step = t * step;
        prev_step = INFINITY;  // a damped step says nothing about quadratic contraction
        trace_row(c, 5, it, t * step, gmax);
      }
    }
    if (!accepted) {
      // Newton step did not lower max|g|: take the SCI step from f instead
      rep->newton_fallbacks++;
      trace_row(c, 4, it, step, gmax);
      rejects++;
      if (rejects >= 3 && step < 1e2 * c->opts.f_tol) {  // at the noise floor of the gradient
        st = MBAR_OK;
        break;
      }
      std::swap(c->f, c->fs);
      s = sci_step_exact(c, L, c->f, c->fs, c->g, c->s, c->logden);
      if (s == MBAR_OK) s = d2h(c, gh.data(), c->g, K);
      if (s == MBAR_OK && cudaStreamSynchronize(c->st) != cudaSuccess) s = MBAR_ECUDA;
      if (s != MBAR_OK) {
        dfree(c, tmp);
        return s;
      }
      gmax = max_abs(gh);
    }
  }
  dfree(c, tmp);
  rep->max_abs_grad = gmax;
  if (st == MBAR_ENOTCONV)
    set_error("Newton phase: no convergence in %d iterations (last step %.3g, max|g| %.3g)", c->opts.max_newton,
              rep->last_step, gmax);
  return st;
}

// A captured sequence of launches on the context's stream, replayed with
// one cudaGraphLaunch (the binned loops of Algorithm 1 launch the same
// kernels with the same arguments many times).
struct Graph {
  cudaGraphExec_t exec = nullptr;
  ~Graph() { reset(); }
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
  }
};

template <typename F>
mbar_status capture(mbar_ctx* c, Graph* g, F&& body) {
  g->reset();
  BUMBAR_CUDA(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
  const mbar_status s = body();
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c->st, &graph);
  if (s != MBAR_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture");
  const cudaError_t e2 = cudaGraphInstantiate(&g->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e2 != cudaSuccess) return cuda_status(e2, "cudaGraphInstantiate");
  return MBAR_OK;
}

// The in-place SCI steps of a small FP32 level over the whole GPU
// (sci_grid_launch): only where this solve has the device to itself -- a
// context that captures graphs; server workers share the GPU with other
// solves, which a cooperative launch of every SM would hold up.
bool use_grid_loop(const mbar_ctx* c, int64_t n) {
  return c->graphs && c->dtype == 4 && sci_grid_supported(c->K, n);
}

// Phase-1 loop of Algorithm 1 on level L: guarded in-place SCI steps until
// s < eps (the guard turns later launches of a batch into no-ops). A binned
// level replays a captured batch of kPhase1Batch launches.
// The first loop on a small FP32 level in single launches (sci_loop.cu): the
// level is transposed to sample-major once; an underflowed step stops the
// kernel and is redone exactly here, then the loop resumes.
mbar_status first_loop_fused(mbar_ctx* c, const Level& L, mbar_report* rep) {
  BUMBAR_CUDA(cudaMemsetAsync(c->ctrl, 0, sizeof(Ctrl), c->st));
  float* vT = nullptr;
  BUMBAR_TRY(dalloc(c, reinterpret_cast<void**>(&vT), sci_loop_level_bytes(c->K, L.n)));
  mbar_status s = level_to_samples(static_cast<const float*>(L.v), c->K, L.n, L.ld, vT, c->st);
  void* grid_scr = nullptr;
  if (s == MBAR_OK && use_grid_loop(c, L.n)) s = dalloc(c, &grid_scr, sci_grid_scratch_bytes(c->K));
  SciLoopParams q{};
  q.K = static_cast<int>(c->K);
  q.n = static_cast<int>(L.n);
  q.H = L.H;
  q.f = c->f;
  q.logN = c->logN_d;
  q.Nk = c->Nk_d;
  q.ctrl = c->ctrl;
  q.s_out = c->s;
  q.d_out = nullptr;
  q.err = err_word(c);
  q.eps = c->opts.eps;
  q.noise = c->opts.noise_floor;
  int64_t done_iters = 0;
  while (s == MBAR_OK) {
    q.max_steps = c->opts.max_sci - done_iters;
    time_mark(c, true, 5, 0.0);
    s = grid_scr ? sci_grid_launch(vT, q, grid_scr, c->st) : sci_loop_launch(vT, q, c->st);
    time_mark(c, false, 5, 0.0);
    if (s == MBAR_OK) s = read_status(c);
    // the launch streamed the level once per step it took
    if (s == MBAR_OK && c->timing && !c->recs.empty())
      c->recs.back().bytes = static_cast<double>(c->hstat->ctrl.iters - done_iters) * c->K * L.n * 4.0;
    if (s != MBAR_OK) break;
    const bool redo = take_underflow(c);
    if (redo) {
      s = log_sci_step(c, L, c->f, c->f, nullptr, c->s, c->opts.eps, nullptr, c->opts.noise_floor);
      if (s == MBAR_OK) s = read_status(c);
      if (s != MBAR_OK) break;
    }
    const Ctrl h = c->hstat->ctrl;
    done_iters = h.iters;
    if (h.done || done_iters >= c->opts.max_sci) {
      trace_row(c, 1, static_cast<double>(L.n_sched), h.last_s, static_cast<double>(done_iters));
      break;
    }
    if (!redo) {
      set_error("first loop: the fused SCI kernel stopped without converging");
      s = MBAR_ENOTCONV;
    }
  }
  dfree(c, vT);
  dfree(c, grid_scr);
  if (s == MBAR_OK) rep->iters_first_loop += done_iters;
  return s;
}

constexpr double kFusedFirstBytes = 4.0 * (1 << 20);

// The first loop through the context's batcher: the level sample-major, one
// item of a shared persistent launch (batch_loop.cu); a loop that stopped on
// an underflowed step continues with the one-problem path, which redoes it.
mbar_status first_loop_batched(mbar_ctx* c, const Level& L, mbar_report* rep) {
  float* vT = nullptr;
  BUMBAR_TRY(dalloc(c, reinterpret_cast<void**>(&vT), sci_loop_level_bytes(c->K, L.n)));
  mbar_status s = level_to_samples(static_cast<const float*>(L.v), c->K, L.n, L.ld, vT, c->st);
  if (s == MBAR_OK && cudaMemsetAsync(c->ctrl, 0, sizeof(Ctrl), c->st) != cudaSuccess) s = MBAR_ECUDA;
  if (s == MBAR_OK && cudaStreamSynchronize(c->st) != cudaSuccess) s = MBAR_ECUDA;
  if (s == MBAR_OK) {
    BatchLoopItem q{};
    q.vT = vT;
    q.K = static_cast<int>(c->K);
    q.n = static_cast<int>(L.n);
    q.Kp = static_cast<int>(stage_pitch(c->K));
    q.H = L.H;
    q.f = c->f;
    q.logN = c->logN_d;
    q.Nk = c->Nk_d;
    q.ctrl = c->ctrl;
    q.s_out = c->s;
    q.eps = c->opts.eps;
    q.noise = c->opts.noise_floor;
    q.max_steps = c->opts.max_sci;
    s = first_loop_batcher_run(c->batcher, q);
  }
  if (s == MBAR_OK) s = read_status(c);
  dfree(c, vT);
  if (s != MBAR_OK) return s;
  const Ctrl h = c->hstat->ctrl;
  rep->iters_first_loop += h.iters;
  if (!h.underflow && (h.done || h.iters >= c->opts.max_sci)) {
    trace_row(c, 1, static_cast<double>(L.n_sched), h.last_s, static_cast<double>(h.iters));
    return MBAR_OK;
  }
  return first_loop_fused(c, L, rep);
}

mbar_status first_loop(mbar_ctx* c, const Level& L, mbar_report* rep) {
  if (c->batcher && c->dtype == 4 && L.binned && first_loop_batch_supported(c->K, L.n))
    return first_loop_batched(c, L, rep);
  if (c->dtype == 4 && L.binned && (use_grid_loop(c, L.n) || sci_loop_supported(c->K, L.n, kFusedFirstBytes)))
    return first_loop_fused(c, L, rep);
  BUMBAR_CUDA(cudaMemsetAsync(c->ctrl, 0, sizeof(Ctrl), c->st));
  auto batch = [&]() -> mbar_status {
    for (int b = 0; b < kPhase1Batch; ++b)
      BUMBAR_TRY(run_lse(c, L, c->f, kLseModeSci, c->f, nullptr, c->s, c->opts.eps, 1, nullptr, nullptr,
                         c->opts.noise_floor));
    return MBAR_OK;
  };
  Graph g;
  const bool use_graph = L.binned && c->graphs;  // unbinned launches carry timing events
  if (use_graph) BUMBAR_TRY(capture(c, &g, batch));
  int64_t done_iters = 0;
  for (;;) {
    if (use_graph) {
      BUMBAR_CUDA(cudaGraphLaunch(g.exec, c->st));
      count_launches(kPhase1Batch);
    } else {
      BUMBAR_TRY(batch());
    }
    BUMBAR_TRY(read_status(c));
    if (take_underflow(c)) {  // the batch stopped at that step: redo it exactly
      BUMBAR_TRY(log_sci_step(c, L, c->f, c->f, nullptr, c->s, c->opts.eps, nullptr, c->opts.noise_floor));
      BUMBAR_TRY(read_status(c));
    }
    const Ctrl h = c->hstat->ctrl;
    done_iters = h.iters;
    if (h.done || done_iters >= c->opts.max_sci) {
      trace_row(c, 1, static_cast<double>(L.n_sched), h.last_s, static_cast<double>(done_iters));
      break;
    }
  }
  rep->iters_first_loop += done_iters;
  return MBAR_OK;
}

// The width rule for several bin counts at once. Each search is the
// sequential procedure of width_search (halving, then at most 64 geometric
// bisections); one counting pass serves all of them: a halving search
// contributes its current width, a bisecting one the midpoints of the next
// d levels of its bisection tree, the 15 widths of a pass shared out so that
// d is as large as the share allows. Results are those of the sequential
// searches, one by one.
struct WidthSearch {
  int64_t n = 0;
  double w_lo = 0.0, w_hi = 0.0;
  int phase = 0;  // 0 halving, 1 bisecting, 2 done
  bool found = true;
  int steps = 0;
};

mbar_status width_search_multi(mbar_ctx* c, const int64_t* n, int count, double* w_out, bool* found) {
  const double t0 = now_s();
  BUMBAR_TRY(ensure_sorted(c));
  const double R = c->phi_hi - c->phi_lo;
  std::vector<WidthSearch> ss(count);
  for (int i = 0; i < count; ++i) {
    WidthSearch& q = ss[i];
    q.n = n[i];
    if (n[i] <= 1 || R == 0.0) {
      q.phase = 2;
      q.w_lo = R > 0.0 ? 2.0 * R : 1.0;
      continue;
    }
    q.w_hi = 2.0 * R;
    q.w_lo = R / static_cast<double>(n[i]);
  }
  for (;;) {
    // halving searches first: one width each (or done when out of range)
    std::vector<int> halving, bisecting;
    for (int i = 0; i < count; ++i) {
      WidthSearch& q = ss[i];
      if (q.phase == 0 && R / q.w_lo > kMaxIndex) {
        q.phase = 2;
        q.found = false;
      }
      if (q.phase == 0) halving.push_back(i);
      if (q.phase == 1) bisecting.push_back(i);
    }
    if (halving.empty() && bisecting.empty()) break;
    double ws[kWidthsPerPass];
    int nw = 0;
    std::vector<int> first(count, 0), depth(count, 0);
    for (int i : halving) {
      if (nw == kWidthsPerPass) break;
      first[i] = nw;
      depth[i] = 1;
      ws[nw++] = ss[i].w_lo;
    }
    // bisection trees: the deepest d with 2^d - 1 widths within the share
    const int left = kWidthsPerPass - nw;
    const int nb = static_cast<int>(bisecting.size());
    std::vector<std::array<double, 16>> mids(count);
    for (int j = 0; j < nb && nw < kWidthsPerPass; ++j) {
      const int i = bisecting[j];
      const int share = left / nb + (j < left % nb ? 1 : 0);
      int d = 0;
      while (d < 4 && (1 << (d + 1)) - 1 <= share) ++d;
      if (d == 0) continue;  // no room this pass
      double a[16], b[16];
      auto& mid = mids[i];
      a[1] = ss[i].w_lo;
      b[1] = ss[i].w_hi;
      const int nodes = (1 << d) - 1;
      for (int node = 1; node <= nodes; ++node) {
        mid[node] = std::sqrt(a[node] * b[node]);
        if (2 * node <= nodes) {
          a[2 * node] = a[node];
          b[2 * node] = mid[node];
          a[2 * node + 1] = mid[node];
          b[2 * node + 1] = b[node];
        }
      }
      first[i] = nw;
      depth[i] = d;
      for (int node = 1; node <= nodes; ++node) ws[nw++] = mid[node];
    }
    int64_t g[kWidthsPerPass];
    BUMBAR_TRY(count_at(c, ws, nw, g));
    for (int i : halving) {
      if (depth[i] == 0) continue;
      WidthSearch& q = ss[i];
      if (g[first[i]] >= q.n) {
        q.phase = 1;
      } else {
        q.w_hi = q.w_lo;
        q.w_lo = q.w_lo * 0.5;
      }
    }
    for (int i : bisecting) {
      if (depth[i] == 0) continue;
      WidthSearch& q = ss[i];
      const auto& mid = mids[i];
      int node = 1;
      for (int lev = 0; lev < depth[i] && q.steps < 64; ++lev) {
        const double m = mid[node];
        if (!(q.w_lo < m && m < q.w_hi)) {
          q.phase = 2;
          break;
        }
        ++q.steps;
        if (g[first[i] + node - 1] >= q.n) {
          q.w_lo = m;
          node = 2 * node + 1;
        } else {
          q.w_hi = m;
          node = 2 * node;
        }
      }
      if (q.steps >= 64) q.phase = 2;
    }
  }
  for (int i = 0; i < count; ++i) {
    w_out[i] = ss[i].w_lo;
    found[i] = ss[i].found;
  }
  c->t_width += now_s() - t0;
  return MBAR_OK;
}

// Width (or unbinned) of level `idx` of Algorithm 1's schedule without
// building it: n0 * inc^idx bins by the width rule, or width h0 / inc^idx.
mbar_status plan_level(mbar_ctx* c, int idx, bool* binned, double* w, int64_t* n_sched) {
  const mbar_opts& o = c->opts;
  *binned = false;
  BUMBAR_TRY(ensure_sorted(c));
  const double R = c->phi_hi - c->phi_lo;
  if (o.h0 > 0.0) {
    const double ww = o.h0 / std::pow(static_cast<double>(o.inc), idx);
    if (R / ww > kMaxIndex) return MBAR_OK;
    *binned = true;
    *w = ww;
    *n_sched = -1;  // the histogram's size
    return MBAR_OK;
  }
  const double nt = static_cast<double>(o.n0) * std::pow(static_cast<double>(o.inc), idx);
  if (nt > static_cast<double>(c->N) * 4.0) return MBAR_OK;  // far past the data: unbinned
  const int64_t n_target = static_cast<int64_t>(nt);
  bool found = false;
  BUMBAR_TRY(width_search(c, n_target, w, &found));
  if (!found) return MBAR_OK;
  *binned = true;
  *n_sched = n_target;
  return MBAR_OK;
}

// The FP32/FP64 stores of L binned levels (segments seg[l], run starts
// start[l], nb[l] bins): bin means of the unbinned store in one read, or for
// a factorised context the bin means of the sorted coordinate and the
// stores generated from them (a_k + b_k phibar_b).
mbar_status fill_level_stores(mbar_ctx* c, int L, const int32_t* const* seg, const int32_t* const* start,
                              const int64_t* nb, void* const* out, const int64_t* ld) {
  const int64_t N = c->N, K = c->K;
  if (L <= 0) return MBAR_OK;
  if (!c->fact) {
    void* mt = nullptr;
    const size_t mbytes = bin_means_multi_tmp_bytes(K, N, L, nb);
    BUMBAR_TRY(dalloc(c, &mt, mbytes));
    const mbar_status s = bin_means_multi(c->v, c->dtype, K, N, c->ld, L, seg, start, nb, out, ld, mt, mbytes, c->st);
    dfree(c, mt);
    return s;
  }
  std::vector<double*> phibar(L, nullptr);
  std::vector<void*> pout(L);
  std::vector<int64_t> pld(L);
  mbar_status s = MBAR_OK;
  size_t gen_bytes = 0;
  for (int l = 0; l < L && s == MBAR_OK; ++l) {
    s = dalloc_t(c, &phibar[l], std::max<int64_t>(nb[l], 1));
    pout[l] = phibar[l];
    pld[l] = nb[l];
    gen_bytes = std::max(gen_bytes, fact_level_tmp_bytes(K, nb[l]));
  }
  void* mt = nullptr;
  const size_t mbytes = std::max(bin_means_multi_tmp_bytes(1, N, L, nb), gen_bytes);
  if (s == MBAR_OK) s = dalloc(c, &mt, mbytes);
  // the coordinate is the one-row "store" whose bin means are phibar
  if (s == MBAR_OK)
    s = bin_means_multi(c->phi_sorted, 8, 1, N, N, L, seg, start, nb, pout.data(), pld.data(), mt,
                        bin_means_multi_tmp_bytes(1, N, L, nb), c->st);
  for (int l = 0; l < L && s == MBAR_OK; ++l)
    s = fact_level_store(c->fa, c->fb, phibar[l], K, nb[l], static_cast<float*>(out[l]), ld[l], mt, c->st);
  dfree(c, mt);
  for (double* q : phibar) dfree(c, q);
  return s;
}

// Every level Algorithm 1 can visit, built up front: the histograms one by
// one (each needs only the sorted coordinate), then all bin means in one read
// of the data. Level 0 and 1 always; level 2 when level 1 is binned; level
// j + 1 (j >= 2) when level j is binned and 2 inc n_j <= N -- the levels the
// second loop would build as it goes. An unbinned entry ends the list.
mbar_status prebuild_levels(mbar_ctx* c, std::vector<Level>* levels) {
  const mbar_opts& o = c->opts;
  const int64_t N = c->N, K = c->K;
  std::vector<int32_t*> segs, starts;
  void* tmp = nullptr;
  int64_t* keys_full = nullptr;
  int32_t* H_full = nullptr;
  const size_t htmp = hist_tmp_bytes(N);
  auto cleanup = [&]() {
    for (auto* q : segs) dfree(c, q);
    for (auto* q : starts) dfree(c, q);
    dfree(c, tmp);
    dfree(c, keys_full);
    dfree(c, H_full);
  };
  auto fail = [&](mbar_status s) {
    cleanup();
    for (auto& L : *levels) level_free(c, &L);
    levels->clear();
    return s;
  };
  mbar_status s = dalloc(c, &tmp, htmp);
  if (s == MBAR_OK) s = dalloc_t(c, &keys_full, N);
  if (s == MBAR_OK) s = dalloc_t(c, &H_full, N);
  if (s != MBAR_OK) return fail(s);
  // bin-count schedule: the targets are known, so all width searches run
  // together; the list stops where the second loop would stop building
  std::vector<double> wpre;
  std::vector<bool> fpre;
  std::vector<int64_t> npre;
  if (o.h0 <= 0.0) {
    s = ensure_sorted(c);
    if (s != MBAR_OK) return fail(s);
    for (int idx = 0; idx < kMaxBinLevels; ++idx) {
      const double nt = static_cast<double>(o.n0) * std::pow(static_cast<double>(o.inc), idx);
      if (nt > static_cast<double>(N) * 4.0) break;
      npre.push_back(static_cast<int64_t>(nt));
      if (!(idx < 2 || 2.0 * o.inc * nt <= static_cast<double>(N))) break;
    }
    wpre.resize(npre.size());
    std::unique_ptr<bool[]> fb(new bool[npre.size() + 1]);
    if (!npre.empty()) {
      s = width_search_multi(c, npre.data(), static_cast<int>(npre.size()), wpre.data(), fb.get());
      if (s != MBAR_OK) return fail(s);
    }
    for (size_t i = 0; i < npre.size(); ++i) fpre.push_back(fb[i]);
  }
  for (int idx = 0; idx < kMaxBinLevels; ++idx) {
    bool binned = false;
    double w = 0.0;
    int64_t n_sched = 0;
    if (o.h0 > 0.0) {
      s = plan_level(c, idx, &binned, &w, &n_sched);
      if (s != MBAR_OK) return fail(s);
    } else if (idx < static_cast<int>(npre.size())) {
      binned = fpre[idx];
      w = wpre[idx];
      n_sched = npre[idx];
    }
    if (!binned) {
      levels->push_back(c->full);
      break;
    }
    const double t0 = now_s();
    int32_t *seg = nullptr, *start = nullptr;
    s = dalloc_t(c, &seg, N);
    if (s == MBAR_OK) {
      segs.push_back(seg);
      s = dalloc_t(c, &start, N + 1);
    }
    if (s == MBAR_OK) {
      starts.push_back(start);
      s = build_histogram(c->d_pairs, c->d_sorted, N, w, seg, start, H_full, keys_full, c->nb_dev, tmp, htmp, c->st);
    }
    int32_t nb = 0;
    if (s == MBAR_OK) {
      cudaError_t e = cudaMemcpyAsync(&nb, c->nb_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, c->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
      if (e != cudaSuccess) s = cuda_status(e, "histogram size");
    }
    Level L;
    if (s == MBAR_OK) {
      L.binned = true;
      L.n = nb;
      L.ld = round_up(nb, 32);
      L.w = w;
      L.n_sched = n_sched >= 0 ? n_sched : nb;
      s = dalloc(c, &L.v, static_cast<size_t>(K) * L.ld * c->dtype);
    }
    if (s == MBAR_OK) s = dalloc_t(c, &L.H, nb);
    if (s == MBAR_OK) s = dalloc_t(c, &L.keys, nb);
    if (s == MBAR_OK) {
      cudaError_t e = cudaMemcpyAsync(L.H, H_full, nb * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(L.keys, keys_full, nb * sizeof(int64_t), cudaMemcpyDeviceToDevice, c->st);
      if (e != cudaSuccess) s = cuda_status(e, "histogram copy");
    }
    if (s == MBAR_OK) s = level_tmap(c, &L);
    c->t_levels += now_s() - t0;
    if (s != MBAR_OK) {
      level_free(c, &L);
      return fail(s);
    }
    levels->push_back(L);
    const bool more = idx < 2 || 2.0 * o.inc * static_cast<double>(L.n_sched) <= static_cast<double>(N);
    if (!more) break;
  }
  // all bin means in one read of the data (up to kMaxBinLevels per call)
  const double t0 = now_s();
  std::vector<const int32_t*> sg, stt;
  std::vector<int64_t> nbs, lds;
  std::vector<void*> outs;
  for (size_t i = 0; i < segs.size(); ++i) {
    sg.push_back(segs[i]);
    stt.push_back(starts[i]);
    nbs.push_back((*levels)[i].n);
    outs.push_back((*levels)[i].v);
    lds.push_back((*levels)[i].ld);
  }
  const int L = static_cast<int>(sg.size());
  if (L > 0) {
    s = fill_level_stores(c, L, sg.data(), stt.data(), nbs.data(), outs.data(), lds.data());
    if (s != MBAR_OK) return fail(s);
  }
  c->t_levels += now_s() - t0;
  cleanup();
  return MBAR_OK;
}

mbar_status algorithm1(mbar_ctx* c, mbar_report* rep) {
  const mbar_opts& o = c->opts;
  std::vector<Level> levels;
  BUMBAR_TRY(prebuild_levels(c, &levels));
  // level idx of the schedule; ownership passes to the caller
  auto take = [&](int idx) -> Level {
    if (idx < static_cast<int>(levels.size())) {
      Level L = levels[idx];
      levels[idx] = c->full;
      return L;
    }
    return c->full;
  };
  auto free_rest = [&]() {
    for (auto& L : levels) level_free(c, &L);
  };
  Level L0 = take(0);
  rep->n_rebins += L0.binned ? 1 : 0;
  mbar_status s = first_loop(c, L0, rep);
  level_free(c, &L0);
  if (s != MBAR_OK) {
    free_rest();
    return s;
  }
  int idx = 1;
  Level cur = take(idx), nxt;
  rep->n_rebins += cur.binned ? 1 : 0;
  if (!cur.binned) {
    free_rest();
    return MBAR_OK;
  }
  nxt = take(idx + 1);
  rep->n_rebins += nxt.binned ? 1 : 0;
  const int64_t N = c->N;
  const int64_t K = c->K;
  // MIXED: the pair's FP32 data re-centred per column at the current f, so
  // the step-to-step rounding of the exponents is that of numbers near 0
  // (Eq. 3 and the noise floor compare steps at that rounding level). A
  // column's largest exponent lies between min_k a_k and max_k a_k (v >= 0),
  // so this only matters when some |a_k| is large: below 64 kT the FP32
  // spacing there is under 1e-5 kT per entry and the data stay as they are.
  float* cur_vT = nullptr;  // owned: the current level sample-major (small levels, large ones in exclusive mode)
  void* grid_scr = nullptr;  // owned: scratch of the grid-wide loop, when it runs the level
  bool cur_loop = false;     // the current level's in-place steps run in one launch
  // Levels up to 4 MB take the one-launch loop (a cluster of 8 SMs streaming
  // the level from L2). Without CUDA graphs (server workers, with other
  // solves on the GPU beside them) a round on a larger level is 2 x 21
  // separate full-grid launches of a few microseconds each from a host
  // thread; there the cluster loop runs up to 32 MB: 8 SMs per solve leave
  // the rest of the GPU to the other solves.
  const double kFusedRoundBytes = (c->graphs ? 4.0 : 32.0) * (1 << 20);
  const double kSmajLevelMaxBytes = 4.0 * (1 << 30);
  auto recenter_pair = [&]() -> mbar_status {
    if (c->dtype != 4) return MBAR_OK;
    BUMBAR_TRY(d2h(c, c->f_h.data(), c->f, K));
    BUMBAR_CUDA(cudaStreamSynchronize(c->st));
    double amax = 0.0;
    for (int64_t k = 0; k < K; ++k) amax = std::max(amax, std::fabs(c->f_h[k] + std::log(c->Nk_h[k])));
    if (amax > 64.0)
      for (Level* L : {&cur, &nxt})
        if (L->binned)
          BUMBAR_TRY(recenter_columns(static_cast<float*>(L->v), K, L->n, L->ld, c->f, c->logN_d, c->st));
    // a small current level: its in-place steps run in one launch on its
    // sample-major copy (sci_loop.cu): over the whole GPU with the level in
    // shared memory when this solve has the device to itself (graphs), else
    // on one cluster
    dfree(c, cur_vT);
    cur_vT = nullptr;
    cur.vT = nullptr;
    dfree(c, grid_scr);
    grid_scr = nullptr;
    const bool grid = cur.binned && use_grid_loop(c, cur.n);
    cur_loop = cur.binned && (grid || sci_loop_supported(K, cur.n, kFusedRoundBytes));
    // a larger current level, in exclusive mode: a sample-major copy for its
    // N_intermediate + 1 passes (one transpose; the copy is not in a
    // server's memory budget, hence exclusive mode only)
    const double lbytes = static_cast<double>(sci_loop_level_bytes(K, cur.n));
    const bool smaj_copy = !cur_loop && cur.binned && c->graphs && c->dtype == 4 && lse_smaj_preferred(K) &&
                           lbytes <= kSmajLevelMaxBytes;
    if (cur_loop || smaj_copy) {
      BUMBAR_TRY(dalloc(c, reinterpret_cast<void**>(&cur_vT), sci_loop_level_bytes(K, cur.n)));
      BUMBAR_TRY(level_to_samples(static_cast<const float*>(cur.v), K, cur.n, cur.ld, cur_vT, c->st));
      if (grid) BUMBAR_TRY(dalloc(c, &grid_scr, sci_grid_scratch_bytes(K)));
      if (smaj_copy) cur.vT = cur_vT;
    }
    return MBAR_OK;
  };
  s = recenter_pair();
  if (s != MBAR_OK) {
    dfree(c, cur_vT);
    dfree(c, grid_scr);
    level_free(c, &cur);
    level_free(c, &nxt);
    free_rest();
    return s;
  }
  // one round: N_intermediate in-place steps on cur, the probe at n (-> ft)
  // and the probe at n * inc (-> fts); the f buffers keep their addresses so
  // the captured round stays valid until the level pair changes
  auto round_body = [&]() -> mbar_status {
    if (cur_loop) {
      SciLoopParams q{};
      q.K = static_cast<int>(K);
      q.n = static_cast<int>(cur.n);
      q.H = cur.H;
      q.f = c->f;
      q.logN = c->logN_d;
      q.Nk = c->Nk_d;
      q.ctrl = c->ctrl;
      q.err = err_word(c);
      q.max_steps = o.n_intermediate;  // eps = noise = 0: exactly these steps
      if (grid_scr)
        BUMBAR_TRY(sci_grid_launch(cur_vT, q, grid_scr, c->st));
      else
        BUMBAR_TRY(sci_loop_launch(cur_vT, q, c->st));
    } else {
      for (int i = 0; i < o.n_intermediate; ++i)
        BUMBAR_TRY(run_lse(c, cur, c->f, kLseModeSci, c->f, nullptr, nullptr, 0.0, 0, nullptr));
    }
    BUMBAR_TRY(run_lse(c, cur, c->f, kLseModeSci, c->ft, nullptr, c->s, 0.0, 0, nullptr, c->d));
    BUMBAR_TRY(run_lse(c, nxt, c->f, kLseModeSci, c->fts, nullptr, c->s2, 0.0, 0, nullptr));
    return MBAR_OK;
  };
  // the steps of one round in order: n_intermediate in-place steps on cur,
  // then the probes at n (-> ft, s, d) and at n * inc (-> fts, s2)
  auto round_step = [&](int idx, bool exact_log) -> mbar_status {
    const Level& L = idx <= o.n_intermediate ? cur : nxt;
    double* out = idx < o.n_intermediate ? c->f : (idx == o.n_intermediate ? c->ft : c->fts);
    double* so = idx < o.n_intermediate ? nullptr : (idx == o.n_intermediate ? c->s : c->s2);
    double* dd = idx == o.n_intermediate ? c->d : nullptr;
    if (exact_log) {
      BUMBAR_TRY(log_sci_step(c, L, c->f, out, nullptr, so, 0.0, dd, 0.0));
      return read_status(c);
    }
    return sci_step_exact(c, L, c->f, out, nullptr, so, nullptr, dd);
  };
  Graph g;
  bool captured = false;
  constexpr int kStallRounds = 40;
  double d_mark = INFINITY;
  int stall = 0;
  for (int64_t round = 0; s == MBAR_OK; ++round) {
    if (rep->iters_second_loop >= o.max_sci) break;
    const int64_t iters_before = c->hstat->ctrl.iters;
    const bool use_graph = cur.binned && nxt.binned && c->graphs;
    if (use_graph && !captured) {
      s = capture(c, &g, round_body);
      if (s != MBAR_OK) break;
      captured = true;
    }
    // algorithmic bytes of a round: N_intermediate + 1 passes over the
    // current level and one over the next
    time_mark(c, true, 4,
              static_cast<double>(K) * c->dtype *
                  ((o.n_intermediate + 1.0) * static_cast<double>(cur.n) + static_cast<double>(nxt.n)));
    if (use_graph) {
      cudaError_t e = cudaGraphLaunch(g.exec, c->st);
      if (e != cudaSuccess) {
        s = cuda_status(e, "cudaGraphLaunch");
        break;
      }
      count_launches(o.n_intermediate + 2);
    } else {
      s = round_body();
    }
    time_mark(c, false, 4, 0.0);
    if (s == MBAR_OK) s = read_status(c);
    if (s == MBAR_OK && take_underflow(c)) {
      // the round stopped at step `first`: that step exactly, then the rest
      const int first = static_cast<int>(c->hstat->ctrl.iters - iters_before);
      for (int idx = first; idx < o.n_intermediate + 2 && s == MBAR_OK; ++idx) s = round_step(idx, idx == first);
    }
    if (s != MBAR_OK) break;
    const double s_n = c->hstat->s, s_next = c->hstat->s2, d_n = c->hstat->d;
    rep->iters_second_loop += o.n_intermediate + 2;
    trace_row(c, 2, static_cast<double>(cur.n_sched), s_n, s_next);
    // MIXED: SCI contracts geometrically, so a level whose step max|df|
    // has not halved in kStallRounds rounds is moving on the FP32 rounding of
    // its own evaluation (which can sit above the fixed noise floor)
    if (d_n <= 0.5 * d_mark) {
      d_mark = d_n;
      stall = 0;
    } else {
      ++stall;
    }
    const bool stalled = c->dtype == 4 && stall >= kStallRounds;
    // Eq. 3, plus: a step under the evaluation's rounding floor means the
    // level has converged as far as this arithmetic can tell
    if (2.0 * s_next > static_cast<double>(o.inc) * s_n || (o.noise_floor > 0.0 && d_n < o.noise_floor) || stalled) {
      d_mark = INFINITY;
      stall = 0;
      if (cudaMemcpyAsync(c->f, c->fts, K * sizeof(double), cudaMemcpyDeviceToDevice, c->st) != cudaSuccess) {
        s = MBAR_ECUDA;
        break;
      }
      g.reset();
      captured = false;
      level_free(c, &cur);
      cur = nxt;
      nxt = Level{};
      idx++;
      if (!cur.binned || 2.0 * o.inc * static_cast<double>(cur.n_sched) > static_cast<double>(N)) break;
      nxt = take(idx + 1);
      rep->n_rebins += nxt.binned ? 1 : 0;
      s = recenter_pair();
      if (s != MBAR_OK) break;
    } else {
      if (cudaMemcpyAsync(c->f, c->ft, K * sizeof(double), cudaMemcpyDeviceToDevice, c->st) != cudaSuccess) {
        s = MBAR_ECUDA;
        break;
      }
    }
  }
  g.reset();
  rep->final_bins = cur.binned ? cur.n : 0;
  dfree(c, cur_vT);
  dfree(c, grid_scr);
  level_free(c, &cur);
  level_free(c, &nxt);
  free_rest();
  return s;
}

// plain MBAR warm-up: unbinned SCI until max_k |g_k|/N_k < warm_tol
mbar_status plain_warmup(mbar_ctx* c, mbar_report* rep) {
  std::vector<double> gh(c->K);
  for (int64_t it = 0; it < c->opts.max_sci; ++it) {
    BUMBAR_TRY(sci_step_exact(c, c->full, c->f, c->fs, c->g, c->s, nullptr));
    BUMBAR_TRY(d2h(c, gh.data(), c->g, c->K));
    BUMBAR_CUDA(cudaStreamSynchronize(c->st));
    double r = 0.0;
    for (int64_t k = 0; k < c->K; ++k) r = std::max(r, std::fabs(gh[k]) / c->Nk_h[k]);
    if (r < c->opts.warm_tol) break;
    std::swap(c->f, c->fs);
    rep->iters_first_loop++;
  }
  return MBAR_OK;
}

mbar_status upload_f(mbar_ctx* c, const double* f_host, double* dst) {
  std::vector<double> g(f_host, f_host + c->K);
  BUMBAR_TRY(h2d(c, dst, g.data(), c->K));
  BUMBAR_CUDA(cudaStreamSynchronize(c->st));
  return MBAR_OK;
}

#define CHECK_CTX(c)                         \
  do {                                       \
    if (!(c)) {                              \
      set_error("null context");             \
      return MBAR_EINVAL;                    \
    }                                        \
  } while (0)

// Orders the context's internal stream after the caller's stream on entry
// and the caller's stream after the internal one on exit.
struct StreamFence {
  mbar_ctx* c;
  explicit StreamFence(mbar_ctx* ctx) : c(ctx) {
    cudaEventRecord(c->ev_in, c->ust);
    cudaStreamWaitEvent(c->st, c->ev_in, 0);
  }
  ~StreamFence() {
    cudaEventRecord(c->ev_out, c->st);
    cudaStreamWaitEvent(c->ust, c->ev_out, 0);
  }
};

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
namespace bumbar {
void ctx_set_graphs(mbar_ctx* c, bool on) {
  if (c) c->graphs = on;
}

void ctx_set_batcher(mbar_ctx* c, FirstLoopBatcher* b) {
  if (c) c->batcher = b;
}
}  // namespace bumbar

extern "C" {

const char* mbar_status_string(mbar_status s) {
  switch (s) {
    case MBAR_OK: return "ok";
    case MBAR_EINVAL: return "invalid argument";
    case MBAR_ENOMEM: return "out of memory";
    case MBAR_ECUDA: return "CUDA error";
    case MBAR_ENOTCONV: return "not converged";
    case MBAR_ESTATE: return "invalid state";
    case MBAR_ETIMEOUT: return "device wait timed out";
    case MBAR_EUNSUPPORTED: return "unsupported size";
  }
  return "unknown status";
}

const char* mbar_last_error(void) { return bumbar::last_error(); }

mbar_status mbar_opts_default(mbar_opts* o, int32_t precision) {
  if (!o) {
    set_error("opts is NULL");
    return MBAR_EINVAL;
  }
  if (precision != MBAR_FP64 && precision != MBAR_MIXED) {
    set_error("unknown precision %d", precision);
    return MBAR_EINVAL;
  }
  std::memset(o, 0, sizeof(*o));
  o->precision = precision;
  o->n0 = 100;
  o->eps = 1e-3;
  o->inc = 10;
  o->n_intermediate = 20;
  o->h0 = 0.0;
  o->use_binning = 1;
  o->f_tol = precision == MBAR_FP64 ? 1e-10 : 1e-5;
  o->warm_tol = 1e-3;
  o->max_newton = 50;
  o->max_sci = 200000;
  o->noise_floor = precision == MBAR_FP64 ? 1e-11 : 2e-6;
  return MBAR_OK;
}

}  // extern "C"

namespace {

// Context creation from u_kn (dense) or, with fa != nullptr, from the
// factorised form u_kn = fa_k + fb_k fphi_n without any K x N store (MIXED,
// K <= 1024: the caller checks).
mbar_status create_impl(mbar_ctx** out, int64_t K, int64_t N, const int64_t* N_k, const double* u_kn,
                        int32_t u_on_device, const double* fa_in, const double* fb_in, const double* fphi_in,
                        const mbar_opts* opts, void* cuda_stream) {
  const bool fact = fa_in != nullptr;
  if (!out || !N_k || (!fact && !u_kn)) {
    set_error("mbar_create: null pointer argument");
    return MBAR_EINVAL;
  }
  *out = nullptr;
  if (K < 1 || N < 1) {
    set_error("mbar_create: need K >= 1 and N >= 1 (got K=%lld N=%lld)", (long long)K, (long long)N);
    return MBAR_EINVAL;
  }
  if (K > 1024) {
    set_error("mbar_create: K=%lld exceeds the supported maximum of 1024 states", (long long)K);
    return MBAR_EUNSUPPORTED;
  }
  if (N > 2000000000LL) {
    set_error("mbar_create: N=%lld exceeds the supported maximum of 2e9 samples", (long long)N);
    return MBAR_EUNSUPPORTED;
  }
  int64_t sum = 0;
  for (int64_t k = 0; k < K; ++k) {
    if (N_k[k] < 1) {
      set_error("mbar_create: N_k[%lld] = %lld must be positive", (long long)k, (long long)N_k[k]);
      return MBAR_EINVAL;
    }
    sum += N_k[k];
  }
  if (sum != N) {
    set_error("mbar_create: sum of N_k (%lld) != N (%lld)", (long long)sum, (long long)N);
    return MBAR_EINVAL;
  }
  mbar_opts o;
  if (opts) {
    o = *opts;
  } else {
    mbar_opts_default(&o, MBAR_MIXED);
  }
  if ((o.precision != MBAR_FP64 && o.precision != MBAR_MIXED) || o.n0 < 1 || o.inc < 2 || !(o.eps > 0) ||
      o.n_intermediate < 0 || o.h0 < 0 || !(o.f_tol > 0) || o.max_newton < 1 || o.max_sci < 1 ||
      !(o.noise_floor >= 0)) {
    set_error("mbar_create: invalid options");
    return MBAR_EINVAL;
  }
  auto* c = new (std::nothrow) mbar_ctx();
  if (!c) {
    set_error("mbar_create: host allocation failed");
    return MBAR_ENOMEM;
  }
  {
    // keep freed stream-ordered allocations cached in the device's default
    // pool (level buffers are allocated and released on every rebin)
    int dev = 0;
    cudaMemPool_t pool;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
  }
  c->K = K;
  c->N = N;
  c->opts = o;
  c->dtype = o.precision == MBAR_MIXED ? 4 : 8;
  c->ust = static_cast<cudaStream_t>(cuda_stream);
  if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    mbar_status st = cuda_status(cudaGetLastError(), "stream/event creation");
    mbar_destroy(c);
    return st;
  }
  // u_kn may have been produced on the caller's stream
  cudaEventRecord(c->ev_in, c->ust);
  cudaStreamWaitEvent(c->st, c->ev_in, 0);
  c->ld = round_up(N, 32);
  c->Nk_h.resize(K);
  c->f_h.assign(K, 0.0);
  std::vector<double> logN(K);
  for (int64_t k = 0; k < K; ++k) {
    c->Nk_h[k] = static_cast<double>(N_k[k]);
    logN[k] = std::log(c->Nk_h[k]);
  }
  auto fail = [&](mbar_status s) {
    mbar_destroy(c);
    return s;
  };
  mbar_status s = MBAR_OK;
#define TRYC(x)               \
  do {                        \
    s = (x);                  \
    if (s != MBAR_OK) return fail(s); \
  } while (0)
  TRYC(dalloc_t(c, &c->Nk_d, K));
  TRYC(dalloc_t(c, &c->logN_d, K));
  TRYC(h2d(c, c->Nk_d, c->Nk_h.data(), K));
  TRYC(h2d(c, c->logN_d, logN.data(), K));
  for (double** p : {&c->f, &c->fs, &c->ft, &c->fts, &c->g, &c->gt, &c->Q, &c->delta}) TRYC(dalloc_t(c, p, K));
  {
    void* st = nullptr;
    TRYC(dalloc(c, &st, sizeof(DevStatus)));
    c->stat = static_cast<DevStatus*>(st);
    if (cudaMemsetAsync(c->stat, 0, sizeof(DevStatus), c->st) != cudaSuccess) return fail(MBAR_ECUDA);
    if (cudaMallocHost(reinterpret_cast<void**>(&c->hstat), sizeof(DevStatus)) != cudaSuccess)
      return fail(cuda_status(cudaGetLastError(), "cudaMallocHost"));
    c->s = &c->stat->s;
    c->s2 = &c->stat->s2;
    c->d = &c->stat->d;
    c->ctrl = &c->stat->ctrl;
  }
  TRYC(dalloc_t(c, &c->hess, K * K));
  TRYC(dalloc_t(c, &c->info, 1));
  TRYC(dalloc_t(c, &c->bad, 1));
  TRYC(dalloc_t(c, &c->count, kWidthsPerPass));
  TRYC(dalloc_t(c, &c->nb_dev, 1));

  if (cudaMemsetAsync(c->bad, 0, sizeof(int), c->st) != cudaSuccess) return fail(MBAR_ECUDA);
  if (cudaMemsetAsync(c->f, 0, K * sizeof(double), c->st) != cudaSuccess) return fail(MBAR_ECUDA);
  if (fact) {
    c->fact = true;
    TRYC(dalloc_t(c, &c->fa, K));
    TRYC(dalloc_t(c, &c->fb, K));
    TRYC(dalloc_t(c, &c->fphi, N));
    const cudaMemcpyKind kind = u_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (cudaMemcpyAsync(c->fa, fa_in, K * sizeof(double), kind, c->st) != cudaSuccess ||
        cudaMemcpyAsync(c->fb, fb_in, K * sizeof(double), kind, c->st) != cudaSuccess ||
        cudaMemcpyAsync(c->fphi, fphi_in, N * sizeof(double), kind, c->st) != cudaSuccess)
      return fail(cuda_status(cudaGetLastError(), "mbar_create_factorised: upload"));
    TRYC(check_finite(c->fa, K, c->bad, c->st));
    TRYC(check_finite(c->fb, K, c->bad, c->st));
    TRYC(check_finite(c->fphi, N, c->bad, c->st));
    TRYC(dalloc_t(c, &c->logden64, N));
    TRYC(dalloc(c, &c->fref, lse_fact_ref_bytes()));
    TRYC(dalloc(c, &c->logden, static_cast<size_t>(N) * c->dtype));  // binned levels
    TRYC(dalloc_t(c, &c->perm, N));
    TRYC(dalloc_t(c, &c->seg, N));
    TRYC(dalloc_t(c, &c->start, N + 1));
    TRYC(dalloc_t(c, &c->phi_sorted, N));
    TRYC(dalloc_t(c, &c->d_sorted, N));
    TRYC(dalloc_t(c, &c->d_pairs, N));
    // the coordinate is phi: sorted once here (the samples themselves are
    // never reordered, so perm stays the identity)
    {
      std::vector<int32_t> id(N);
      std::iota(id.begin(), id.end(), 0);
      if (cudaMemcpyAsync(c->perm, id.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice, c->st) != cudaSuccess)
        return fail(cuda_status(cudaGetLastError(), "mbar_create_factorised: identity"));
      const size_t stmp = sort_tmp_bytes(N);
      void* tmp = nullptr;
      int32_t* order = nullptr;
      s = dalloc(c, &tmp, stmp);
      if (s == MBAR_OK) s = dalloc_t(c, &order, N);
      if (s == MBAR_OK) s = sort_coordinate(c->fphi, N, c->phi_sorted, order, tmp, stmp, c->st);
      if (s == MBAR_OK) s = offsets_from_min(c->phi_sorted, N, c->d_sorted, c->d_pairs, c->st);
      if (s == MBAR_OK && (cudaMemcpyAsync(&c->phi_lo, c->phi_sorted, sizeof(double), cudaMemcpyDeviceToHost,
                                           c->st) != cudaSuccess ||
                           cudaMemcpyAsync(&c->phi_hi, c->phi_sorted + N - 1, sizeof(double), cudaMemcpyDeviceToHost,
                                           c->st) != cudaSuccess))
        s = cuda_status(cudaGetLastError(), "coordinate range");
      int bad = 0;
      if (s == MBAR_OK && cudaMemcpyAsync(&bad, c->bad, sizeof(int), cudaMemcpyDeviceToHost, c->st) != cudaSuccess)
        s = MBAR_ECUDA;
      if (s == MBAR_OK && cudaStreamSynchronize(c->st) != cudaSuccess) s = cuda_status(cudaGetLastError(), "create");
      dfree(c, tmp);
      dfree(c, order);
      if (s == MBAR_OK && bad) {
        set_error("mbar_create_factorised: a, b or phi has non-finite entries");
        s = MBAR_EINVAL;
      }
      if (s != MBAR_OK) return fail(s);
      c->sorted = true;
    }
    {
      // one CTA per SM bounds every plan's grid, tuned shapes included
      const int grid = std::max({lse_plan(K, N, c->dtype).grid, lse_fact_plan(K, N).grid, num_sms()});
      c->scratch_bytes = lse_scratch_for_grid(K, grid);
      TRYC(dalloc(c, &c->scratch, c->scratch_bytes));
      if (cudaMemsetAsync(c->scratch, 0, c->scratch_bytes, c->st) != cudaSuccess) return fail(MBAR_ECUDA);
    }
    c->full.binned = false;
    c->full.fact = true;
    c->full.n = N;
    c->full.ld = N;
    c->full.v = nullptr;
    c->full.n_sched = N;
    c->cur = c->full;
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return fail(cuda_status(cudaGetLastError(), "mbar_create"));
    *out = c;
    return MBAR_OK;
  }
  TRYC(dalloc(c, &c->vst, static_cast<size_t>(stage_pitch(K)) * N * c->dtype + 16));
  c->smaj = c->dtype == 4 && lse_smaj_preferred(K);
  if (c->smaj) TRYC(dalloc_t(c, &c->logden_orig, N));
  TRYC(dalloc(c, &c->logden, static_cast<size_t>(N) * c->dtype));
  TRYC(dalloc_t(c, &c->perm, N));
  TRYC(dalloc_t(c, &c->seg, N));
  TRYC(dalloc_t(c, &c->start, N + 1));
  TRYC(dalloc_t(c, &c->phi0, N));
  TRYC(dalloc_t(c, &c->phi_sorted, N));
  TRYC(dalloc_t(c, &c->d_sorted, N));
  TRYC(dalloc_t(c, &c->d_pairs, N));
  // the samples of u_kn on the device in FP64
  const double* u_dev = u_kn;
  double* u_tmp = nullptr;
  if (!u_on_device) {
    TRYC(dalloc_t(c, &u_tmp, K * N));
    if (cudaMemcpyAsync(u_tmp, u_kn, K * N * sizeof(double), cudaMemcpyHostToDevice, c->st) != cudaSuccess) {
      dfree(c, u_tmp);
      return fail(cuda_status(cudaGetLastError(), "u_kn upload"));
    }
    u_dev = u_tmp;
  }
  if (c->dtype == 4) s = dalloc_t(c, &c->cshift, N);
  if (s == MBAR_OK) s = stage_samples(u_dev, K, N, N, c->cshift, c->vst, c->dtype, c->bad, &c->stat->err, c->st);
  if (s == MBAR_OK && cudaMemcpyAsync(c->phi0, u_dev, N * sizeof(double), cudaMemcpyDeviceToDevice, c->st) != cudaSuccess)
    s = MBAR_ECUDA;
  {
    // identity permutation
    std::vector<int32_t> id(N);
    std::iota(id.begin(), id.end(), 0);
    if (s == MBAR_OK && cudaMemcpyAsync(c->perm, id.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice, c->st) != cudaSuccess)
      s = MBAR_ECUDA;
    int bad = 0;
    if (s == MBAR_OK && cudaMemcpyAsync(&bad, c->bad, sizeof(int), cudaMemcpyDeviceToHost, c->st) != cudaSuccess)
      s = MBAR_ECUDA;
    if (s == MBAR_OK && cudaStreamSynchronize(c->st) != cudaSuccess) s = MBAR_ECUDA;
    if (s == MBAR_OK && bad) {
      set_error("mbar_create: u_kn has non-finite entries");
      s = MBAR_EINVAL;
    }
    if (s == MBAR_OK) s = read_status(c);  // a bounded wait of the staging that gave up
  }
  dfree(c, u_tmp);
  if (s == MBAR_ECUDA) set_error("mbar_create: %s", cudaGetErrorString(cudaGetLastError()));
  if (s != MBAR_OK) return fail(s);
  // LSE scratch sized for the widest grid of this K
  {
    const LsePlan pl = lse_plan(K, N, c->dtype);
    int grid = pl.grid;
    // one CTA per SM bounds the sample-major plans' grids, tuned shapes included
    if (c->smaj) grid = std::max({grid, lse_smaj_plan(K, N).grid, num_sms()});
    c->scratch_bytes = lse_scratch_for_grid(K, grid);
    TRYC(dalloc(c, &c->scratch, c->scratch_bytes));
    if (cudaMemsetAsync(c->scratch, 0, c->scratch_bytes, c->st) != cudaSuccess) return fail(MBAR_ECUDA);
  }
  c->full.binned = false;
  c->full.n = N;
  c->full.ld = c->ld;
  c->full.v = nullptr;  // formed from the staging by the first call that needs it
  c->full.n_sched = N;
  c->cur = c->full;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return fail(cuda_status(cudaGetLastError(), "mbar_create"));
#undef TRYC
  *out = c;
  return MBAR_OK;
}

}  // namespace

extern "C" {

mbar_status mbar_create(mbar_ctx** out, int64_t K, int64_t N, const int64_t* N_k, const double* u_kn,
                        int32_t u_on_device, const mbar_opts* opts, void* cuda_stream) {
  cudaGetLastError();  // drop stale errors of earlier, unrelated runtime calls
  if (!u_kn) {
    set_error("mbar_create: null pointer argument");
    if (out) *out = nullptr;
    return MBAR_EINVAL;
  }
  return create_impl(out, K, N, N_k, u_kn, u_on_device, nullptr, nullptr, nullptr, opts, cuda_stream);
}

mbar_status mbar_create_factorised(mbar_ctx** out, int64_t K, int64_t N, const int64_t* N_k, const double* a,
                                   const double* b, const double* phi, int32_t on_device, const mbar_opts* opts,
                                   void* cuda_stream) {
  cudaGetLastError();  // drop stale errors of earlier, unrelated runtime calls
  if (!out || !N_k || !a || !b || !phi) {
    set_error("mbar_create_factorised: null pointer argument");
    return MBAR_EINVAL;
  }
  *out = nullptr;
  if (K < 1 || N < 1 || K > 1024 || N > 2000000000LL) {
    set_error("mbar_create_factorised: bad sizes K=%lld N=%lld", (long long)K, (long long)N);
    return K > 1024 || N > 2000000000LL ? MBAR_EUNSUPPORTED : MBAR_EINVAL;
  }
  {
    // MIXED: the store-free factorised context
    mbar_opts o;
    if (opts) {
      o = *opts;
    } else {
      mbar_opts_default(&o, MBAR_MIXED);
    }
    if (o.precision == MBAR_MIXED && o.use_binning)
      return create_impl(out, K, N, N_k, nullptr, on_device, a, b, phi, &o, cuda_stream);
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  double* buf = nullptr;  // [a | b | phi] when given on the host, then u
  double* u = nullptr;
  const size_t in_bytes = static_cast<size_t>(2 * K + N) * sizeof(double);
  const size_t u_bytes = static_cast<size_t>(K) * static_cast<size_t>(N) * sizeof(double);
  auto release = [&]() {
    if (u) cudaFreeAsync(u, st);
    if (buf) cudaFreeAsync(buf, st);
    cudaStreamSynchronize(st);
  };
  const double *ad = a, *bd = b, *pd = phi;
  if (!on_device) {
    if (cudaMallocAsync(reinterpret_cast<void**>(&buf), in_bytes, st) != cudaSuccess) {
      cudaGetLastError();
      set_error("mbar_create_factorised: cannot allocate %zu bytes", in_bytes);
      return MBAR_ENOMEM;
    }
    if (cudaMemcpyAsync(buf, a, K * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(buf + K, b, K * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(buf + 2 * K, phi, N * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess) {
      mbar_status e = cuda_status(cudaGetLastError(), "mbar_create_factorised: upload");
      release();
      return e;
    }
    ad = buf;
    bd = buf + K;
    pd = buf + 2 * K;
  }
  if (cudaMallocAsync(reinterpret_cast<void**>(&u), u_bytes, st) != cudaSuccess) {
    cudaGetLastError();
    release();
    set_error("mbar_create_factorised: cannot allocate %zu bytes for u", u_bytes);
    return MBAR_ENOMEM;
  }
  mbar_status s = factorised_u(ad, bd, pd, K, N, u, st);
  // mbar_create validates u (non-finite a, b or phi give EINVAL there),
  // stages it on the context's stream after the work queued on `st`
  if (s == MBAR_OK) s = mbar_create(out, K, N, N_k, u, 1, opts, cuda_stream);
  if (s == MBAR_OK) {
    // the context's copy is complete before u is released
    if (cudaStreamSynchronize((*out)->st) != cudaSuccess) s = cuda_status(cudaGetLastError(), "create");
  }
  if (s == MBAR_OK) s = mbar_set_coordinate(*out, pd, 1);
  // the context's reads of phi are complete before the buffers are released
  if (s == MBAR_OK && cudaStreamSynchronize((*out)->st) != cudaSuccess) s = cuda_status(cudaGetLastError(), "create");
  release();
  if (s != MBAR_OK && *out) {
    mbar_destroy(*out);
    *out = nullptr;
  }
  return s;
}

mbar_status mbar_set_coordinate(mbar_ctx* c, const double* phi, int32_t phi_on_device) {
  cudaGetLastError();  // drop stale errors of earlier, unrelated runtime calls
  CHECK_CTX(c);
  if (c->fact) {
    set_error("mbar_set_coordinate: the bin coordinate of a factorised context is its phi");
    return MBAR_EUNSUPPORTED;
  }
  StreamFence fence(c);
  if (!phi) {
    set_error("mbar_set_coordinate: phi is NULL");
    return MBAR_EINVAL;
  }
  double* pd = nullptr;
  BUMBAR_TRY(dalloc_t(c, &pd, c->N));
  cudaError_t e = cudaMemcpyAsync(pd, phi, c->N * sizeof(double),
                                  phi_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->st);
  int bad = 0;
  mbar_status s = e == cudaSuccess ? MBAR_OK : cuda_status(e, "phi upload");
  if (s == MBAR_OK) s = cudaMemsetAsync(c->bad, 0, sizeof(int), c->st) == cudaSuccess ? MBAR_OK : MBAR_ECUDA;
  if (s == MBAR_OK) s = check_finite(pd, c->N, c->bad, c->st);
  if (s == MBAR_OK && cudaMemcpyAsync(&bad, c->bad, sizeof(int), cudaMemcpyDeviceToHost, c->st) != cudaSuccess)
    s = MBAR_ECUDA;
  if (s == MBAR_OK && cudaStreamSynchronize(c->st) != cudaSuccess) s = MBAR_ECUDA;
  if (s == MBAR_OK && bad) {
    set_error("mbar_set_coordinate: phi has non-finite entries");
    s = MBAR_EINVAL;
  }
  if (s == MBAR_OK) s = set_coordinate_dev(c, pd);
  dfree(c, pd);
  return s;
}

mbar_status mbar_bin(mbar_ctx* c, double h, int64_t* n_bins_out) {
  cudaGetLastError();  // drop stale errors of earlier, unrelated runtime calls
  CHECK_CTX(c);
  StreamFence fence(c);
  if (!(h >= 0.0) || !std::isfinite(h)) {
    set_error("mbar_bin: h must be finite and >= 0");
    return MBAR_EINVAL;
  }
  BUMBAR_TRY(ensure_sorted(c));
  if (h == 0.0) {
    level_free(c, &c->cur);
    c->cur = c->full;
  } else {
    if ((c->phi_hi - c->phi_lo) / h > kMaxIndex) {
      set_error("mbar_bin: width too small for exact bin indices (range/h > 2^52)");
      return MBAR_EINVAL;
    }
    Level L;
    BUMBAR_TRY(make_level_w(c, h, &L));
    level_free(c, &c->cur);
    c->cur = L;
  }
  if (n_bins_out) *n_bins_out = c->cur.n;
  return MBAR_OK;
}

mbar_status mbar_bin_count(mbar_ctx* c, int64_t n, double* w_out, int64_t* n_bins_out) {
  cudaGetLastError();  // drop stale errors of earlier, unrelated runtime calls
  CHECK_CTX(c);
  StreamFence fence(c);
  if (n < 1) {
    set_error("mbar_bin_count: n must be >= 1");
    return MBAR_EINVAL;
  }
  double w = 0.0;
  bool found = false;
  BUMBAR_TRY(width_search(c, n, &w, &found));
  if (!found) {
    level_free(c, &c->cur);
    c->cur = c->full;
    if (w_out) *w_out = 0.0;
  } else {
    Level L;
    BUMBAR_TRY(make_level_w(c, w, &L));
    level_free(c, &c->cur);
    c->cur = L;
    if (w_out) *w_out = w;
  }
  if (n_bins_out) *n_bins_out = c->cur.n;
  return MBAR_OK;
}

mbar_status mbar_get_bins(mbar_ctx* c, int64_t* keys, int64_t* H, double* u_kp) {
  CHECK_CTX(c);
  StreamFence fence(c);
  if (!c->cur.binned) {
    set_error("mbar_get_bins: the current level is unbinned");
    return MBAR_ESTATE;
  }
  const int64_t nb = c->cur.n;
  if (keys) BUMBAR_CUDA(cudaMemcpyAsync(keys, c->cur.keys, nb * sizeof(int64_t), cudaMemcpyDeviceToHost, c->st));
  std::vector<int32_t> h32;
  if (H) {
    h32.resize(nb);
    BUMBAR_CUDA(cudaMemcpyAsync(h32.data(), c->cur.H, nb * sizeof(int32_t), cudaMemcpyDeviceToHost, c->st));
  }
  std::vector<unsigned char> raw;
  if (u_kp) {
    raw.resize(static_cast<size_t>(c->K) * c->cur.ld * c->dtype);
    BUMBAR_CUDA(cudaMemcpyAsync(raw.data(), c->cur.v, raw.size(), cudaMemcpyDeviceToHost, c->st));
  }
  BUMBAR_CUDA(cudaStreamSynchronize(c->st));
  if (H)
    for (int64_t b = 0; b < nb; ++b) H[b] = h32[b];
  if (u_kp) {
    for (int64_t k = 0; k < c->K; ++k)
      for (int64_t b = 0; b < nb; ++b) {
        const size_t idx = static_cast<size_t>(k) * c->cur.ld + b;
        u_kp[k * nb + b] = c->dtype == 4 ? static_cast<double>(reinterpret_cast<float*>(raw.data())[idx])
                                         : reinterpret_cast<double*>(raw.data())[idx];
      }
  }
  return MBAR_OK;
}

mbar_status mbar_sci_step(mbar_ctx* c, const double* f_in, double* f_out, double* grad, double* s_out,
                          double* logden) {
  cudaGetLastError();  // drop stale errors of earlier, unrelated runtime calls
  CHECK_CTX(c);
  StreamFence fence(c);
  BUMBAR_TRY(ensure_store(c));
  if (!f_in) {
    set_error("mbar_sci_step: f_in is NULL");
    return MBAR_EINVAL;
  }
  const int64_t K = c->K;
  BUMBAR_TRY(upload_f(c, f_in, c->ft));
  BUMBAR_TRY(sci_step_exact(c, c->cur, c->ft, c->fts, c->gt, c->s2, logden ? c->logden : nullptr));
  if (f_out) BUMBAR_TRY(d2h(c, f_out, c->fts, K));
  if (grad) BUMBAR_TRY(d2h(c, grad, c->gt, K));
  if (s_out) BUMBAR_TRY(d2h(c, s_out, c->s2, 1));
  const int64_t n = c->cur.n;
  std::vector<unsigned char> raw;
  std::vector<int32_t> perm;
  std::vector<double> shift;
  const bool fact_ld = c->fact && !c->cur.binned;  // FP64, original sample order
  if (logden && fact_ld) {
    BUMBAR_CUDA(cudaMemcpyAsync(logden, c->logden64, n * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  } else if (logden) {
    raw.resize(static_cast<size_t>(n) * c->dtype);
    BUMBAR_CUDA(cudaMemcpyAsync(raw.data(), c->logden, raw.size(), cudaMemcpyDeviceToHost, c->st));
    if (!c->cur.binned) {
      perm.resize(n);
      BUMBAR_CUDA(cudaMemcpyAsync(perm.data(), c->perm, n * sizeof(int32_t), cudaMemcpyDeviceToHost, c->st));
      if (c->cshift) {
        shift.resize(n);
        BUMBAR_CUDA(cudaMemcpyAsync(shift.data(), c->cshift, n * sizeof(double), cudaMemcpyDeviceToHost, c->st));
      }
    }
  }
  BUMBAR_CUDA(cudaStreamSynchronize(c->st));
  if (logden && !fact_ld) {
    for (int64_t i = 0; i < n; ++i) {
      double v = c->dtype == 4 ? static_cast<double>(reinterpret_cast<float*>(raw.data())[i])
                               : reinterpret_cast<double*>(raw.data())[i];
      if (!c->cur.binned) {
        if (c->cshift) v -= shift[i];  // v_kn = u_kn - c_n  =>  logden(u) = logden(v) - c_n
        logden[perm[i]] = v;
      } else {
        logden[i] = v;
      }
    }
  }
  return MBAR_OK;
}

mbar_status mbar_hessian(mbar_ctx* c, const double* f_in, double* hess_out) {
  cudaGetLastError();  // drop stale errors of earlier, unrelated runtime calls
  CHECK_CTX(c);
  StreamFence fence(c);
  BUMBAR_TRY(ensure_store(c));
  if (!f_in || !hess_out) {
    set_error("mbar_hessian: null pointer argument");
    return MBAR_EINVAL;
  }
  const int64_t K = c->K;
  const Level& L = c->cur;
  BUMBAR_TRY(upload_f(c, f_in, c->ft));
  BUMBAR_TRY(run_lse(c, L, c->ft, kLseModePass, nullptr, nullptr, nullptr, 0.0, 0, c->logden));
  const size_t htmp = hessian_tmp_bytes(K, L.n);
  void* tmp = nullptr;
  BUMBAR_TRY(dalloc(c, &tmp, htmp));
  time_mark(c, true, 1, static_cast<double>(K) * L.n * c->dtype);
  mbar_status s = level_hessian(c, L, c->ft, tmp, htmp);
  time_mark(c, false, 1, 0);
  if (s == MBAR_OK) s = check_device_errors(c);
  if (s == MBAR_OK) s = d2h(c, hess_out, c->hess, K * K);
  if (s == MBAR_OK && cudaStreamSynchronize(c->st) != cudaSuccess) s = MBAR_ECUDA;
  dfree(c, tmp);
  return s;
}

// Asymptotic covariance of f at the context's current f (after mbar_solve),
// from the Hessian of the MBAR objective on the unbinned data.
mbar_status mbar_covariance(mbar_ctx* c, double* cov_out) {
  cudaGetLastError();  // drop stale errors of earlier, unrelated runtime calls
  CHECK_CTX(c);
  StreamFence fence(c);
  if (!cov_out) {
    set_error("mbar_covariance: cov_out is NULL");
    return MBAR_EINVAL;
  }
  BUMBAR_TRY(ensure_store(c));
  const int64_t K = c->K;
  const Level& L = c->full;
  BUMBAR_TRY(run_lse(c, L, c->f, kLseModePass, nullptr, nullptr, nullptr, 0.0, 0, c->logden));
  const size_t htmp = std::max(hessian_tmp_bytes(K, L.n), covariance_tmp_bytes(K));
  void* tmp = nullptr;
  double* cov = nullptr;
  BUMBAR_TRY(dalloc(c, &tmp, htmp));
  mbar_status s = dalloc_t(c, &cov, K * K);
  if (s == MBAR_OK)
    s = level_hessian(c, L, c->f, tmp, htmp);
  if (s == MBAR_OK) s = check_device_errors(c);
  int info = 0;
  if (s == MBAR_OK && cudaMemsetAsync(c->info, 0, sizeof(int), c->st) != cudaSuccess) s = MBAR_ECUDA;
  if (s == MBAR_OK) s = covariance(c->hess, K, c->Nk_d, cov, c->info, tmp, htmp, c->st);
  if (s == MBAR_OK) s = d2h(c, cov_out, cov, K * K);
  if (s == MBAR_OK && cudaMemcpyAsync(&info, c->info, sizeof(int), cudaMemcpyDeviceToHost, c->st) != cudaSuccess)
    s = MBAR_ECUDA;
  if (s == MBAR_OK && cudaStreamSynchronize(c->st) != cudaSuccess) s = MBAR_ECUDA;
  if (s == MBAR_OK && info) {
    set_error("mbar_covariance: the reduced Hessian is not positive definite (states without overlap)");
    s = MBAR_ENOTCONV;
  }
  dfree(c, cov);
  dfree(c, tmp);
  return s;
}

mbar_status mbar_newton_step(mbar_ctx* c, const double* f_in, double* f_out, double* step_max_abs) {
  cudaGetLastError();  // drop stale errors of earlier, unrelated runtime calls
  CHECK_CTX(c);
  StreamFence fence(c);
  BUMBAR_TRY(ensure_store(c));
  if (!f_in) {
    set_error("mbar_newton_step: f_in is NULL");
    return MBAR_EINVAL;
  }
  const int64_t K = c->K;
  const Level& L = c->cur;
  BUMBAR_TRY(upload_f(c, f_in, c->ft));
  BUMBAR_TRY(sci_step_exact(c, L, c->ft, c->fts, c->gt, c->s2, c->logden));
  const size_t htmp = hessian_tmp_bytes(K, L.n), ntmp = newton_tmp_bytes(K);
  void* tmp = nullptr;
  BUMBAR_TRY(dalloc(c, &tmp, std::max(htmp, ntmp)));
  mbar_status s = level_hessian(c, L, c->ft, tmp, htmp);
  if (s == MBAR_OK) s = cudaMemsetAsync(c->info, 0, sizeof(int), c->st) == cudaSuccess ? MBAR_OK : MBAR_ECUDA;
  if (s == MBAR_OK) s = newton_solve(c->hess, K, c->gt, c->delta, c->info, tmp, ntmp, c->st);
  if (s == MBAR_OK) s = vec_add_gauge(c->ft, c->delta, c->fts, K, c->st);
  std::vector<double> d(K);
  int info = 0;
  if (s == MBAR_OK) s = check_device_errors(c);
  if (s == MBAR_OK) s = d2h(c, d.data(), c->delta, K);
  if (s == MBAR_OK && f_out) s = d2h(c, f_out, c->fts, K);
  if (s == MBAR_OK && cudaMemcpyAsync(&info, c->info, sizeof(int), cudaMemcpyDeviceToHost, c->st) != cudaSuccess)
    s = MBAR_ECUDA;
  if (s == MBAR_OK && cudaStreamSynchronize(c->st) != cudaSuccess) s = MBAR_ECUDA;
  dfree(c, tmp);
  BUMBAR_TRY(s);
  if (step_max_abs) *step_max_abs = max_abs(d);
  if (info) {
    set_error("mbar_newton_step: reduced Hessian not positive definite");
    return MBAR_ENOTCONV;
  }
  return MBAR_OK;
}

mbar_status mbar_solve(mbar_ctx* c, const double* f_init, mbar_report* report) {
  cudaGetLastError();  // drop stale errors of earlier, unrelated runtime calls
  CHECK_CTX(c);
  StreamFence fence(c);
  // Algorithm 1 bins: store the data directly in the coordinate's order
  if (c->opts.use_binning && c->K > 1) BUMBAR_TRY(ensure_sorted(c));
  BUMBAR_TRY(ensure_store(c));
  mbar_report rep{};
  const int64_t K = c->K;
  if (f_init) {
    std::vector<double> f0(f_init, f_init + K);
    for (int64_t k = K - 1; k >= 0; --k) f0[k] -= f0[0];
    BUMBAR_TRY(h2d(c, c->f, f0.data(), K));
  } else {
    BUMBAR_CUDA(cudaMemsetAsync(c->f, 0, K * sizeof(double), c->st));
  }
  c->trace.clear();
  c->t_width = c->t_levels = 0.0;
  mbar_status s = MBAR_OK;
  if (K > 1) {
    const double t0 = now_s();
    if (c->opts.use_binning)
      s = algorithm1(c, &rep);
    else
      s = plain_warmup(c, &rep);
    const double t1 = now_s();
    if (s == MBAR_OK) s = newton_phase(c, &rep);
    rep.seconds_newton = now_s() - t1;
    rep.seconds_width = c->t_width;
    rep.seconds_levels = c->t_levels;
    rep.seconds_sci = (t1 - t0) - c->t_width - c->t_levels;
  }
  mbar_status s2 = d2h(c, c->f_h.data(), c->f, K);
  if (s2 == MBAR_OK && cudaStreamSynchronize(c->st) != cudaSuccess) s2 = MBAR_ECUDA;
  if (report) *report = rep;
  if (s != MBAR_OK) return s;
  return s2;
}

// Eqs. 5-6 at the context's current f on the unbinned data.
mbar_status mbar_reweight(mbar_ctx* c, const double* u0, int32_t u0_on_device, double* p_out, double* log_C) {
  CHECK_CTX(c);
  if (!u0) {
    set_error("mbar_reweight: u0 is NULL");
    return MBAR_EINVAL;
  }
  cudaGetLastError();
  StreamFence fence(c);
  BUMBAR_TRY(ensure_store(c));
  const int64_t N = c->N;
  double* u0_dev = nullptr;
  void* tmp = nullptr;
  double* logc_dev = nullptr;
  mbar_status s = MBAR_OK;
  if (!c->weights) s = dalloc_t(c, &c->weights, N);
  if (s == MBAR_OK) s = dalloc(c, &tmp, reweight_tmp_bytes(N));
  if (s == MBAR_OK) s = dalloc_t(c, &logc_dev, 1);
  const double* u0d = u0;
  if (s == MBAR_OK && !u0_on_device) {
    s = dalloc_t(c, &u0_dev, N);
    if (s == MBAR_OK && cudaMemcpyAsync(u0_dev, u0, N * sizeof(double), cudaMemcpyHostToDevice, c->st) != cudaSuccess)
      s = cuda_status(cudaGetLastError(), "mbar_reweight: copy of u0");
    u0d = u0_dev;
  }
  int bad = 0;
  if (s == MBAR_OK) s = cudaMemsetAsync(c->bad, 0, sizeof(int), c->st) == cudaSuccess ? MBAR_OK : MBAR_ECUDA;
  if (s == MBAR_OK) s = check_finite(u0d, N, c->bad, c->st);
  if (s == MBAR_OK && (cudaMemcpyAsync(&bad, c->bad, sizeof(int), cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
                       cudaStreamSynchronize(c->st) != cudaSuccess))
    s = MBAR_ECUDA;
  if (s == MBAR_OK && bad) {
    set_error("mbar_reweight: u0 has non-finite entries");
    s = MBAR_EINVAL;
  }
  if (s == MBAR_OK) s = run_lse(c, c->full, c->f, kLseModePass, nullptr, nullptr, nullptr, 0.0, 0, c->logden);
  if (s == MBAR_OK)
    s = c->fact ? reweight_weights(u0d, c->perm, c->logden64, 8, nullptr, N, c->weights, logc_dev, tmp,
                                   reweight_tmp_bytes(N), c->st)
                : reweight_weights(u0d, c->perm, c->logden, c->dtype, c->cshift, N, c->weights, logc_dev, tmp,
                                   reweight_tmp_bytes(N), c->st);
  double logc = 0.0;
  if (s == MBAR_OK && p_out &&
      cudaMemcpyAsync(p_out, c->weights, N * sizeof(double), cudaMemcpyDeviceToHost, c->st) != cudaSuccess)
    s = cuda_status(cudaGetLastError(), "mbar_reweight: copy of p");
  if (s == MBAR_OK && cudaMemcpyAsync(&logc, logc_dev, sizeof(double), cudaMemcpyDeviceToHost, c->st) != cudaSuccess)
    s = cuda_status(cudaGetLastError(), "mbar_reweight: copy of log C");
  if (s == MBAR_OK) s = read_status(c);  // syncs
  if (s == MBAR_OK && log_C) *log_C = logc;
  dfree(c, u0_dev);
  dfree(c, tmp);
  dfree(c, logc_dev);
  return s;
}

mbar_status mbar_weighted_histogram2d(mbar_ctx* c, const double* x, const double* y, int32_t on_device, double x0,
                                      double dx, int64_t nx, double y0, double dy, int64_t ny, double* out) {
  CHECK_CTX(c);
  if (!x || !y || !out || !(dx > 0.0) || !(dy > 0.0) || nx < 1 || ny < 1 || nx * ny > (int64_t(1) << 31)) {
    set_error("mbar_weighted_histogram2d: bad arguments");
    return MBAR_EINVAL;
  }
  if (!c->weights) {
    set_error("mbar_weighted_histogram2d: call mbar_reweight first");
    return MBAR_ESTATE;
  }
  cudaGetLastError();
  StreamFence fence(c);
  const int64_t N = c->N;
  double *xd = nullptr, *yd = nullptr, *hd = nullptr;
  mbar_status s = dalloc_t(c, &hd, nx * ny);
  const double* xs = x;
  const double* ys = y;
  if (s == MBAR_OK && !on_device) {
    s = dalloc_t(c, &xd, N);
    if (s == MBAR_OK) s = dalloc_t(c, &yd, N);
    if (s == MBAR_OK && (cudaMemcpyAsync(xd, x, N * 8, cudaMemcpyHostToDevice, c->st) != cudaSuccess ||
                         cudaMemcpyAsync(yd, y, N * 8, cudaMemcpyHostToDevice, c->st) != cudaSuccess))
      s = cuda_status(cudaGetLastError(), "mbar_weighted_histogram2d: copy of x, y");
    xs = xd;
    ys = yd;
  }
  if (s == MBAR_OK) s = weighted_hist2d(xs, ys, c->weights, N, x0, dx, nx, y0, dy, ny, hd, c->st);
  if (s == MBAR_OK &&
      cudaMemcpyAsync(out, hd, static_cast<size_t>(nx) * ny * 8, cudaMemcpyDeviceToHost, c->st) != cudaSuccess)
    s = cuda_status(cudaGetLastError(), "mbar_weighted_histogram2d: copy of the histogram");
  if (s == MBAR_OK && cudaStreamSynchronize(c->st) != cudaSuccess) s = cuda_status(cudaGetLastError(), "sync");
  dfree(c, xd);
  dfree(c, yd);
  dfree(c, hd);
  return s;
}

mbar_status mbar_free_energies(mbar_ctx* c, double* f_out) {
  CHECK_CTX(c);
  if (!f_out) {
    set_error("mbar_free_energies: f_out is NULL");
    return MBAR_EINVAL;
  }
  std::copy(c->f_h.begin(), c->f_h.end(), f_out);
  return MBAR_OK;
}

mbar_status mbar_device_bytes(mbar_ctx* c, int64_t* bytes) {
  CHECK_CTX(c);
  if (bytes) *bytes = c->bytes;
  return MBAR_OK;
}

mbar_status mbar_set_exclusive(mbar_ctx* c, int32_t exclusive) {
  CHECK_CTX(c);
  c->graphs = exclusive != 0;
  return MBAR_OK;
}

mbar_status mbar_set_timing(mbar_ctx* c, int32_t enable) {
  CHECK_CTX(c);
  BUMBAR_CUDA(cudaStreamSynchronize(c->st));
  for (auto& r : c->recs) {
    c->pool.push_back(r.a);
    c->pool.push_back(r.b);
  }
  c->recs.clear();
  c->timing = enable != 0;
  return MBAR_OK;
}

mbar_status mbar_get_timing(mbar_ctx* c, int32_t kind, int64_t* launches, double* total_ms, double* bytes) {
  CHECK_CTX(c);
  BUMBAR_CUDA(cudaStreamSynchronize(c->st));
  int64_t n = 0;
  double ms = 0.0, by = 0.0;
  for (auto& r : c->recs) {
    if (r.kind != kind) continue;
    float t = 0.f;
    BUMBAR_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
    ++n;
    ms += t;
    by += r.bytes;
  }
  if (launches) *launches = n;
  if (total_ms) *total_ms = ms;
  if (bytes) *bytes = by;
  return MBAR_OK;
}

mbar_status mbar_get_trace(mbar_ctx* c, int64_t* rows, double* out, int64_t capacity) {
  CHECK_CTX(c);
  const int64_t n = static_cast<int64_t>(c->trace.size() / 4);
  if (rows) *rows = n;
  if (out) std::copy(c->trace.begin(), c->trace.begin() + 4 * std::min(n, std::max<int64_t>(capacity, 0)), out);
  return MBAR_OK;
}

mbar_status mbar_set_hessian_path(int32_t path) {
  if (path < 0 || path > 3) {
    set_error("mbar_set_hessian_path: path must be 0, 1, 2 or 3");
    return MBAR_EINVAL;
  }
  set_hessian_path(path);
  return MBAR_OK;
}

mbar_status mbar_kernel_launches(int64_t* count) {
  if (!count) {
    set_error("mbar_kernel_launches: count is NULL");
    return MBAR_EINVAL;
  }
  *count = launches_so_far();
  return MBAR_OK;
}

mbar_status mbar_destroy(mbar_ctx* c) {
  if (!c) return MBAR_OK;
  for (auto& r : c->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : c->pool) cudaEventDestroy(e);
  level_free(c, &c->cur);
  void* ptrs[] = {c->weights, c->Nk_d, c->logN_d, c->v, c->vst, c->logden_orig, c->cshift, c->perm,  c->phi0,    c->phi_sorted, c->d_sorted, c->d_pairs, c->f,
                  c->fs,   c->ft,     c->fts,   c->g,      c->gt,    c->Q,       c->stat,
                  c->hess, c->delta,  c->info,  c->bad,    c->logden,  c->scratch,    c->seg,
                  c->start, c->count, c->nb_dev, c->fa, c->fb, c->fphi, c->logden64, c->fref};
  if (c->st) {
    for (void* p : ptrs) dfree(c, p);
    cudaStreamSynchronize(c->st);
    cudaStreamDestroy(c->st);
  }
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->hstat) cudaFreeHost(c->hstat);
  delete c;
  return MBAR_OK;
}

size_t mbar_lse_scratch_bytes(int64_t K, int64_t n, int32_t dtype_bytes) {
  if (K < 1 || K > 1024 || n < 1 || (dtype_bytes != 4 && dtype_bytes != 8)) return 0;
  return lse_scratch_bytes(K, n, dtype_bytes);
}

mbar_status mbar_lse_pass(const void* v, int32_t dtype_bytes, int64_t K, int64_t n, int64_t ld, const double* f,
                          const double* log_N, const int32_t* H, double* Q, void* logden, void* scratch,
                          size_t scratch_bytes, void* stream) {
  cudaGetLastError();  // drop stale errors of earlier, unrelated runtime calls
  if (!v || !f || !log_N || !Q || !scratch) {
    set_error("mbar_lse_pass: null pointer argument");
    return MBAR_EINVAL;
  }
  if (dtype_bytes != 4 && dtype_bytes != 8) {
    set_error("mbar_lse_pass: dtype_bytes must be 4 or 8");
    return MBAR_EINVAL;
  }
  if (K < 1 || n < 1 || ld < n || n > 2000000000LL) {
    set_error("mbar_lse_pass: bad sizes K=%lld n=%lld ld=%lld", (long long)K, (long long)n, (long long)ld);
    return MBAR_EINVAL;
  }
  if (K > 1024) {
    set_error("mbar_lse_pass: K=%lld exceeds 1024", (long long)K);
    return MBAR_EUNSUPPORTED;
  }
  if ((reinterpret_cast<uintptr_t>(scratch) & 15) != 0 || scratch_bytes < mbar_lse_scratch_bytes(K, n, dtype_bytes)) {
    set_error("mbar_lse_pass: scratch must be 16-byte aligned and at least mbar_lse_scratch_bytes()");
    return MBAR_EINVAL;
  }
  CUtensorMap map;
  const int C = 128 / dtype_bytes;
  const int box_rows = static_cast<int>(std::min<int64_t>(256, round_up(K, 8)));
  BUMBAR_TRY(make_tmap_2d(&map, v, dtype_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                          dtype_bytes, K, n, ld, C, box_rows));
  const LsePlan pl = lse_plan(K, n, dtype_bytes);
  LseParams p{};
  p.K = static_cast<int>(K);
  p.n = static_cast<int>(n);
  p.f = f;
  p.logN = log_N;
  p.H = H;
  unsigned char* sc = static_cast<unsigned char*>(scratch);
  p.counter = reinterpret_cast<unsigned*>(sc);
  p.err = reinterpret_cast<unsigned*>(sc + 4);
  p.partials = reinterpret_cast<double*>(sc + 256);
  p.Q = Q;
  p.logden = logden;
  p.mode = kLseModePass;
  return lse_launch(map, pl, p, dtype_bytes, static_cast<cudaStream_t>(stream));
}

size_t mbar_lse_samples_scratch_bytes(int64_t K, int64_t n) {
  if (K < 1 || K > 1024 || n < 1) return 0;
  // tuned shapes (mbar_autotune_enable) take at most one CTA per SM
  return lse_scratch_for_grid(K, std::max(lse_smaj_plan(K, n).grid, num_sms()));
}

mbar_status mbar_lse_pass_samples(const float* v_nk, int64_t K, int64_t n, const double* f, const double* log_N,
                                  const int32_t* H, double* Q, float* logden, void* scratch, size_t scratch_bytes,
                                  void* stream) {
  cudaGetLastError();  // drop stale errors of earlier, unrelated runtime calls
  if (!v_nk || !f || !log_N || !Q || !scratch) {
    set_error("mbar_lse_pass_samples: null pointer argument");
    return MBAR_EINVAL;
  }
  if (K < 1 || n < 1 || n > 2000000000LL) {
    set_error("mbar_lse_pass_samples: bad sizes K=%lld n=%lld", (long long)K, (long long)n);
    return MBAR_EINVAL;
  }
  if (K > 1024) {
    set_error("mbar_lse_pass_samples: K=%lld exceeds 1024", (long long)K);
    return MBAR_EUNSUPPORTED;
  }
  if ((reinterpret_cast<uintptr_t>(v_nk) & 15) != 0) {
    set_error("mbar_lse_pass_samples: v_nk must be 16-byte aligned");
    return MBAR_EINVAL;
  }
  if ((reinterpret_cast<uintptr_t>(scratch) & 15) != 0 || scratch_bytes < mbar_lse_samples_scratch_bytes(K, n)) {
    set_error("mbar_lse_pass_samples: scratch must be 16-byte aligned and at least mbar_lse_samples_scratch_bytes()");
    return MBAR_EINVAL;
  }
  LseParams p{};
  p.K = static_cast<int>(K);
  p.n = static_cast<int>(n);
  p.f = f;
  p.logN = log_N;
  p.H = H;
  unsigned char* sc = static_cast<unsigned char*>(scratch);
  p.counter = reinterpret_cast<unsigned*>(sc);
  p.err = reinterpret_cast<unsigned*>(sc + 4);
  p.partials = reinterpret_cast<double*>(sc + 256);
  p.Q = Q;
  p.logden = logden;
  p.mode = kLseModePass;
  p.exact_max = 1;
  return lse_smaj_launch(v_nk, lse_smaj_plan(K, n), p, static_cast<cudaStream_t>(stream));
}

size_t mbar_lse_factorised_scratch_bytes(int64_t K, int64_t n) {
  if (K < 1 || K > 1024 || n < 1) return 0;
  // the pass's own scratch, then (256-byte aligned) the reference-state table
  return round_up(static_cast<int64_t>(lse_scratch_for_grid(K, std::max(lse_fact_plan(K, n).grid, num_sms()))),
                  256) +
         lse_fact_ref_bytes();
}

mbar_status mbar_lse_pass_factorised(const double* a, const double* b, const double* phi, int64_t K, int64_t n,
                                     const double* f, const double* log_N, const int32_t* H, double* Q,
                                     double* logden, void* scratch, size_t scratch_bytes, void* stream) {
  cudaGetLastError();  // drop stale errors of earlier, unrelated runtime calls
  if (!a || !b || !phi || !f || !log_N || !Q || !scratch) {
    set_error("mbar_lse_pass_factorised: null pointer argument");
    return MBAR_EINVAL;
  }
  if (K < 1 || n < 1 || n > 2000000000LL) {
    set_error("mbar_lse_pass_factorised: bad sizes K=%lld n=%lld", (long long)K, (long long)n);
    return MBAR_EINVAL;
  }
  if (K > 1024) {
    set_error("mbar_lse_pass_factorised: K=%lld exceeds 1024", (long long)K);
    return MBAR_EUNSUPPORTED;
  }
  if ((reinterpret_cast<uintptr_t>(scratch) & 15) != 0 || scratch_bytes < mbar_lse_factorised_scratch_bytes(K, n)) {
    set_error("mbar_lse_pass_factorised: scratch must be 16-byte aligned and at least "
              "mbar_lse_factorised_scratch_bytes()");
    return MBAR_EINVAL;
  }
  LseParams p{};
  p.K = static_cast<int>(K);
  p.n = static_cast<int>(n);
  p.f = f;
  p.logN = log_N;
  p.H = H;
  unsigned char* sc = static_cast<unsigned char*>(scratch);
  p.counter = reinterpret_cast<unsigned*>(sc);
  p.err = reinterpret_cast<unsigned*>(sc + 4);
  p.partials = reinterpret_cast<double*>(sc + 256);
  p.Q = Q;
  p.logden = logden;
  p.mode = kLseModePass;
  p.exact_max = 1;
  const LsePlan pl = lse_fact_plan(K, n);
  void* ref = sc + round_up(static_cast<int64_t>(lse_scratch_for_grid(K, std::max(pl.grid, num_sms()))), 256);
  return lse_fact_launch(a, b, phi, pl, p, nullptr, nullptr, 0, ref, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
