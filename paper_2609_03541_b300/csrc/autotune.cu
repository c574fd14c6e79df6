// Autotuning of the launch shapes of the two streaming LSE passes that take
// several compiled shapes: the sample-major FP32 pass (lse_smaj.cu) and the
// factorised pass (lse_fact.cu).
//
// A key is (device name, pass family, K rounded up to a power of two >= 4,
// floor(log2 n)). The candidates for a key are every compiled lane shape
// (lanes per sample, chunks of 4 states per lane) that covers the key's K,
// with the fewest chunks that do, and for the sample-major pass stage sizes
// of 24 to 96 KB. Each candidate runs on resident synthetic data of the
// caller's size (capped at 1 GB): one warm-up, then three timed rounds of the
// Newton-driving pass (exact split of the largest weight) followed by the
// plain pass, CUDA events on the tuning stream; the median round decides.
// The winner goes into an in-memory table and, when a cache file is set, is
// appended to it as one text line, so a later process starts from it.
//
// Plans consult the table only while tuning is enabled: another shape sums
// the FP32 partials in another order, so results move at their rounding
// level. With tuning off the built-in shape rules are used, as without this
// file.
#include <sys/stat.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace bumbar {
namespace {

struct TuneKey {
  std::string dev;
  int family;
  int64_t kb;  // K rounded up to a power of two
  int nb;      // floor(log2 n)
  bool operator<(const TuneKey& o) const {
    return std::tie(dev, family, kb, nb) < std::tie(o.dev, o.family, o.kb, o.nb);
  }
};

struct TuneEntry {
  int lps = 0, nk = 0, nt = 0, stage = 0, candidates = 0;
  double ms = 0.0, heuristic_ms = 0.0;
};

std::mutex& tune_mutex() {
  static std::mutex m;
  return m;
}
std::map<TuneKey, TuneEntry>& tune_table() {
  static std::map<TuneKey, TuneEntry> t;
  return t;
}
bool g_enabled = false;
std::string g_path;

// the compiled lane shapes of both passes (their dispatch tables)
constexpr int kShapes[][2] = {{1, 1}, {1, 2}, {1, 4}, {2, 4}, {4, 4}, {8, 4}, {16, 4},
                              {32, 3}, {32, 4}, {32, 5}, {32, 6}, {32, 7}, {32, 8}};
constexpr int kStageChoices[] = {24 * 1024, 32 * 1024, 48 * 1024, 64 * 1024, 96 * 1024};

const std::string& device_name() {
  static std::string name;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    cudaDeviceProp p{};
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&p, dev) == cudaSuccess) {
      name = p.name;
    } else {
      cudaGetLastError();
      name = "unknown";
    }
    std::replace(name.begin(), name.end(), ' ', '_');
  });
  return name;
}

int64_t k_bucket(int64_t K) {
  int64_t b = 4;
  while (b < K) b <<= 1;
  return b;
}

int n_bucket(int64_t n) {
  int b = 0;
  while ((int64_t{2} << b) <= n) ++b;
  return b;
}

void append_line(const TuneKey& k, const TuneEntry& e) {
  if (g_path.empty()) return;
  FILE* fp = std::fopen(g_path.c_str(), "a");
  if (!fp) return;
  std::fprintf(fp, "%s %d %lld %d %d %d %d %d %d %.6f %.6f\n", k.dev.c_str(), k.family,
               static_cast<long long>(k.kb), k.nb, e.lps, e.nk, e.nt, e.stage, e.candidates, e.ms, e.heuristic_ms);
  std::fclose(fp);
}

void load_file_locked(const std::string& path) {
  FILE* fp = std::fopen(path.c_str(), "r");
  if (!fp) return;
  char dev[256];
  int family = 0, nb = 0;
  long long kb = 0;
  TuneEntry e;
  while (std::fscanf(fp, "%255s %d %lld %d %d %d %d %d %d %lf %lf", dev, &family, &kb, &nb, &e.lps, &e.nk, &e.nt,
                     &e.stage, &e.candidates, &e.ms, &e.heuristic_ms) == 11) {
    tune_table()[TuneKey{dev, family, kb, nb}] = e;  // later lines win
  }
  std::fclose(fp);
}

// synthetic inputs: uniform values from a counter hash (FP32 store values in
// [0, 16), phi in [-16, 0)); padding states of the sample-major store are 0
__global__ void tune_fill_samples(float* v, int64_t K, int64_t Kp, int64_t n) {
  const int64_t total = Kp * n;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t k = i % Kp;
    uint32_t h = static_cast<uint32_t>(i) * 2654435761u ^ static_cast<uint32_t>(i >> 32) * 40503u;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    v[i] = k < K ? static_cast<float>(h >> 8) * (16.0f / 16777216.0f) : 0.0f;
  }
}

__global__ void tune_fill_factorised(double* phi, int64_t n, double* a, double* b, int64_t K) {
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    uint32_t h = static_cast<uint32_t>(i) * 2654435761u;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    phi[i] = -16.0 * static_cast<double>(h >> 8) / 16777216.0;
  }
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < K) {
    a[t] = 0.0;
    b[t] = 1.0 + static_cast<double>(t) / static_cast<double>(K);
  }
}

struct TuneBuffers {
  void* data = nullptr;     // sample-major store, or phi
  double* small = nullptr;  // f, logN, Q, a, b [5][K]
  float* logden = nullptr;  // FP32 logden (sample-major) / FP64 (factorised)
  void* scratch = nullptr;
  void* ref = nullptr;
  ~TuneBuffers() {
    for (void* p : {data, static_cast<void*>(small), static_cast<void*>(logden), scratch, ref})
      if (p) cudaFree(p);
  }
};

// median over three rounds (pass with the exact split, then the plain pass)
mbar_status time_candidate(int family, const LsePlan& pl, const TuneBuffers& b, int64_t K, int64_t n,
                           cudaStream_t st, double* ms) {
  LseParams p{};
  p.K = static_cast<int>(K);
  p.n = static_cast<int>(n);
  p.f = b.small;
  p.logN = b.small + K;
  p.H = nullptr;
  unsigned char* sc = static_cast<unsigned char*>(b.scratch);
  p.counter = reinterpret_cast<unsigned*>(sc);
  p.err = reinterpret_cast<unsigned*>(sc + 4);
  p.partials = reinterpret_cast<double*>(sc + 256);
  p.Q = b.small + 2 * K;
  p.logden = b.logden;
  p.mode = kLseModePass;
  auto run = [&](int exact) -> mbar_status {
    p.exact_max = exact;
    if (family == kTuneSamples) return lse_smaj_launch(static_cast<const float*>(b.data), pl, p, st);
    return lse_fact_launch(b.small + 3 * K, b.small + 4 * K, static_cast<const double*>(b.data), pl, p, nullptr,
                           nullptr, 0, b.ref, st);
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  BUMBAR_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_status(cudaGetLastError(), "cudaEventCreate");
  }
  mbar_status s = run(1);
  if (s == MBAR_OK) s = run(0);
  std::vector<float> t;
  for (int r = 0; r < 3 && s == MBAR_OK; ++r) {
    cudaEventRecord(e0, st);
    s = run(1);
    if (s == MBAR_OK) s = run(0);
    cudaEventRecord(e1, st);
    if (s == MBAR_OK && cudaEventSynchronize(e1) == cudaSuccess) {
      float v = 0.f;
      cudaEventElapsedTime(&v, e0, e1);
      t.push_back(v);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != MBAR_OK) return s;
  if (t.size() != 3) return cuda_status(cudaGetLastError(), "autotune timing");
  std::sort(t.begin(), t.end());
  *ms = t[1];
  return MBAR_OK;
}

mbar_status search(int family, int64_t K, int64_t n, int64_t kb, TuneEntry* best) {
  const int64_t Kp = round_up(K, 4);
  const int64_t nt = std::min<int64_t>(n, std::max<int64_t>(1024, (int64_t{1} << 28) / Kp));  // <= 1 GB
  TuneBuffers b;
  const size_t data_bytes = family == kTuneSamples ? static_cast<size_t>(Kp) * nt * 4 : static_cast<size_t>(nt) * 8;
  // scratch for the largest grid any plan takes (one CTA per SM)
  const size_t scratch_bytes = lse_scratch_for_grid(K, num_sms());
  if (cudaMalloc(&b.data, data_bytes) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&b.small), 5 * K * sizeof(double)) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&b.logden), static_cast<size_t>(nt) * 8) != cudaSuccess ||
      cudaMalloc(&b.scratch, scratch_bytes) != cudaSuccess ||
      cudaMalloc(&b.ref, lse_fact_ref_bytes()) != cudaSuccess) {
    cudaGetLastError();
    set_error("autotune: cannot allocate the synthetic inputs (%zu bytes)", data_bytes);
    return MBAR_ENOMEM;
  }
  cudaStream_t st = nullptr;
  BUMBAR_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  mbar_status s = MBAR_OK;
  if (cudaMemsetAsync(b.small, 0, 5 * K * sizeof(double), st) != cudaSuccess ||
      cudaMemsetAsync(b.scratch, 0, scratch_bytes, st) != cudaSuccess)
    s = cuda_status(cudaGetLastError(), "autotune setup");
  if (s == MBAR_OK) {
    if (family == kTuneSamples)
      tune_fill_samples<<<4 * num_sms(), 256, 0, st>>>(static_cast<float*>(b.data), K, Kp, nt);
    else
      tune_fill_factorised<<<4 * num_sms(), 256, 0, st>>>(static_cast<double*>(b.data), nt, b.small + 3 * K,
                                                           b.small + 4 * K, K);
    count_launches(1);
    if (cudaGetLastError() != cudaSuccess) s = MBAR_ECUDA;
  }
  // the built-in rule's choice, for the record
  double heuristic = 0.0;
  if (s == MBAR_OK) {
    const LsePlan h = family == kTuneSamples ? lse_smaj_plan_rule(K, nt) : lse_fact_plan_rule(K, nt);
    s = time_candidate(family, h, b, K, nt, st, &heuristic);
  }
  TuneEntry win;
  win.ms = INFINITY;
  for (const auto& sh : kShapes) {
    if (s != MBAR_OK) break;
    const int lps = sh[0], nk = sh[1];
    if (4 * lps * nk < kb) continue;  // does not cover the bucket's K
    // the fewest chunks that cover it for this lane count
    bool fewer = false;
    for (const auto& o : kShapes)
      if (o[0] == lps && o[1] < nk && 4 * lps * o[1] >= kb) fewer = true;
    if (fewer) continue;
    const int nthreads = family == kTuneSamples ? (nk <= 4 ? 512 : 256) : fact_threads(nk);
    const int nstage = family == kTuneSamples ? static_cast<int>(sizeof(kStageChoices) / sizeof(int)) : 1;
    for (int si = 0; si < nstage && s == MBAR_OK; ++si) {
      const int stage = family == kTuneSamples ? kStageChoices[si] : 0;
      const LsePlan pl = family == kTuneSamples ? lse_smaj_plan_for(K, nt, lps, nk, nthreads, stage)
                                                : lse_fact_plan_for(K, nt, lps, nk);
      if (!pl.ok) continue;
      double ms = 0.0;
      s = time_candidate(family, pl, b, K, nt, st, &ms);
      ++win.candidates;
      if (s == MBAR_OK && ms < win.ms) {
        win.lps = lps;
        win.nk = nk;
        win.nt = nthreads;
        win.stage = stage;
        win.ms = ms;
      }
    }
  }
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
  if (s != MBAR_OK) return s;
  if (win.candidates == 0) {
    set_error("autotune: no compiled shape covers K=%lld", static_cast<long long>(K));
    return MBAR_EUNSUPPORTED;
  }
  win.heuristic_ms = heuristic;
  *best = win;
  return MBAR_OK;
}

}  // namespace

bool tuned_shape(int family, int64_t K, int64_t n, int* lps, int* nk, int* nt, int* stage_bytes) {
  std::lock_guard<std::mutex> lk(tune_mutex());
  if (!g_enabled) return false;
  auto it = tune_table().find(TuneKey{device_name(), family, k_bucket(K), n_bucket(n)});
  if (it == tune_table().end()) return false;
  // a bucket's shape covers its largest K; a smaller K in it is covered too
  *lps = it->second.lps;
  *nk = it->second.nk;
  *nt = it->second.nt;
  *stage_bytes = it->second.stage;
  return true;
}

}  // namespace bumbar

using namespace bumbar;

extern "C" {

mbar_status mbar_autotune_lse(int32_t family, int64_t K, int64_t n, mbar_tune_result* out) {
  cudaGetLastError();  // drop stale errors of earlier, unrelated runtime calls
  if (!out || (family != kTuneSamples && family != kTuneFactorised)) {
    set_error("mbar_autotune_lse: bad arguments (family %d)", family);
    return MBAR_EINVAL;
  }
  if (K < 1 || K > 1024 || n < 1 || n > 2000000000LL) {
    set_error("mbar_autotune_lse: bad sizes K=%lld n=%lld", static_cast<long long>(K), static_cast<long long>(n));
    return K > 1024 ? MBAR_EUNSUPPORTED : MBAR_EINVAL;
  }
  const TuneKey key{device_name(), family, k_bucket(K), n_bucket(n)};
  TuneEntry e;
  bool found = false;
  {
    std::lock_guard<std::mutex> lk(tune_mutex());
    auto it = tune_table().find(key);
    if (it != tune_table().end()) {
      e = it->second;
      found = true;
    }
  }
  if (!found) {
    // the search runs outside the lock (plans of other threads keep using the table)
    BUMBAR_TRY(search(family, std::max<int64_t>(K, 1), n, key.kb, &e));
    std::lock_guard<std::mutex> lk(tune_mutex());
    tune_table()[key] = e;
    append_line(key, e);
  }
  out->family = family;
  out->lanes_per_sample = e.lps;
  out->chunks_per_lane = e.nk;
  out->threads = e.nt;
  out->stage_bytes = e.stage;
  out->candidates = e.candidates;
  out->ms = e.ms;
  out->heuristic_ms = e.heuristic_ms;
  out->cached = found ? 1 : 0;
  out->pad = 0;
  return MBAR_OK;
}

mbar_status mbar_autotune_enable(int32_t on) {
  std::lock_guard<std::mutex> lk(tune_mutex());
  g_enabled = on != 0;
  return MBAR_OK;
}

mbar_status mbar_autotune_cache(const char* path) {
  std::lock_guard<std::mutex> lk(tune_mutex());
  g_path = path ? path : "";
  if (!g_path.empty()) load_file_locked(g_path);
  return MBAR_OK;
}

mbar_status mbar_autotune_clear(void) {
  std::lock_guard<std::mutex> lk(tune_mutex());
  tune_table().clear();
  return MBAR_OK;
}

}  // extern "C"
