// Serving and batching on top of mbar_ctx: a pool of worker threads, each
// with its own CUDA stream, runs admitted solves to completion; requests are
// admitted while their device footprint fits the server's budget, so solves
// of different sizes overlap on the GPU and later, smaller requests may pass
// a large one that is waiting for memory (continuous batching). Each request
// is an independent context: its kernels, launch shapes and reduction orders
// depend only on its own K, N and options, so its result is the same whether
// it runs alone or next to others.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace bumbar {
namespace {

using Clock = std::chrono::steady_clock;

double seconds_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double>(b - a).count();
}

struct Request {
  int64_t id = 0;
  int64_t K = 0, N = 0;
  std::vector<int64_t> Nk;
  const double* u = nullptr;
  int32_t u_on_device = 0;
  const double* phi = nullptr;
  int32_t phi_on_device = 0;
  // factorised form u_kn = fa_k + fb_k phi_n (phi above; same residence)
  bool factorised = false;
  const double* fa = nullptr;
  const double* fb = nullptr;
  uint64_t bytes = 0;
  int state = 0;  // 0 queued, 1 running, 2 done
  int passed_over = 0;
  mbar_status status = MBAR_OK;
  std::string error;
  std::vector<double> f;
  mbar_report report{};
  Clock::time_point t_submit, t_admit, t_done;
};

// Peak device memory of one solve: creation holds an FP64 staging copy of
// host u beside the stored data; the solve holds the stored data, the binned
// levels of Algorithm 1 (< 0.6 of the data), one reordering buffer,
// per-sample vectors, the Hessian and its partials.
uint64_t footprint(int64_t K, int64_t N, int32_t precision, int32_t use_binning, int32_t u_on_device) {
  if (K < 1 || N < 1) return 0;
  const uint64_t e = static_cast<uint64_t>(K) * static_cast<uint64_t>(round_up(N, 32));
  const uint64_t el = precision == MBAR_FP64 ? 8 : 4;
  // creation: the FP64 upload (host input) and the sample-major copy; the
  // coordinate: that copy and the row-major store; the solve: the store,
  // the sample-major copy where MIXED's LSE passes stream it, and the levels
  const uint64_t es = static_cast<uint64_t>(stage_pitch(K)) * static_cast<uint64_t>(N) + 4;
  const uint64_t create = (u_on_device ? 0 : e * 8) + es * el;
  const uint64_t coord = es * el + e * el;
  const bool keeps_copy = precision != MBAR_FP64 && lse_smaj_preferred(K);
  const uint64_t solve = e * el + (keeps_copy ? es * 4 : 0) + (use_binning ? e * el * 6 / 10 : 0);
  const uint64_t fixed = static_cast<uint64_t>(N) * 96 + static_cast<uint64_t>(K) * K * 8 * 4 + (64ull << 20);
  return std::max(std::max(create, coord), solve) + fixed;
}

// Peak device memory of a solve from the factorised form. MIXED with
// binning keeps no K x N store: Algorithm 1's binned levels (as above), the
// FP64 a, b, phi and per-sample vectors (sort keys, permutations, bin
// segments, FP64 and FP32 logden), and the Hessian's scratch. Other options
// materialise u as a K x N FP64 buffer on the device first.
uint64_t footprint_factorised(int64_t K, int64_t N, int32_t precision, int32_t use_binning) {
  if (K < 1 || N < 1) return 0;
  if (precision == MBAR_MIXED && use_binning) {
    const uint64_t e = static_cast<uint64_t>(K) * static_cast<uint64_t>(round_up(N, 32));
    const uint64_t fixed = static_cast<uint64_t>(N) * 192 + static_cast<uint64_t>(K) * K * 8 * 4 +
                           hessian_tmp_bytes(K, N) + (64ull << 20);
    return e * 4 * 6 / 10 + fixed;
  }
  return static_cast<uint64_t>(K) * static_cast<uint64_t>(N) * 8 + footprint(K, N, precision, use_binning, 1);
}

}  // namespace
}  // namespace bumbar

using namespace bumbar;

struct mbar_server {
  mbar_server_config cfg{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work;   // workers: an admitted request is ready, or shutdown
  std::condition_variable cv_done;   // waiters: a request finished
  std::deque<std::shared_ptr<Request>> queue;     // submitted, not admitted (arrival order)
  std::deque<std::shared_ptr<Request>> admitted;  // admitted, not yet picked by a worker
  std::unordered_map<int64_t, std::shared_ptr<Request>> all;
  int64_t next_id = 1;
  uint64_t bytes_in_use = 0;
  int running = 0;  // admitted and not finished
  bool stop = false;
  std::vector<std::thread> workers;
  FirstLoopBatcher* batcher = nullptr;  // MBAR_BATCH_PERSISTENT: the workers' first loops, batched
  // statistics
  uint64_t peak_bytes = 0;
  int peak_running = 0;
  int64_t completed = 0;

  // Admits queued requests in arrival order while a worker slot and memory
  // are free. A request that does not fit is passed over, but once it has
  // been passed over 4 x workers times nothing behind it is admitted until it
  // fits (no starvation of large requests). Called with `mu` held.
  void admit_locked() {
    for (auto it = queue.begin(); it != queue.end() && running < cfg.workers;) {
      Request& r = **it;
      if (bytes_in_use + r.bytes <= cfg.hbm_budget_bytes) {
        r.state = 1;
        r.t_admit = Clock::now();
        bytes_in_use += r.bytes;
        ++running;
        peak_bytes = std::max(peak_bytes, bytes_in_use);
        peak_running = std::max(peak_running, running);
        admitted.push_back(*it);
        it = queue.erase(it);
        cv_work.notify_one();
      } else {
        if (++r.passed_over > 4 * cfg.workers) break;
        ++it;
      }
    }
  }

  void run_one(Request& r, cudaStream_t st) {
    mbar_ctx* ctx = nullptr;
    mbar_status s = r.factorised ? mbar_create_factorised(&ctx, r.K, r.N, r.Nk.data(), r.fa, r.fb, r.phi,
                                                          r.phi_on_device, &cfg.opts, st)
                                 : mbar_create(&ctx, r.K, r.N, r.Nk.data(), r.u, r.u_on_device, &cfg.opts, st);
    // no stream capture on worker threads: the caller's other threads may
    // synchronise the whole device at any time
    if (s == MBAR_OK) ctx_set_graphs(ctx, false);
    if (s == MBAR_OK && batcher) ctx_set_batcher(ctx, batcher);
    if (s == MBAR_OK && r.phi && !r.factorised) s = mbar_set_coordinate(ctx, r.phi, r.phi_on_device);
    if (s == MBAR_OK || s == MBAR_ENOTCONV) {
      if (s == MBAR_OK) s = mbar_solve(ctx, nullptr, &r.report);
      r.f.assign(static_cast<size_t>(r.K), 0.0);
      const mbar_status s2 = mbar_free_energies(ctx, r.f.data());
      if (s == MBAR_OK) s = s2;
    }
    if (s != MBAR_OK) r.error = mbar_last_error();
    const mbar_status s3 = mbar_destroy(ctx);
    if (s == MBAR_OK) s = s3;
    r.status = s;
  }

  void worker_main() {
    cudaSetDevice(device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (;;) {
      std::shared_ptr<Request> r;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] { return stop || !admitted.empty(); });
        if (admitted.empty()) break;  // stop requested and nothing left to run
        r = admitted.front();
        admitted.pop_front();
      }
      run_one(*r, st);
      {
        std::lock_guard<std::mutex> lk(mu);
        r->state = 2;
        r->t_done = Clock::now();
        bytes_in_use -= r->bytes;
        --running;
        ++completed;
        admit_locked();
      }
      cv_done.notify_all();
    }
    if (st) cudaStreamDestroy(st);
  }
};

namespace {

// Charges, records and queues a prepared request (its footprint in
// r->bytes); `who` names the entry point in error messages.
mbar_status enqueue(mbar_server* s, const std::shared_ptr<Request>& r, int64_t* id, const char* who) {
  if (r->bytes > s->cfg.hbm_budget_bytes) {
    set_error("%s: the request needs about %llu bytes of device memory, more than the server's budget of %llu", who,
              static_cast<unsigned long long>(r->bytes), static_cast<unsigned long long>(s->cfg.hbm_budget_bytes));
    return MBAR_EUNSUPPORTED;
  }
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      set_error("%s: the server is shutting down", who);
      return MBAR_ESTATE;
    }
    r->id = s->next_id++;
    s->all[r->id] = r;
    s->queue.push_back(r);
    s->admit_locked();
  }
  *id = r->id;
  return MBAR_OK;
}

}  // namespace

extern "C" {

uint64_t mbar_footprint_factorised_bytes(int64_t K, int64_t N, int32_t precision, int32_t use_binning) {
  return footprint_factorised(K, N, precision, use_binning);
}

uint64_t mbar_footprint_bytes(int64_t K, int64_t N, int32_t precision, int32_t use_binning) {
  return footprint(K, N, precision, use_binning, 0);
}

mbar_status mbar_server_create(mbar_server** out, const mbar_server_config* cfg) {
  if (!out || !cfg) {
    set_error("mbar_server_create: null pointer argument");
    return MBAR_EINVAL;
  }
  *out = nullptr;
  if (cfg->workers < 1 || cfg->workers > 256 || cfg->hbm_budget_bytes == 0) {
    set_error("mbar_server_create: need 1 <= workers <= 256 and a nonzero memory budget");
    return MBAR_EINVAL;
  }
  auto* s = new (std::nothrow) mbar_server();
  if (!s) {
    set_error("mbar_server_create: out of host memory");
    return MBAR_ENOMEM;
  }
  s->cfg = *cfg;
  cudaGetDevice(&s->device);
  if ((cfg->flags & MBAR_BATCH_PERSISTENT) && cfg->opts.precision == MBAR_MIXED && cfg->opts.use_binning) {
    s->batcher = first_loop_batcher_create();
    if (!s->batcher) {
      delete s;
      set_error("mbar_server_create: cannot start the first-loop batcher");
      return MBAR_ENOMEM;
    }
  }
  try {
    for (int i = 0; i < cfg->workers; ++i) s->workers.emplace_back([s] { s->worker_main(); });
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    first_loop_batcher_destroy(s->batcher);
    delete s;
    set_error("mbar_server_create: cannot start worker threads");
    return MBAR_ENOMEM;
  }
  *out = s;
  return MBAR_OK;
}

mbar_status mbar_server_submit(mbar_server* s, int64_t K, int64_t N, const int64_t* N_k, const double* u_kn,
                               int32_t u_on_device, const double* phi, int32_t phi_on_device, int64_t* id) {
  if (!s || !N_k || !u_kn || !id) {
    set_error("mbar_server_submit: null pointer argument");
    return MBAR_EINVAL;
  }
  if (K < 1 || N < 1 || K > 1024) {
    set_error("mbar_server_submit: need 1 <= K <= 1024 and N >= 1");
    return K > 1024 ? MBAR_EUNSUPPORTED : MBAR_EINVAL;
  }
  auto r = std::make_shared<Request>();
  r->K = K;
  r->N = N;
  r->Nk.assign(N_k, N_k + K);
  r->u = u_kn;
  r->u_on_device = u_on_device;
  r->phi = phi;
  r->phi_on_device = phi_on_device;
  r->bytes = footprint(K, N, s->cfg.opts.precision, s->cfg.opts.use_binning, u_on_device);
  return enqueue(s, r, id, "mbar_server_submit");
}

mbar_status mbar_server_submit_factorised(mbar_server* s, int64_t K, int64_t N, const int64_t* N_k,
                                          const double* a, const double* b, const double* phi, int32_t on_device,
                                          int64_t* id) {
  if (!s || !N_k || !a || !b || !phi || !id) {
    set_error("mbar_server_submit_factorised: null pointer argument");
    return MBAR_EINVAL;
  }
  if (K < 1 || N < 1 || K > 1024) {
    set_error("mbar_server_submit_factorised: need 1 <= K <= 1024 and N >= 1");
    return K > 1024 ? MBAR_EUNSUPPORTED : MBAR_EINVAL;
  }
  auto r = std::make_shared<Request>();
  r->K = K;
  r->N = N;
  r->Nk.assign(N_k, N_k + K);
  r->factorised = true;
  r->fa = a;
  r->fb = b;
  r->phi = phi;
  r->phi_on_device = on_device;
  r->bytes = footprint_factorised(K, N, s->cfg.opts.precision, s->cfg.opts.use_binning);
  return enqueue(s, r, id, "mbar_server_submit_factorised");
}

mbar_status mbar_server_poll(mbar_server* s, int64_t id, int32_t* state) {
  if (!s || !state) {
    set_error("mbar_server_poll: null pointer argument");
    return MBAR_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) {
    set_error("mbar_server_poll: unknown request id %lld", static_cast<long long>(id));
    return MBAR_EINVAL;
  }
  *state = it->second->state;
  return MBAR_OK;
}

mbar_status mbar_server_wait(mbar_server* s, int64_t id, double* f_out, mbar_report* report, double* latency_s,
                             double* run_s) {
  if (!s) {
    set_error("mbar_server_wait: null server");
    return MBAR_EINVAL;
  }
  std::shared_ptr<Request> r;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) {
      set_error("mbar_server_wait: unknown request id %lld", static_cast<long long>(id));
      return MBAR_EINVAL;
    }
    r = it->second;
    s->cv_done.wait(lk, [&] { return r->state == 2; });
    s->all.erase(id);
  }
  if (f_out && !r->f.empty()) std::copy(r->f.begin(), r->f.end(), f_out);
  if (report) *report = r->report;
  if (latency_s) *latency_s = seconds_between(r->t_submit, r->t_done);
  if (run_s) *run_s = seconds_between(r->t_admit, r->t_done);
  if (r->status != MBAR_OK) set_error("request %lld: %s", static_cast<long long>(id), r->error.c_str());
  return r->status;
}

mbar_status mbar_server_stats(mbar_server* s, int64_t* completed, int32_t* peak_running, uint64_t* peak_bytes) {
  if (!s) {
    set_error("mbar_server_stats: null server");
    return MBAR_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (completed) *completed = s->completed;
  if (peak_running) *peak_running = s->peak_running;
  if (peak_bytes) *peak_bytes = s->peak_bytes;
  return MBAR_OK;
}

mbar_status mbar_server_destroy(mbar_server* s) {
  if (!s) return MBAR_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (auto& r : s->queue) {  // never admitted: dropped
      r->state = 2;
      r->status = MBAR_ESTATE;
      r->error = "server destroyed before the request was admitted";
    }
    s->queue.clear();
  }
  s->cv_work.notify_all();
  s->cv_done.notify_all();
  for (auto& t : s->workers) t.join();
  first_loop_batcher_destroy(s->batcher);  // after the workers: nothing is queued any more
  delete s;
  return MBAR_OK;
}

mbar_status mbar_batch_solve(int32_t P, const int64_t* K, const int64_t* N, const int64_t* const* N_k,
                             const double* const* u_kn, int32_t u_on_device, const double* const* phi,
                             int32_t phi_on_device, const mbar_server_config* cfg, double* const* f_out,
                             mbar_report* reports, mbar_status* statuses) {
  if (P < 0 || (P > 0 && (!K || !N || !N_k || !u_kn || !f_out))) {
    set_error("mbar_batch_solve: bad arguments");
    return MBAR_EINVAL;
  }
  mbar_server* s = nullptr;
  BUMBAR_TRY(mbar_server_create(&s, cfg));
  std::vector<int64_t> ids(static_cast<size_t>(P), -1);
  mbar_status first_err = MBAR_OK;
  for (int32_t p = 0; p < P; ++p) {
    const mbar_status st = mbar_server_submit(s, K[p], N[p], N_k[p], u_kn[p], u_on_device, phi ? phi[p] : nullptr,
                                              phi_on_device, &ids[p]);
    if (st != MBAR_OK) {
      if (statuses) statuses[p] = st;
      if (first_err == MBAR_OK) first_err = st;
    }
  }
  for (int32_t p = 0; p < P; ++p) {
    if (ids[p] < 0) continue;
    const mbar_status st = mbar_server_wait(s, ids[p], f_out[p], reports ? &reports[p] : nullptr, nullptr, nullptr);
    if (statuses) statuses[p] = st;
    if (st != MBAR_OK && first_err == MBAR_OK) first_err = st;
  }
  mbar_server_destroy(s);
  return first_err;
}

}  // extern "C"
