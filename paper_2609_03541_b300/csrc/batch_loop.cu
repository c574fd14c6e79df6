// Algorithm 1's first loop for many independent problems in ONE persistent
// launch (FP32 data, MIXED): a device work queue of problems (an atomic
// counter over an array of descriptors); each CTA takes the next problem,
// copies its first-loop level (sample-major, vT[p * Kp + k], ~100 bins) into
// shared memory once, and repeats the Eq. 1 step on chip -- logden and Q over
// the level, the update, the gauge, Eq. 2's relative step and the stopping
// test -- until s < eps, the step falls under the noise floor, a step
// underflows or the step budget runs out; then it takes the next problem.
//
// The arithmetic per step is that of the one-problem loop kernel
// (sci_loop.cu): exponents from the FP32 pairs (a_k log2 e as hi + lo,
// log2 e as kLog2e + kLog2eLo), per-warp FP32 row partials added in warp
// order, the update in FP64, a step whose Q_k < 1e-20 N_k not applied
// (ctrl->underflow: the host redoes it exactly). Only the work split differs
// (one CTA per problem, each lane holding up to kBatchStates / 32 states),
// so the sums add in another order: results agree with the one-problem
// kernel at FP32 rounding, not bit for bit.
#include <cmath>
#include <condition_variable>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace bumbar {

namespace {

constexpr int kBatchThreads = 256;
constexpr int kBatchWarps = kBatchThreads / 32;
constexpr int kBatchStates = 256;               // K limit of the batched loop
constexpr int kBatchPer = kBatchStates / 32;    // states per lane

struct BatchShared {
  double d_red[kBatchWarps];
  float s_red[kBatchWarps];
  int flags_red[kBatchWarps];
  int item;
  int decision;
};

__global__ void __launch_bounds__(kBatchThreads, 1)
    first_loop_batch_kernel(const BatchLoopItem* __restrict__ items, int count, int* __restrict__ next) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BatchShared* sh = reinterpret_cast<BatchShared*>(smem_raw);
  double* f_s = reinterpret_cast<double*>(smem_raw + 256);  // [kBatchStates]
  double* fn_s = f_s + kBatchStates;                          // [kBatchStates]
  float* ah_s = reinterpret_cast<float*>(fn_s + kBatchStates);  // [kBatchStates] a_k log2(e), hi
  float* al_s = ah_s + kBatchStates;                            // and lo
  float* part = al_s + kBatchStates;                            // [kBatchWarps][kBatchStates]
  float* lvl = part + kBatchWarps * kBatchStates;               // the level, n x Kp
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  for (;;) {
    if (tid == 0) sh->item = atomicAdd(next, 1);
    __syncthreads();
    const int it = sh->item;
    if (it >= count) break;
    const BatchLoopItem q = items[it];
    const int K = q.K, n = q.n, Kp = q.Kp;

    // the level into shared memory (16-byte vectors; n * Kp is a multiple of 4)
    {
      const float4* src = reinterpret_cast<const float4*>(q.vT);
      float4* dst = reinterpret_cast<float4*>(lvl);
      const int nv = n * Kp / 4;
      for (int i = tid; i < nv; i += kBatchThreads) dst[i] = src[i];
    }
    auto set_offset = [&](int k, double fk) {
      if (k < K) {
        const double a = (fk + q.logN[k]) * 1.4426950408889634;
        const float hi = static_cast<float>(a);
        ah_s[k] = hi;
        al_s[k] = isfinite(hi) ? static_cast<float>(a - static_cast<double>(hi)) : 0.f;  // N_k = 0: -inf
      } else {
        ah_s[k] = -INFINITY;
        al_s[k] = 0.f;
      }
    };
    for (int k = tid; k < kBatchStates; k += kBatchThreads) {
      f_s[k] = k < K ? q.f[k] : 0.0;
      set_offset(k, f_s[k]);
    }
    __syncthreads();

    int applied = 0;
    float last_s = INFINITY;
    double last_d = 0.0;
    int dec = 0;
    for (int64_t step = 0; step < q.max_steps; ++step) {
      // this lane's states: lane + 32 i, i < kBatchPer
      float ahi[kBatchPer], alo[kBatchPer], acc[kBatchPer];
#pragma unroll
      for (int i = 0; i < kBatchPer; ++i) {
        ahi[i] = ah_s[lane + 32 * i];
        alo[i] = al_s[lane + 32 * i];
        acc[i] = 0.f;
      }
      for (int p = warp; p < n; p += kBatchWarps) {
        const float* col = lvl + static_cast<size_t>(p) * Kp;
        float x[kBatchPer];
        float m = -INFINITY;
#pragma unroll
        for (int i = 0; i < kBatchPer; ++i) {
          const int k = lane + 32 * i;
          const float v = k < Kp ? col[k] : 0.f;
          x[i] = fmaf(-v, kLog2e, ahi[i]) + fmaf(-v, kLog2eLo, alo[i]);
          m = fmaxf(m, x[i]);
        }
        m = warp_max_f32(m);
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < kBatchPer; ++i) {
          x[i] = ex2_approx(x[i] - m);
          s += x[i];
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const float w = (q.H ? static_cast<float>(q.H[p]) : 1.f) / s;
#pragma unroll
        for (int i = 0; i < kBatchPer; ++i) acc[i] = fmaf(x[i], w, acc[i]);
      }
#pragma unroll
      for (int i = 0; i < kBatchPer; ++i) part[warp * kBatchStates + lane + 32 * i] = acc[i];
      __syncthreads();
      // epilogue 1: Q_k (the warps' partials in order), the update, underflow
      int under = 0;
      for (int k = tid; k < K; k += kBatchThreads) {
        float Q = 0.f;
        for (int w = 0; w < kBatchWarps; ++w) Q += part[w * kBatchStates + k];
        under |= !(static_cast<double>(Q) >= 1e-20 * q.Nk[k]);
        fn_s[k] = f_s[k] + q.logN[k] - static_cast<double>(logf(Q));
      }
      __syncthreads();
      const double f0n = fn_s[0], f0 = f_s[0];
      // epilogue 2: gauge, Eq. 2 (states with f_k = 0 skipped), max|df|
      float smax = -1.f;
      double dmax = 0.0;
      int finite = 1;
      for (int k = tid; k < K; k += kBatchThreads) {
        const double fo = fn_s[k] - f0n, fi = f_s[k];
        if (!isfinite(fo)) finite = 0;
        if (fi != 0.0) smax = fmaxf(smax, fabsf(static_cast<float>(fo - fi) / static_cast<float>(fi)));
        dmax = fmax(dmax, fabs(fo - (fi - f0)));
      }
      __syncthreads();  // every thread has read fn_s[0]
      for (int k = tid; k < K; k += kBatchThreads) fn_s[k] -= f0n;
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) {
        smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, o));
        dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        finite &= __shfl_xor_sync(0xffffffffu, finite, o);
        under |= __shfl_xor_sync(0xffffffffu, under, o);
      }
      if (lane == 0) {
        sh->s_red[warp] = smax;
        sh->d_red[warp] = dmax;
        sh->flags_red[warp] = finite | (under << 1);
      }
      __syncthreads();
      if (tid == 0) {
        float sm = -1.f;
        double dm = 0.0;
        int fl = 0, fin = 1;
        for (int w = 0; w < kBatchWarps; ++w) {
          sm = fmaxf(sm, sh->s_red[w]);
          dm = fmax(dm, sh->d_red[w]);
          fin &= sh->flags_red[w] & 1;
          fl |= sh->flags_red[w];
        }
        const float sv = sm < 0.f ? INFINITY : sm;
        int d = 0;
        if (fl & 2) {
          d = 1 | 2;  // keep f: the host redoes this step exactly
        } else {
          ++applied;
          last_s = sv;
          last_d = dm;
          if (!fin) q.ctrl->nonfinite = 1;
          if ((q.eps > 0.0 && sv < q.eps) || (q.noise > 0.0 && dm < q.noise) || !fin) d = 1;
        }
        sh->decision = d;
      }
      __syncthreads();
      dec = sh->decision;
      if (!(dec & 2))
        for (int k = tid; k < K; k += kBatchThreads) {
          f_s[k] = fn_s[k];
          set_offset(k, fn_s[k]);
        }
      __syncthreads();
      if (dec & 1) break;
    }
    if (tid == 0) {
      q.ctrl->iters += applied;
      if (applied > 0) q.ctrl->last_s = static_cast<double>(last_s);
      if ((dec & (1 | 2)) == 1 && applied > 0 &&
          ((q.eps > 0.0 && last_s < q.eps) || (q.noise > 0.0 && last_d < q.noise)))
        q.ctrl->done = 1;
      if (dec & 2) {
        q.ctrl->underflow = 1;
        if (q.s_out) *q.s_out = INFINITY;
      } else if (q.s_out && applied > 0) {
        *q.s_out = static_cast<double>(last_s);
      }
    }
    for (int k = tid; k < K; k += kBatchThreads) q.f[k] = f_s[k];
    __syncthreads();  // before the next item reuses shared memory
  }
}

size_t batch_fixed_smem() {
  return 256 + 2 * kBatchStates * sizeof(double) + 2 * kBatchStates * sizeof(float) +
         static_cast<size_t>(kBatchWarps) * kBatchStates * sizeof(float);
}

int batch_optin() {
  static int optin = -1;
  std::lock_guard<std::recursive_mutex> lock(init_mutex());
  if (optin < 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaGetLastError();
    optin = v;
  }
  return optin;
}

}  // namespace

bool first_loop_batch_supported(int64_t K, int64_t n) {
  if (K < 1 || K > kBatchStates || n < 1) return false;
  const size_t need = batch_fixed_smem() + static_cast<size_t>(n) * stage_pitch(K) * sizeof(float);
  return need <= static_cast<size_t>(batch_optin());
}

mbar_status first_loop_batch_launch(const BatchLoopItem* items_dev, int count, int* next_dev, size_t level_floats,
                                    cudaStream_t st) {
  if (count <= 0) return MBAR_OK;
  const size_t smem = batch_fixed_smem() + level_floats * sizeof(float);
  if (smem > static_cast<size_t>(batch_optin())) {
    set_error("first_loop_batch_launch: a level of %zu floats exceeds shared memory", level_floats);
    return MBAR_EUNSUPPORTED;
  }
  {
    std::lock_guard<std::recursive_mutex> lock(init_mutex());
    static bool init = false;
    if (!init) {
      cudaFuncSetAttribute(first_loop_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, batch_optin());
      init = true;
    }
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, first_loop_batch_kernel, kBatchThreads, smem) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  // persistent: as many CTAs as can be resident, none more than the problems
  const int grid = std::max(1, std::min(count, per_sm * num_sms()));
  BUMBAR_CUDA(cudaMemsetAsync(next_dev, 0, sizeof(int), st));
  first_loop_batch_kernel<<<grid, kBatchThreads, smem, st>>>(items_dev, count, next_dev);
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return MBAR_OK;
}

// Continuous batching of first loops for concurrent solves: a thread takes
// every item queued so far, runs them in one persistent launch on its own
// stream, wakes their submitters, and repeats; items that arrive while a
// launch runs go into the next one.
struct FirstLoopBatcher {
  static constexpr int kCapacity = 1024;  // items per launch
  struct Req {
    BatchLoopItem item;
    bool done = false;
    mbar_status st = MBAR_OK;
  };
  std::mutex mu;
  std::condition_variable cv_new, cv_done;
  std::vector<Req*> queue;
  bool stop = false;
  cudaStream_t st = nullptr;
  BatchLoopItem* items_d = nullptr;
  int* next_d = nullptr;
  std::thread th;
  int device = 0;
  int64_t launches = 0, items_run = 0;

  void loop() {
    cudaSetDevice(device);
    std::vector<Req*> batch;
    std::vector<BatchLoopItem> host;
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_new.wait(lk, [&] { return stop || !queue.empty(); });
        if (queue.empty()) break;  // stop requested and nothing left
        const size_t take = std::min<size_t>(queue.size(), kCapacity);
        batch.assign(queue.begin(), queue.begin() + static_cast<std::ptrdiff_t>(take));
        queue.erase(queue.begin(), queue.begin() + static_cast<std::ptrdiff_t>(take));
      }
      host.clear();
      size_t level_floats = 0;
      for (Req* r : batch) {
        host.push_back(r->item);
        level_floats = std::max(level_floats, static_cast<size_t>(r->item.n) * r->item.Kp);
      }
      mbar_status s = MBAR_OK;
      if (cudaMemcpyAsync(items_d, host.data(), host.size() * sizeof(BatchLoopItem), cudaMemcpyHostToDevice, st) !=
          cudaSuccess)
        s = cuda_status(cudaGetLastError(), "first-loop batch: descriptors");
      if (s == MBAR_OK) s = first_loop_batch_launch(items_d, static_cast<int>(host.size()), next_d, level_floats, st);
      if (s == MBAR_OK && cudaStreamSynchronize(st) != cudaSuccess)
        s = cuda_status(cudaGetLastError(), "first-loop batch");
      {
        std::lock_guard<std::mutex> lk(mu);
        ++launches;
        items_run += static_cast<int64_t>(batch.size());
        for (Req* r : batch) {
          r->st = s;
          r->done = true;
        }
      }
      cv_done.notify_all();
    }
  }
};

FirstLoopBatcher* first_loop_batcher_create() {
  auto* b = new (std::nothrow) FirstLoopBatcher();
  if (!b) return nullptr;
  cudaGetDevice(&b->device);
  if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&b->items_d), FirstLoopBatcher::kCapacity * sizeof(BatchLoopItem)) !=
          cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&b->next_d), sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    first_loop_batcher_destroy(b);
    return nullptr;
  }
  try {
    b->th = std::thread([b] { b->loop(); });
  } catch (...) {
    first_loop_batcher_destroy(b);
    return nullptr;
  }
  return b;
}

void first_loop_batcher_destroy(FirstLoopBatcher* b) {
  if (!b) return;
  {
    std::lock_guard<std::mutex> lk(b->mu);
    b->stop = true;
  }
  b->cv_new.notify_all();
  if (b->th.joinable()) b->th.join();
  if (b->items_d) cudaFree(b->items_d);
  if (b->next_d) cudaFree(b->next_d);
  if (b->st) cudaStreamDestroy(b->st);
  delete b;
}

mbar_status first_loop_batcher_run(FirstLoopBatcher* b, const BatchLoopItem& item) {
  FirstLoopBatcher::Req r;
  r.item = item;
  std::unique_lock<std::mutex> lk(b->mu);
  if (b->stop) {
    set_error("first-loop batch: the batcher is shutting down");
    return MBAR_ESTATE;
  }
  b->queue.push_back(&r);
  b->cv_new.notify_one();
  b->cv_done.wait(lk, [&] { return r.done; });
  if (r.st != MBAR_OK) set_error("first-loop batch: a batched launch failed");
  return r.st;
}

void first_loop_batcher_stats(FirstLoopBatcher* b, int64_t* launches, int64_t* items) {
  std::lock_guard<std::mutex> lk(b->mu);
  if (launches) *launches = b->launches;
  if (items) *items = b->items_run;
}

}  // namespace bumbar
