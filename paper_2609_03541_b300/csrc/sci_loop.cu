// Algorithm 1's SCI iterations on a small binned level in ONE launch (FP32
// data, MIXED): one cluster of 8 CTAs keeps f on chip and repeats the Eq. 1
// step — logden and Q over the level, the update, the gauge, Eq. 2's
// relative step and the stopping test — until s < eps (first loop), the
// step falls under the noise floor, or an iteration budget runs out.
//
// A level of ~100 bins is far too small to fill the GPU: as separate
// launches each step costs a pass (~15 us, a handful of CTAs) plus the
// epilogue (~13 us), nearly all of it latency. Here a step is a sweep of the
// level, sample-major (vT[p * Kp + k]), split over the cluster's CTAs, each
// through a ring of 1-D bulk copies from L2 (a producer warp streams its
// share again and again; the data do not depend on f), the per-sample work
// of the sample-major LSE pass on the compute warps, the CTAs' row partials
// exchanged over distributed shared memory, and an epilogue on the compute
// warps of every CTA (named barrier):
//   Q_k  = sum_p H_p 2^(x_kp - m_p) / s_p   (FP32 partials per warp, summed
//          in warp order, then over the CTAs in rank order),
//   f'_k = f_k + ln N_k - ln Q_k (FP64, with ln Q_k from the FP32 sum), gauge
//          f'_0 = 0, s = max over f_k != 0 of |f'_k / f_k - 1|, d = max|f'_k - f_k|,
// then the new offsets a_k log2(e) as FP32 (hi, lo) pairs, once per state
// (FP64 arithmetic is slow on this part).
// A step whose Q_k falls under 1e-20 N_k is not applied: the kernel stops
// with ctrl->underflow set, as the separate launches do, and the host redoes
// that step exactly in the log domain.
#include <cmath>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"
#include "smaj_core.cuh"

namespace bumbar {

namespace {

constexpr uint32_t kLoopSpin = 1u << 28;
constexpr int kLoopCluster = 8;  // CTAs (SMs) that share one level; each streams every 8th chunk
constexpr uint64_t kLoopWaitNs = 1000000000ull;  // bounded waits on the peers: 1 s

__device__ __forceinline__ void compute_barrier(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}
__device__ __forceinline__ uint32_t loop_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t loop_mapa(uint32_t addr, uint32_t rank) {
  uint32_t o;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(o) : "r"(addr), "r"(rank));
  return o;
}
__device__ __forceinline__ float ld_cluster_f32(uint32_t addr) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
  return v;
}
// a peer's step counter: store with release at cluster scope, read with
// acquire (every step a CTA finishes publishing raises its counter in every
// CTA; counters only grow, so a reader never confuses steps)
__device__ __forceinline__ void st_release_cluster_u32(uint32_t addr, uint32_t v) {
  asm volatile("st.release.cluster.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire_cluster_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.cluster.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t loop_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// wait until every CTA of the cluster has published step `target` (its
// counter here reached it); gives up after ~1 s
__device__ __forceinline__ bool wait_peers(const uint32_t* seq, uint32_t target) {
  const uint64_t t0 = loop_ns();
  for (int r = 0; r < kLoopCluster; ++r) {
    for (uint32_t i = 0;; ++i) {
      if (ld_acquire_cluster_u32(seq + r) >= target) break;
      if (i >= kLoopSpin || ((i & 255u) == 255u && loop_ns() - t0 > kLoopWaitNs)) return false;
    }
  }
  return true;
}
__device__ __forceinline__ void loop_cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

struct LoopShared {
  double d_red[32];
  float s_red[32];
  int flags_red[32];
  int stop;      // set by the compute warps: the producer stops issuing
  int decision;  // bit 0: stop the loop, bit 1: underflow, bit 3: timeout (bits 1, 3: step not applied)
};

}  // namespace

// One cluster of kLoopCluster CTAs per level: CTA r streams the chunks
// r, r + 8, ... of the level; after each sweep every CTA publishes its row
// partials (double-buffered) and raises its step counter in every peer,
// then each CTA adds the 8 partials in rank order (the same sums everywhere)
// and runs the same epilogue, so all CTAs take the same decisions; rank 0
// writes the results.
template <int LPS, int NK, int NT>
__global__ void __launch_bounds__(NT, 1) sci_loop_kernel(const float* __restrict__ vT, int Kp, int S, int stages,
                                                         SciLoopParams q) {
  constexpr int SPW = 32 / LPS;
  constexpr int NWC = NT / 32 - 1;
  constexpr int E = 4 * NK;
  constexpr int NC = NWC * 32;  // compute threads
  constexpr int CL = kLoopCluster;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int K = q.K;
  const int n = q.n;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rank = static_cast<int>(loop_ctarank());
  const size_t sbytes = static_cast<size_t>(S) * Kp * 4;
  float* part = reinterpret_cast<float*>(smem + stages * sbytes);                    // [NWC][Kp] warp partials
  float* cpart = part + static_cast<size_t>(NWC) * Kp;                              // [2][Kp] this CTA's partials
  double* f_s = reinterpret_cast<double*>(cpart + 2 * static_cast<size_t>(Kp) + 4);  // [Kp] current f
  double* fn_s = f_s + Kp;                                                          // [Kp] next f
  float* ah_s = reinterpret_cast<float*>(fn_s + Kp);                                // [Kp] a_k log2(e), hi
  float* al_s = ah_s + Kp;                                                          // [Kp] and lo
  uint64_t* full = reinterpret_cast<uint64_t*>(al_s + Kp);
  uint64_t* empty = full + stages;
  uint32_t* seq = reinterpret_cast<uint32_t*>(empty + stages);  // [CL] steps published by each CTA
  LoopShared* sh = reinterpret_cast<LoopShared*>(seq + 2 * CL);
  const int nchunks = (n + S - 1) / S;
  const int my_nch = nchunks > rank ? (nchunks - 1 - rank) / CL + 1 : 0;  // chunks rank, rank + CL, ...

  // a_k log2(e) as an FP32 (hi, lo) pair, once per state
  auto set_offset = [&](int k, double fk) {
    if (k < K) {
      const double a = (fk + q.logN[k]) * 1.4426950408889634;
      const float hi = static_cast<float>(a);
      ah_s[k] = hi;
      al_s[k] = isfinite(hi) ? static_cast<float>(a - static_cast<double>(hi)) : 0.f;  // N_k = 0: -inf
    } else {
      ah_s[k] = -INFINITY;  // padding rows: weight 0
      al_s[k] = 0.f;
    }
  };
  if (tid == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NWC);
    }
    for (int r = 0; r < CL; ++r) seq[r] = 0;
    sh->stop = 0;
    sh->decision = 0;
    fence_barrier_init();
  }
  for (int k = tid; k < Kp; k += NT) {
    f_s[k] = k < K ? q.f[k] : 0.0;
    set_offset(k, f_s[k]);
  }
  for (int i = tid; i < NWC * Kp; i += NT) part[i] = 0.f;
  __syncthreads();
  loop_cluster_sync();  // the peers' counters are zero before anyone publishes

  if (warp == 0) {
    // ---- producer: this CTA's chunks of the level, over and over ----
    if (lane == 0 && my_nch > 0) {
      int64_t issued = 0;
      bool failed = false;
      for (int64_t g = 0;; ++g) {
        const int s = static_cast<int>(g % stages);
        if (g >= stages) {
          const uint32_t par = static_cast<uint32_t>((g / stages - 1) & 1);
          bool ok = false;
          for (uint32_t spin = 0; spin < kLoopSpin; ++spin) {
            if (mbar_try_wait(&empty[s], par)) {
              ok = true;
              break;
            }
            if (*reinterpret_cast<volatile int*>(&sh->stop)) break;
          }
          if (!ok) {
            if (!*reinterpret_cast<volatile int*>(&sh->stop)) failed = true;
            break;
          }
        }
        if (*reinterpret_cast<volatile int*>(&sh->stop)) break;
        const int c = rank + CL * static_cast<int>(g % my_nch);
        const int n0 = c * S;
        const int ns = (n - n0 < S) ? n - n0 : S;
        const uint32_t bytes = static_cast<uint32_t>(static_cast<size_t>(ns) * Kp * 4);
        mbar_expect_tx(&full[s], bytes);
        bulk_load_1d(smem + s * sbytes, vT + static_cast<size_t>(n0) * Kp, bytes, &full[s]);
        ++issued;
      }
      if (failed) atomicAdd(q.err, 1u);
      // copies still in flight: wait for them (bounded) before the CTA ends
      for (int64_t g = (issued > stages ? issued - stages : 0); g < issued; ++g)
        (void)mbar_wait_bounded(&full[g % stages], static_cast<uint32_t>((g / stages) & 1), kLoopSpin);
    }
    __syncwarp();
  } else {
    // ---- compute warps ----
    const int cw = warp - 1, tc = tid - 32;
    const int lig = lane % LPS, grp = lane / LPS;
    float* mypart = part + static_cast<size_t>(cw) * Kp;
    const int npairs_full = (S + 2 * SPW - 1) / (2 * SPW);
    int64_t g = 0;  // chunks consumed so far
    int applied = 0;
    float last_s = INFINITY;
    double last_d = 0.0;
    bool timed_out = false;
    for (int64_t step = 0; step < q.max_steps; ++step) {
      float ahi[E], alo[E];
#pragma unroll
      for (int i = 0; i < NK; ++i) {
        const int k4 = 4 * (lig + LPS * i);
        float4 h = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY), l = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k4 < Kp) {
          h = *reinterpret_cast<const float4*>(ah_s + k4);
          l = *reinterpret_cast<const float4*>(al_s + k4);
        }
        ahi[4 * i] = h.x;
        ahi[4 * i + 1] = h.y;
        ahi[4 * i + 2] = h.z;
        ahi[4 * i + 3] = h.w;
        alo[4 * i] = l.x;
        alo[4 * i + 1] = l.y;
        alo[4 * i + 2] = l.z;
        alo[4 * i + 3] = l.w;
      }
      float acc[E];
#pragma unroll
      for (int e = 0; e < E; ++e) acc[e] = 0.f;
      for (int j = 0; j < my_nch; ++j, ++g) {
        const int s = static_cast<int>(g % stages);
        if (!timed_out) {
          const bool ok = mbar_wait_bounded(&full[s], static_cast<uint32_t>((g / stages) & 1), kLoopSpin);
          timed_out = !__all_sync(0xffffffffu, ok);
        }
        if (!timed_out) {
          const int n0 = (rank + CL * j) * S;
          const int ns = (n - n0 < S) ? n - n0 : S;
          const unsigned char* stage = smem + s * sbytes;
          const int npairs = (ns + 2 * SPW - 1) / (2 * SPW);
          // pairs round-robin over the compute warps across chunks
          int ps = cw - static_cast<int>((g * npairs_full) % NWC);
          if (ps < 0) ps += NWC;
          for (; ps < npairs; ps += NWC) {
            const int j0 = (2 * ps) * SPW + grp, j1 = (2 * ps + 1) * SPW + grp;
            const bool v0 = j0 < ns, v1 = j1 < ns;
            const float* c0 = reinterpret_cast<const float*>(stage + static_cast<size_t>(v0 ? j0 : 0) * Kp * 4);
            const float* c1 = reinterpret_cast<const float*>(stage + static_cast<size_t>(v1 ? j1 : 0) * Kp * 4);
            float x0[E], x1[E], m0, m1, s0, s1;
            smaj_pair<LPS, NK>(c0, c1, lig, Kp, ahi, alo, x0, x1, m0, m1, s0, s1);
            const float w0 = v0 ? (q.H ? static_cast<float>(q.H[n0 + j0]) : 1.f) / s0 : 0.f;
            const float w1 = v1 ? (q.H ? static_cast<float>(q.H[n0 + j1]) : 1.f) / s1 : 0.f;
#pragma unroll
            for (int e = 0; e < E; ++e) acc[e] = fmaf(x1[e], w1, fmaf(x0[e], w0, acc[e]));
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
      }
      // this warp's row partials (its lane groups added)
#pragma unroll
      for (int i = 0; i < NK; ++i)
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          float v = acc[4 * i + t];
#pragma unroll
          for (int o = LPS; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          const int k = 4 * (lig + LPS * i) + t;
          if (grp == 0 && k < Kp) mypart[k] = v;
        }
      compute_barrier(NC);
      // this CTA's row partials (warps in order), published to the cluster
      float* cp = cpart + static_cast<size_t>(step & 1) * Kp;
      for (int k = tc; k < K; k += NC) {
        float v = 0.f;
        for (int w = 0; w < NWC; ++w) v += part[static_cast<size_t>(w) * Kp + k];
        cp[k] = v;
      }
      compute_barrier(NC);
      if (tc == 0) {
        asm volatile("fence.acq_rel.cluster;" ::: "memory");
        for (int r = 0; r < CL; ++r)
          st_release_cluster_u32(loop_mapa(smem_u32(seq + rank), static_cast<uint32_t>(r)),
                                 static_cast<uint32_t>(step + 1));
      }
      // the partials of step `step` of every CTA are published; a CTA
      // overwrites this buffer two steps later, after it has seen every
      // CTA's next step, i.e. after every CTA has finished reading this one
      const bool peers_ok = wait_peers(seq, static_cast<uint32_t>(step + 1));
      const bool all_ok = __all_sync(0xffffffffu, peers_ok);
      // epilogue 1: Q_k (the CTAs' partials in rank order), the update
      // f_k + ln N_k - ln Q_k, underflow
      int under = 0;
      for (int k = tc; k < K; k += NC) {
        const uint32_t a = smem_u32(cp + k);
        float Q = 0.f;
        for (int r = 0; r < CL; ++r) Q += ld_cluster_f32(loop_mapa(a, static_cast<uint32_t>(r)));
        under |= !(static_cast<double>(Q) >= 1e-20 * q.Nk[k]);
        fn_s[k] = f_s[k] + q.logN[k] - static_cast<double>(logf(Q));
      }
      compute_barrier(NC);
      const double f0n = fn_s[0], f0 = f_s[0];
      // epilogue 2: gauge, Eq. 2 (states with f_k = 0 skipped), max|df|
      float smax = -1.f;
      double dmax = 0.0;
      int finite = 1;
      for (int k = tc; k < K; k += NC) {
        const double fo = fn_s[k] - f0n, fi = f_s[k];
        if (!isfinite(fo)) finite = 0;
        if (fi != 0.0) smax = fmaxf(smax, fabsf(static_cast<float>(fo - fi) / static_cast<float>(fi)));
        dmax = fmax(dmax, fabs(fo - (fi - f0)));
      }
      compute_barrier(NC);  // every thread has read fn_s[0]
      for (int k = tc; k < K; k += NC) fn_s[k] -= f0n;
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) {
        smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, o));
        dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        finite &= __shfl_xor_sync(0xffffffffu, finite, o);
        under |= __shfl_xor_sync(0xffffffffu, under, o);
      }
      if (lane == 0) {
        sh->s_red[cw] = smax;
        sh->d_red[cw] = dmax;
        sh->flags_red[cw] = finite | (under << 1) | ((timed_out || !all_ok) ? 4 : 0);
      }
      compute_barrier(NC);
      if (tc == 0) {
        float sm = -1.f;
        double dm = 0.0;
        int fl = 0, fin = 1;
        for (int w = 0; w < NWC; ++w) {
          sm = fmaxf(sm, sh->s_red[w]);
          dm = fmax(dm, sh->d_red[w]);
          fin &= sh->flags_red[w] & 1;
          fl |= sh->flags_red[w];
        }
        const float sv = sm < 0.f ? INFINITY : sm;
        int dec = 0;
        if (fl & 4) {
          dec = 1 | 8;  // a bounded wait gave up: stop, keep f
          atomicAdd(q.err, 1u);
        } else if (fl & 2) {
          dec = 1 | 2;  // keep f: the host redoes this step exactly
        } else {
          ++applied;
          last_s = sv;
          last_d = dm;
          if (!fin && rank == 0) q.ctrl->nonfinite = 1;
          if ((q.eps > 0.0 && sv < q.eps) || (q.noise > 0.0 && dm < q.noise) || !fin) dec = 1;
        }
        sh->decision = dec;
      }
      compute_barrier(NC);
      const int dec = sh->decision;
      if (!(dec & (2 | 8)))
        for (int k = tc; k < K; k += NC) {
          f_s[k] = fn_s[k];
          set_offset(k, fn_s[k]);
        }
      compute_barrier(NC);
      if (dec & 1) break;
    }
    if (tc == 0) {
      *reinterpret_cast<volatile int*>(&sh->stop) = 1;  // the producer stops issuing
      if (rank == 0) {
        const int dec = sh->decision;
        q.ctrl->iters += applied;
        if (applied > 0) q.ctrl->last_s = static_cast<double>(last_s);
        if ((dec & (1 | 2 | 8)) == 1 && applied > 0) {
          // stopped by the test (not by an underflow or a timeout)
          if ((q.eps > 0.0 && last_s < q.eps) || (q.noise > 0.0 && last_d < q.noise)) q.ctrl->done = 1;
        }
        if (dec & 2) {
          q.ctrl->underflow = 1;
          if (q.s_out) *q.s_out = INFINITY;
        } else if (q.s_out && applied > 0) {
          *q.s_out = static_cast<double>(last_s);
        }
        if (q.d_out && applied > 0) *q.d_out = last_d;
      }
    }
    if (rank == 0)
      for (int k = tc; k < K; k += NC) q.f[k] = f_s[k];
  }
  // no peer reads this CTA's shared memory or arrives on its barrier after this
  loop_cluster_sync();
}

// ---------------------------------------------------------------------------
// Grid-wide variant for levels that fit in the shared memory of all SMs
// (up to ~25 MB: 148 x ~200 KB): one cooperative launch of one CTA per SM.
// Each CTA loads its contiguous range of the level's bins once and keeps it
// in shared memory for every step, so a step reads nothing from L2 but f
// and the reduction scratch. A step:
//   1. the CTA's row partials of Q_k (FP32, warps in order) -> scratch;
//   2. grid barrier;
//   3. CTA b reduces the states k = b, b + G, ... over the G CTAs in rank
//      order (every CTA also reduces state 0 for the gauge), forms the
//      update, the gauge, Eq. 2's relative step and max|df| for them, and
//      writes f'_k and its per-CTA maxima to scratch;
//   4. grid barrier;
//   5. every CTA reads the G maxima and the new f, and takes the same
//      decision (stop test, underflow, non-finite) as the cluster kernel.
// The arithmetic is that of the cluster kernel, with the row partials
// grouped by CTA instead of by the cluster's chunk order. Every barrier wait
// is bounded (~1 s); a CTA that gives up raises a shared abort word, which
// ends the other CTAs' waits, and the launch reports the timeout.
struct GridShared {
  double d_red[32];
  float s_red[32];
  int flags_red[32];
  int decision;
  int ok;
};

__device__ __forceinline__ unsigned ld_acquire_gpu_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// arrive on the grid barrier and wait until `target` arrivals (all CTAs of
// this and the earlier barriers); false on a timeout or an abort elsewhere
__device__ bool grid_barrier(unsigned* bar, unsigned* abort_w, unsigned target, GridShared* sh) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    bool ok = true;
    const uint64_t t0 = loop_ns();
    for (uint32_t i = 0;; ++i) {
      if (ld_acquire_gpu_u32(bar) >= target) break;
      if ((i & 63u) == 63u) {
        if (ld_acquire_gpu_u32(abort_w) != 0u || loop_ns() - t0 > kLoopWaitNs || i >= kLoopSpin) {
          atomicExch(abort_w, 1u);
          ok = false;
          break;
        }
      }
    }
    __threadfence();
    sh->ok = ok ? 1 : 0;
  }
  __syncthreads();
  return sh->ok != 0;
}

template <int LPS, int NK, int NT>
__global__ void __launch_bounds__(NT, 1) sci_grid_kernel(const float* __restrict__ vT, int Kp, SciLoopParams q,
                                                         unsigned char* __restrict__ scratch) {
  constexpr int SPW = 32 / LPS;
  constexpr int NW = NT / 32;
  constexpr int E = 4 * NK;
  extern __shared__ __align__(16) unsigned char gsm_raw[];
  __shared__ GridShared sh;
  const int G = static_cast<int>(gridDim.x), b = static_cast<int>(blockIdx.x);
  const int K = q.K, n = q.n;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lig = lane % LPS, grp = lane / LPS;
  const int p0 = static_cast<int>(static_cast<int64_t>(b) * n / G);
  const int p1 = static_cast<int>(static_cast<int64_t>(b + 1) * n / G);
  const int nb = p1 - p0;
  float* lv = reinterpret_cast<float*>(gsm_raw);                 // [nb][Kp] this CTA's bins
  float* part = lv + static_cast<size_t>(nb) * Kp;               // [NW][Kp] warp partials
  double* f_s = reinterpret_cast<double*>(part + static_cast<size_t>(NW) * Kp);  // [Kp]
  double* fn_s = f_s + Kp;                                       // [Kp] the step's new f
  float* ah_s = reinterpret_cast<float*>(fn_s + Kp);             // [Kp] a_k log2(e), hi
  float* al_s = ah_s + Kp;                                       // [Kp] and lo
  // the states this CTA reduces: k = b + G i (i < nown), then state 0 for the
  // gauge; red holds their G partials each, qs their sums
  const int nown = b < K ? (K - b + G - 1) / G : 0;
  const int nsr = nown + 1;
  float* red = al_s + Kp;                                        // [nsr][G]
  float* qs = red + static_cast<size_t>(nsr) * G;                // [nsr]
  unsigned* bar = reinterpret_cast<unsigned*>(scratch);
  unsigned* abort_w = bar + 1;
  double* slots = reinterpret_cast<double*>(scratch + 256);      // [G][4]: s, d, flags
  double* fnew = slots + 4 * static_cast<size_t>(G);              // [Kp]
  float* gpart = reinterpret_cast<float*>(fnew + Kp);             // [G][Kp]

  auto set_offset = [&](int k, double fk) {
    if (k < K) {
      const double a = (fk + q.logN[k]) * 1.4426950408889634;
      const float hi = static_cast<float>(a);
      ah_s[k] = hi;
      al_s[k] = isfinite(hi) ? static_cast<float>(a - static_cast<double>(hi)) : 0.f;  // N_k = 0: -inf
    } else {
      ah_s[k] = -INFINITY;  // padding rows: weight 0
      al_s[k] = 0.f;
    }
  };
  {
    const float4* src = reinterpret_cast<const float4*>(vT + static_cast<size_t>(p0) * Kp);
    float4* dst = reinterpret_cast<float4*>(lv);
    const int n4 = nb * (Kp / 4);
    for (int i = tid; i < n4; i += NT) dst[i] = src[i];
  }
  for (int k = tid; k < Kp; k += NT) {
    f_s[k] = k < K ? q.f[k] : 0.0;
    set_offset(k, f_s[k]);
  }
  __syncthreads();

  unsigned nbar = 0;
  int applied = 0;
  float last_s = INFINITY;
  double last_d = 0.0;
  bool aborted = false;
  int dec = 0;
  const int npairs = (nb + 2 * SPW - 1) / (2 * SPW);
  for (int64_t step = 0; step < q.max_steps; ++step) {
    float ahi[E], alo[E];
#pragma unroll
    for (int i = 0; i < NK; ++i) {
      const int k4 = 4 * (lig + LPS * i);
      float4 h = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY), l = make_float4(0.f, 0.f, 0.f, 0.f);
      if (k4 < Kp) {
        h = *reinterpret_cast<const float4*>(ah_s + k4);
        l = *reinterpret_cast<const float4*>(al_s + k4);
      }
      ahi[4 * i] = h.x;
      ahi[4 * i + 1] = h.y;
      ahi[4 * i + 2] = h.z;
      ahi[4 * i + 3] = h.w;
      alo[4 * i] = l.x;
      alo[4 * i + 1] = l.y;
      alo[4 * i + 2] = l.z;
      alo[4 * i + 3] = l.w;
    }
    float acc[E];
#pragma unroll
    for (int e = 0; e < E; ++e) acc[e] = 0.f;
    for (int ps = warp; ps < npairs; ps += NW) {
      const int j0 = (2 * ps) * SPW + grp, j1 = (2 * ps + 1) * SPW + grp;
      const bool v0 = j0 < nb, v1 = j1 < nb;
      const float* c0 = lv + static_cast<size_t>(v0 ? j0 : 0) * Kp;
      const float* c1 = lv + static_cast<size_t>(v1 ? j1 : 0) * Kp;
      float x0[E], x1[E], m0, m1, s0, s1;
      smaj_pair<LPS, NK>(c0, c1, lig, Kp, ahi, alo, x0, x1, m0, m1, s0, s1);
      const float w0 = v0 ? (q.H ? static_cast<float>(q.H[p0 + j0]) : 1.f) / s0 : 0.f;
      const float w1 = v1 ? (q.H ? static_cast<float>(q.H[p0 + j1]) : 1.f) / s1 : 0.f;
#pragma unroll
      for (int e = 0; e < E; ++e) acc[e] = fmaf(x1[e], w1, fmaf(x0[e], w0, acc[e]));
    }
    float* mypart = part + static_cast<size_t>(warp) * Kp;
#pragma unroll
    for (int i = 0; i < NK; ++i)
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        float v = acc[4 * i + t];
#pragma unroll
        for (int o = LPS; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        const int k = 4 * (lig + LPS * i) + t;
        if (grp == 0 && k < Kp) mypart[k] = v;
      }
    __syncthreads();
    for (int k = tid; k < K; k += NT) {
      float v = 0.f;
      for (int w = 0; w < NW; ++w) v += part[static_cast<size_t>(w) * Kp + k];
      gpart[static_cast<size_t>(b) * Kp + k] = v;
    }
    if (!grid_barrier(bar, abort_w, static_cast<unsigned>(G) * ++nbar, &sh)) {
      aborted = true;
      break;
    }
    // Q_k of this CTA's states and of state 0 over the G CTAs' partials: all
    // loads at once into shared memory, then per state the lanes add
    // r = lane, lane + 32, ... in order and a fixed shuffle tree combines
    // them (the same bits for Q_0 in every CTA)
    for (int i = tid; i < nsr * G; i += NT) {
      const int sidx = i / G, r = i - sidx * G;
      const int k = sidx < nown ? b + G * sidx : 0;
      red[i] = __ldcg(gpart + static_cast<size_t>(r) * Kp + k);
    }
    __syncthreads();
    for (int sidx = warp; sidx < nsr; sidx += NW) {
      float v = 0.f;
      for (int r = lane; r < G; r += 32) v += red[sidx * G + r];
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) qs[sidx] = v;
    }
    __syncthreads();
    // the update, the gauge f'_0 = 0, Eq. 2's step and max|df| of the states
    const double f0n = f_s[0] + q.logN[0] - static_cast<double>(logf(qs[nown])), f0 = f_s[0];
    float smax = -1.f;  // -1: no f_k != 0 seen
    double dmax = 0.0;
    int finite = 1, under = 0;
    for (int sidx = tid; sidx < nown; sidx += NT) {
      const int k = b + G * sidx;
      const float Q = qs[sidx];
      under |= !(static_cast<double>(Q) >= 1e-20 * q.Nk[k]);
      const double fo = (f_s[k] + q.logN[k] - static_cast<double>(logf(Q))) - f0n, fi = f_s[k];
      fnew[k] = fo;
      if (!isfinite(fo)) finite = 0;
      if (fi != 0.0) smax = fmaxf(smax, fabsf(static_cast<float>(fo - fi) / static_cast<float>(fi)));
      dmax = fmax(dmax, fabs(fo - (fi - f0)));
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, o));
      dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
      finite &= __shfl_xor_sync(0xffffffffu, finite, o);
      under |= __shfl_xor_sync(0xffffffffu, under, o);
    }
    if (lane == 0) {
      sh.s_red[warp] = smax;
      sh.d_red[warp] = dmax;
      sh.flags_red[warp] = finite | (under << 1);
    }
    __syncthreads();
    if (tid == 0) {
      float sm = -1.f;
      double dm = 0.0;
      int fin = 1, un = 0;
      for (int w = 0; w < NW; ++w) {
        sm = fmaxf(sm, sh.s_red[w]);
        dm = fmax(dm, sh.d_red[w]);
        fin &= sh.flags_red[w] & 1;
        un |= (sh.flags_red[w] >> 1) & 1;
      }
      double* sl = slots + 4 * static_cast<size_t>(b);
      sl[0] = static_cast<double>(sm);
      sl[1] = dm;
      sl[2] = static_cast<double>(fin | (un << 1));
    }
    if (!grid_barrier(bar, abort_w, static_cast<unsigned>(G) * ++nbar, &sh)) {
      aborted = true;
      break;
    }
    // every CTA combines the G maxima (max and or/and do not depend on the
    // order) and takes the same decision
    float sm = -1.f;
    double dm = 0.0;
    int fin = 1, un = 0;
    for (int r = tid; r < G; r += NT) {
      const double* sl = slots + 4 * static_cast<size_t>(r);
      sm = fmaxf(sm, static_cast<float>(__ldcg(sl)));
      dm = fmax(dm, __ldcg(sl + 1));
      const int fl = static_cast<int>(__ldcg(sl + 2));
      fin &= fl & 1;
      un |= (fl >> 1) & 1;
    }
    for (int k = tid; k < K; k += NT) fn_s[k] = __ldcg(fnew + k);  // with the maxima: one round trip
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      sm = fmaxf(sm, __shfl_xor_sync(0xffffffffu, sm, o));
      dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
      fin &= __shfl_xor_sync(0xffffffffu, fin, o);
      un |= __shfl_xor_sync(0xffffffffu, un, o);
    }
    __syncthreads();  // the slice's use of sh.*_red is over
    if (lane == 0) {
      sh.s_red[warp] = sm;
      sh.d_red[warp] = dm;
      sh.flags_red[warp] = fin | (un << 1);
    }
    __syncthreads();
    if (tid == 0) {
      float smf = -1.f;
      double dmf = 0.0;
      int finf = 1, unf = 0;
      for (int w = 0; w < NW; ++w) {
        smf = fmaxf(smf, sh.s_red[w]);
        dmf = fmax(dmf, sh.d_red[w]);
        finf &= sh.flags_red[w] & 1;
        unf |= (sh.flags_red[w] >> 1) & 1;
      }
      const float sv = smf < 0.f ? INFINITY : smf;
      int d = 0;
      if (unf) {
        d = 1 | 2;  // keep f: the host redoes this step exactly
      } else {
        ++applied;
        last_s = sv;
        last_d = dmf;
        if (!finf && b == 0) q.ctrl->nonfinite = 1;
        if ((q.eps > 0.0 && sv < q.eps) || (q.noise > 0.0 && dmf < q.noise) || !finf) d = 1;
      }
      sh.decision = d;
    }
    __syncthreads();
    dec = sh.decision;
    if (!(dec & 2))
      for (int k = tid; k < K; k += NT) {
        f_s[k] = fn_s[k];
        set_offset(k, f_s[k]);
      }
    __syncthreads();
    if (dec & 1) break;
  }
  if (b == 0) {
    if (tid == 0) {
      if (aborted) {
        atomicAdd(q.err, 1u);
        dec = 1 | 8;
      }
      q.ctrl->iters += applied;
      if (applied > 0) q.ctrl->last_s = static_cast<double>(last_s);
      if ((dec & (1 | 2 | 8)) == 1 && applied > 0) {
        // stopped by the test (not by an underflow or a timeout)
        if ((q.eps > 0.0 && last_s < q.eps) || (q.noise > 0.0 && last_d < q.noise)) q.ctrl->done = 1;
      }
      if (dec & 2) {
        q.ctrl->underflow = 1;
        if (q.s_out) *q.s_out = INFINITY;
      } else if (q.s_out && applied > 0) {
        *q.s_out = static_cast<double>(last_s);
      }
      if (q.d_out && applied > 0) *q.d_out = last_d;
    }
    for (int k = tid; k < K; k += NT) q.f[k] = f_s[k];
  }
}

namespace {

template <int LPS, int NK, int NT>
mbar_status loop_run(const float* vT, int Kp, int S, int stages, size_t smem, const SciLoopParams& prm,
                     cudaStream_t st) {
  static bool init = false;
  {
    std::lock_guard<std::recursive_mutex> lock(init_mutex());
    if (!init) {
      int dev = 0, optin = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      cudaFuncSetAttribute(sci_loop_kernel<LPS, NK, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
      init = true;
    }
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kLoopCluster);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kLoopCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  BUMBAR_CUDA(cudaLaunchKernelEx(&cfg, sci_loop_kernel<LPS, NK, NT>, vT, Kp, S, stages, prm));
  count_launches(1);
  return MBAR_OK;
}

struct LoopPlan {
  int lps, nk, nt, S, stages;
  size_t smem;
};

LoopPlan loop_plan(int64_t K) {
  LoopPlan pl{};
  // lanes per sample: as few as give every lane at most 16 states (the
  // per-sample shuffles and reciprocals spread over more entries; the rule
  // of the sample-major pass, which it made 2x faster at K = 16..128)
  const int64_t q = stage_pitch(K) / 4;
  pl.lps = 1;
  while (pl.lps < 32 && pl.lps * 4 < q) pl.lps <<= 1;
  pl.nk = static_cast<int>(ceil_div(q, static_cast<int64_t>(pl.lps)));
  if (pl.lps < 32 && pl.nk == 3) pl.nk = 4;
  pl.nt = pl.nk >= 4 ? 256 : 512;  // the register budget of 512 threads is too small for 16 entries here
  const int64_t Kp = stage_pitch(K);
  const int nwc = pl.nt / 32 - 1;
  int64_t S = std::max<int64_t>(16 * 1024 / (Kp * 4), 1);
  S = std::max<int64_t>(S, static_cast<int64_t>(2 * 32 / pl.lps));
  pl.S = static_cast<int>(S);
  const size_t sb = static_cast<size_t>(S) * Kp * 4;
  const size_t fixed = static_cast<size_t>(nwc) * Kp * 4 + 2 * Kp * 4 + 16 + 2 * Kp * 8 + 2 * Kp * 4 + 1024 + 512;
  pl.stages = 8;
  while (pl.stages > 2 && pl.stages * sb + fixed > 200 * 1024) --pl.stages;
  pl.smem = pl.stages * sb + fixed + 2 * pl.stages * 8 + 8 * kLoopCluster + sizeof(LoopShared);
  return pl;
}

struct GridPlan {
  int lps, nk, nt, G;
  size_t smem;
};

// the cluster kernel's lane shape; at least four bins per CTA (fewer CTAs
// make cheaper barriers on small levels), at most one CTA per SM
GridPlan grid_plan(int64_t K, int64_t n) {
  const LoopPlan lp = loop_plan(K);
  GridPlan g{};
  g.lps = lp.lps;
  g.nk = lp.nk;
  g.nt = lp.nt;
  g.G = static_cast<int>(std::min<int64_t>(num_sms(), std::max<int64_t>(1, n / 4)));
  const int64_t Kp = stage_pitch(K);
  const int64_t nb = ceil_div(n, static_cast<int64_t>(g.G));  // bins of the largest CTA range
  const int64_t nsr = ceil_div(K, static_cast<int64_t>(g.G)) + 1;  // states a CTA reduces
  g.smem = static_cast<size_t>(nb * Kp * 4 + (g.nt / 32) * Kp * 4 + 2 * Kp * 8 + 2 * Kp * 4 + nsr * (g.G + 1) * 4);
  return g;
}

template <int LPS, int NK, int NT>
mbar_status grid_run(const float* vT, int Kp, const GridPlan& pl, const SciLoopParams& prm, void* scratch,
                     cudaStream_t st) {
  static bool init = false;
  {
    std::lock_guard<std::recursive_mutex> lock(init_mutex());
    if (!init) {
      int dev = 0, optin = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      cudaFuncAttributes fa = {};
      BUMBAR_CUDA(cudaFuncGetAttributes(&fa, sci_grid_kernel<LPS, NK, NT>));
      BUMBAR_CUDA(cudaFuncSetAttribute(sci_grid_kernel<LPS, NK, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       optin - static_cast<int>(fa.sharedSizeBytes)));
      init = true;
    }
  }
  BUMBAR_CUDA(cudaMemsetAsync(scratch, 0, 256, st));  // barrier counter and abort word
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(pl.G));
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = pl.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // all CTAs resident at once: they wait on one another
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  BUMBAR_CUDA(cudaLaunchKernelEx(&cfg, sci_grid_kernel<LPS, NK, NT>, vT, Kp, prm,
                                 static_cast<unsigned char*>(scratch)));
  count_launches(1);
  return MBAR_OK;
}

}  // namespace

bool sci_grid_supported(int64_t K, int64_t n) {
  if (K < 1 || K > 1024 || n < 1 || n > (int64_t{1} << 30)) return false;
  return grid_plan(K, n).smem <= 200 * 1024;
}

size_t sci_grid_scratch_bytes(int64_t K) {
  const int64_t Kp = stage_pitch(K);
  return static_cast<size_t>(256 + 4 * 8 * num_sms() + Kp * 8 + static_cast<int64_t>(num_sms()) * Kp * 4);
}

mbar_status sci_grid_launch(const float* vT, const SciLoopParams& prm, void* scratch, cudaStream_t st) {
  if (!sci_grid_supported(prm.K, prm.n)) {
    set_error("sci_grid_launch: unsupported level");
    return MBAR_EUNSUPPORTED;
  }
  const GridPlan pl = grid_plan(prm.K, prm.n);
  const int Kp = static_cast<int>(stage_pitch(prm.K));
  if (pl.lps < 32) {
    switch (pl.lps) {
#define BUMBAR_GRID_SMALL(L)                                                              \
  case L:                                                                                 \
    if (pl.nk == 1) return grid_run<L, 1, 512>(vT, Kp, pl, prm, scratch, st);             \
    if (pl.nk == 2) return grid_run<L, 2, 512>(vT, Kp, pl, prm, scratch, st);             \
    return grid_run<L, 4, 256>(vT, Kp, pl, prm, scratch, st);
      BUMBAR_GRID_SMALL(1)
      BUMBAR_GRID_SMALL(2)
      BUMBAR_GRID_SMALL(4)
      BUMBAR_GRID_SMALL(8)
      BUMBAR_GRID_SMALL(16)
#undef BUMBAR_GRID_SMALL
      default: break;
    }
  } else {
    switch (pl.nk) {
      case 1: return grid_run<32, 1, 512>(vT, Kp, pl, prm, scratch, st);
      case 2: return grid_run<32, 2, 512>(vT, Kp, pl, prm, scratch, st);
      case 3: return grid_run<32, 3, 512>(vT, Kp, pl, prm, scratch, st);
      case 4: return grid_run<32, 4, 256>(vT, Kp, pl, prm, scratch, st);
      case 5: return grid_run<32, 5, 256>(vT, Kp, pl, prm, scratch, st);
      case 6: return grid_run<32, 6, 256>(vT, Kp, pl, prm, scratch, st);
      case 7: return grid_run<32, 7, 256>(vT, Kp, pl, prm, scratch, st);
      case 8: return grid_run<32, 8, 256>(vT, Kp, pl, prm, scratch, st);
      default: break;
    }
  }
  set_error("sci_grid_launch: unsupported shape");
  return MBAR_EUNSUPPORTED;
}

bool sci_loop_supported(int64_t K, int64_t n, double max_bytes) {
  if (K < 1 || K > 1024 || n < 1) return false;
  // one cluster of 8 CTAs sweeps the whole level each step: worth it while
  // the level is small (a separate pass + epilogue costs ~30-40 us of
  // latency per step)
  return static_cast<double>(n) * stage_pitch(K) * 4 <= max_bytes && loop_plan(K).smem <= 220 * 1024;
}

size_t sci_loop_level_bytes(int64_t K, int64_t n) { return static_cast<size_t>(n) * stage_pitch(K) * 4; }

mbar_status sci_loop_launch(const float* vT, const SciLoopParams& prm, cudaStream_t st) {
  const LoopPlan pl = loop_plan(prm.K);
  const int Kp = static_cast<int>(stage_pitch(prm.K));
  if (pl.lps < 32) {
    switch (pl.lps) {
#define BUMBAR_LOOP_SMALL(L)                                                                   \
  case L:                                                                                      \
    if (pl.nk == 1) return loop_run<L, 1, 512>(vT, Kp, pl.S, pl.stages, pl.smem, prm, st);     \
    if (pl.nk == 2) return loop_run<L, 2, 512>(vT, Kp, pl.S, pl.stages, pl.smem, prm, st);     \
    return loop_run<L, 4, 256>(vT, Kp, pl.S, pl.stages, pl.smem, prm, st);
      BUMBAR_LOOP_SMALL(1)
      BUMBAR_LOOP_SMALL(2)
      BUMBAR_LOOP_SMALL(4)
      BUMBAR_LOOP_SMALL(8)
      BUMBAR_LOOP_SMALL(16)
#undef BUMBAR_LOOP_SMALL
      default: break;
    }
  } else {
    switch (pl.nk) {
      case 1: return loop_run<32, 1, 512>(vT, Kp, pl.S, pl.stages, pl.smem, prm, st);
      case 2: return loop_run<32, 2, 512>(vT, Kp, pl.S, pl.stages, pl.smem, prm, st);
      case 3: return loop_run<32, 3, 512>(vT, Kp, pl.S, pl.stages, pl.smem, prm, st);
      case 4: return loop_run<32, 4, 256>(vT, Kp, pl.S, pl.stages, pl.smem, prm, st);
      case 5: return loop_run<32, 5, 256>(vT, Kp, pl.S, pl.stages, pl.smem, prm, st);
      case 6: return loop_run<32, 6, 256>(vT, Kp, pl.S, pl.stages, pl.smem, prm, st);
      case 7: return loop_run<32, 7, 256>(vT, Kp, pl.S, pl.stages, pl.smem, prm, st);
      case 8: return loop_run<32, 8, 256>(vT, Kp, pl.S, pl.stages, pl.smem, prm, st);
      default: break;
    }
  }
  set_error("sci_loop_launch: unsupported shape");
  return MBAR_EUNSUPPORTED;
}

}  // namespace bumbar
