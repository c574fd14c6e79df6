// Sample-major variant of the fused paired-LSE pass (Eq. 1) for FP32 data:
// the unbinned passes of MIXED read the staging copy of the data, where
// every sample is one contiguous K-vector (vst[n * Kp + k], Kp = K rounded
// up to 4, zero padded). For every sample n
//     logden_n = log sum_j exp(a_j - v_jn),          a_j = f_j + log N_j,
//     Q_i     += exp(a_i - v_in - logden_n),
// in one read of v.
//
// Layout and schedule (one persistent CTA per SM):
//   * a stage is S consecutive samples, i.e. ONE contiguous run of S*Kp*4
//     bytes (~48 KB), fetched by a single 1-D bulk copy (cp.async.bulk) into
//     a ring of stages; a producer warp issues the copies, the other warps
//     compute. Stage size measured at K = 500 (4 GB pass): 32 KB x 4 stages
//     0.90 ms, 48 KB x 2 0.81 ms, 64 KB x 2 0.82 ms;
//     Long contiguous runs keep the DRAM pages open: the 2-D strip pattern
//     of the row-major store (128 bytes from each of K rows) measured
//     4.5 TB/s for the copies alone on B300, contiguous runs 7.1 TB/s;
//   * LPS lanes own one sample (LPS = 32 for Kp > 64, fewer for small K, so
//     a warp then takes several samples at once); a lane holds 4*NK entries
//     of the sample in registers (float4 reads from shared memory), with the
//     state offsets a_k log2(e) as FP32 (hi, lo) pairs in registers;
//   * per sample: x = a - v log2(e) (pairs: a_hi, a_lo and kLog2e,
//     kLog2eLo), max and sum by shuffles within the lane group, e = 2^(x -
//     max), and the lanes' row partials acc_k += e / sum (one sample per
//     lane group at a time: two samples at once measured slower with the
//     large stages, 0.92 vs 0.81 ms);
//   * every 64 sample slots a warp folds its FP32 partials (and those of its
//     lane groups) into its row of shared memory, kept as unevaluated FP32
//     sums hi + lo updated by TwoSum (64 FP32 terms <= 1 each: relative
//     error <= 3.8e-6, ~2e-7 typical, before the fold). FP64 adds there (the
//     FP64 pipe of B300 is slow, and the warps fold at about the same time)
//     cost 6.5 % of the pass at K = 500 with folds every 32 slots; TwoSum
//     every 32 slots 2.7 %, every 64 slots 1.4 %. At the end the warps' rows are added in warp order
//     (deterministic, FP64) and written as the CTA's row of the partial
//     sums, which lse_epilogue_kernel reduces;
//   * 1 / sum by rcp.approx (1 ulp; the IEEE division measured 2.3 % of the
//     pass at K = 500, 10 % at K = 16);
//   * the state(s) attaining a sample's maximum exponent contribute exactly 1
//     to its sum, the others r = sum_{k != k*} 2^(x_k - m). With a single
//     maximum its weight 1 / (1 + r) is accumulated as the exact count 1
//     (into the warp's unevaluated row pair with 32 lanes per sample, else
//     into a per-warp integer row in shared memory) plus the small
//     remainder -r / (1 + r): as a plain FP32 term close to 1 its deficit r
//     is rounded away, by the FP32 sum 1 + r itself and by partial sums of
//     ~64 terms close to 1, which biases Q_k (and the gradient Q_k - N_k) by
//     up to ~N_k 6e-8. On poorly overlapping states the Newton solution
//     then moves by that bias over the smallest eigenvalue of the Hessian
//     (1e-3..1e-2 kT for four umbrella windows 1.0 apart in an FP32 emulation
//     of the pass; 3.5e-6 kT with the split). Tied maxima get 1 / sum each.
#include <cmath>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace bumbar {

namespace {

constexpr uint32_t kSmSpin = 1u << 28;  // bounded mbarrier polls
constexpr int kSmFlush = 64;            // sample slots between folds of the FP32 partials
constexpr int kSmStageBytes = 48 * 1024;

}  // namespace

// LPS lanes per sample, NK float4 chunks per lane, NT threads (warp 0 is
// the producer, the other NT / 32 - 1 warps compute). EXACT: each sample's
// largest weight is split into its exact count and remainder (below); the
// plain variant adds every weight as an FP32 term (~30 % fewer instructions).
template <int LPS, int NK, int NT, bool EXACT>
__global__ void __launch_bounds__(NT, 1) lse_smaj_kernel(const float* __restrict__ vst, int Kp, int S, int stages,
                                                         LseParams p) {
  constexpr int SPW = 32 / LPS;  // samples per warp at once
  constexpr int NWC = NT / 32 - 1;  // compute warps
  constexpr int E = 4 * NK;      // entries per lane
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int K = p.K;
  const int64_t n = p.n;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (lse_skip(p)) return;

  const size_t sbytes = static_cast<size_t>(S) * Kp * 4;
  // [NWC][Kp] row partials as unevaluated FP32 sums hi + lo
  float2* rows = reinterpret_cast<float2*>(smem + stages * sbytes);
  uint64_t* full = reinterpret_cast<uint64_t*>(rows + static_cast<size_t>(NWC) * Kp);
  uint64_t* empty = full + stages;
  int* abort_flag = reinterpret_cast<int*>(empty + stages);
  // below 32 lanes per sample: [NWC][Kp] per-warp counts of the samples
  // whose single maximum is state k (a warp's lane groups may share k, so
  // these take shared-memory atomics, private to the warp); with 32 lanes
  // the counts go into the warps' rows directly
  unsigned* cnt = reinterpret_cast<unsigned*>(abort_flag + 4);

  const int64_t nchunks = (n + S - 1) / S;
  const int64_t first = blockIdx.x, stride = gridDim.x;
  const int count = first < nchunks ? static_cast<int>((nchunks - 1 - first) / stride + 1) : 0;

  if (tid == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NWC);
    }
    *abort_flag = 0;
    fence_barrier_init();
  }
  // the state offsets a_k log2(e) as FP32 (hi, lo) pairs, computed once per
  // CTA (the FP64 pipe is slow) into the first compute warp's partial row
  // (2 Kp floats); that row is zeroed once every compute warp
  // has copied its entries to registers
  float* a2 = reinterpret_cast<float*>(rows);
  for (int k = tid; k < Kp; k += NT) {
    float hi = -INFINITY, lo = 0.f;  // padding rows: weight 0
    if (k < K) {
      const double a = (p.f[k] + p.logN[k]) * 1.4426950408889634;
      hi = static_cast<float>(a);
      lo = isfinite(hi) ? static_cast<float>(a - static_cast<double>(hi)) : 0.f;  // N_k = 0: -inf
    }
    a2[k] = hi;
    a2[Kp + k] = lo;
  }
  for (int i = Kp + tid; i < NWC * Kp; i += NT) rows[i] = make_float2(0.f, 0.f);
  if constexpr (LPS < 32)
    for (int i = tid; i < NWC * Kp; i += NT) cnt[i] = 0u;
  __syncthreads();

  const int lig = lane % LPS;  // lane in group
  const int grp = lane / LPS;  // sample group within the warp

  if (warp == 0) {
    // ---- producer: one elected lane issues the ring of bulk copies ----
    if (lane == 0) {
      int issued = 0;
      for (int it = 0; it < count; ++it) {
        const int s = it % stages;
        if (it >= stages) {
          if (!mbar_wait_bounded(&empty[s], static_cast<uint32_t>((it / stages - 1) & 1), kSmSpin)) {
            atomicAdd(p.err, 1u);
            *reinterpret_cast<volatile int*>(abort_flag) = 1;
            break;
          }
        }
        if (*reinterpret_cast<volatile int*>(abort_flag)) break;
        const int64_t chunk = first + static_cast<int64_t>(it) * stride;
        const int64_t n0 = chunk * S;
        const int64_t ns = (n - n0 < S) ? n - n0 : S;
        // the bytes of ns samples, rounded up to 16 (the staging buffer has
        // 16 bytes of slack after its last sample)
        const uint32_t bytes = static_cast<uint32_t>((ns * Kp * 4 + 15) / 16 * 16);
        mbar_expect_tx(&full[s], bytes);
        bulk_load_1d(smem + s * sbytes, vst + n0 * Kp, bytes, &full[s]);
        ++issued;
      }
      // copies still in flight when leaving early: wait for them (bounded)
      for (int it = (issued > stages ? issued - stages : 0); it < issued; ++it)
        (void)mbar_wait_bounded(&full[it % stages], static_cast<uint32_t>((it / stages) & 1), kSmSpin);
    }
  } else {
    // ---- compute warps ----
    const int cw = warp - 1;
    constexpr int E2 = E / 2;
    // this lane's entries: k = 4 * (lig + LPS * i) + t, held as packed pairs
    // (entries 2j, 2j + 1) for the f32x2 instructions
    unsigned long long ahp[E2], alp[E2];
#pragma unroll
    for (int i = 0; i < NK; ++i)
#pragma unroll
      for (int t = 0; t < 4; t += 2) {
        const int k = 4 * (lig + LPS * i) + t;
        ahp[(4 * i + t) / 2] = pk2(k < Kp ? a2[k] : -INFINITY, k + 1 < Kp ? a2[k + 1] : -INFINITY);
        alp[(4 * i + t) / 2] = pk2(k < Kp ? a2[Kp + k] : 0.f, k + 1 < Kp ? a2[Kp + k + 1] : 0.f);
      }
    asm volatile("bar.sync 1, %0;" ::"n"(NWC * 32) : "memory");
    if (cw == 0) {
      for (int k = lane; k < Kp; k += 32) rows[k] = make_float2(0.f, 0.f);
      __syncwarp();
    }
    const unsigned long long nl2e = pk2(-kLog2e, -kLog2e), nl2elo = pk2(-kLog2eLo, -kLog2eLo);
    unsigned long long accp[E2];
#pragma unroll
    for (int j = 0; j < E2; ++j) accp[j] = 0ull;
    int slots = 0;
    float2* myrow = rows + static_cast<size_t>(cw) * Kp;
    auto fold = [&]() {
#pragma unroll
      for (int i = 0; i < NK; ++i)
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int e = 4 * i + t;
          float lo, hi;
          upk2(accp[e / 2], lo, hi);
          float v = (e & 1) ? hi : lo;
#pragma unroll
          for (int o = LPS; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          const int k = 4 * (lig + LPS * i) + t;
          if (grp == 0 && k < Kp) {
            // TwoSum (Knuth): hi + v = s + err exactly; the FP32 pair
            // carries ~48 bits, without the slow FP64 pipe
            const float2 c = myrow[k];
            const float sum = c.x + v, bv = sum - c.x;
            const float err = (c.x - (sum - bv)) + (v - bv);
            myrow[k] = make_float2(sum, c.y + err);
          }
        }
#pragma unroll
      for (int j = 0; j < E2; ++j) accp[j] = 0ull;
    };
    for (int it = 0; it < count; ++it) {
      const int s = it % stages;
      const bool ok = mbar_wait_bounded(&full[s], static_cast<uint32_t>((it / stages) & 1), kSmSpin);
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) {
          atomicAdd(p.err, 1u);
          *reinterpret_cast<volatile int*>(abort_flag) = 1;
        }
        break;
      }
      const int64_t n0 = (first + static_cast<int64_t>(it) * stride) * S;
      const int ns = static_cast<int>((n - n0 < S) ? n - n0 : S);
      const unsigned char* stage = smem + s * sbytes;
      // one sample slot at a time, round-robin over the compute warps
      const int nslots = (ns + SPW - 1) / SPW;
      const int nslots_full = (S + SPW - 1) / SPW;
      int sl = cw - static_cast<int>((static_cast<int64_t>(it) * nslots_full) % NWC);
      if (sl < 0) sl += NWC;
      for (; sl < nslots; sl += NWC) {
        const int j0 = sl * SPW + grp;
        const bool v0 = j0 < ns;
        const float* c0 = reinterpret_cast<const float*>(stage + static_cast<size_t>(v0 ? j0 : 0) * Kp * 4);
        // x = a log2(e) - v log2(e) from the FP32 pairs (a_hi, a_lo) and
        // (kLog2e, kLog2eLo), two entries per f32x2 instruction
        unsigned long long xp[E2];
        float m0 = -INFINITY, m1 = -INFINITY;
#pragma unroll
        for (int i = 0; i < NK; ++i) {
          const int k4 = 4 * (lig + LPS * i);
          float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
          if (k4 < Kp) a = *reinterpret_cast<const float4*>(c0 + k4);
          const unsigned long long v01 = pk2(a.x, a.y), v23 = pk2(a.z, a.w);
          xp[2 * i] = add2(fma2(v01, nl2e, ahp[2 * i]), fma2(v01, nl2elo, alp[2 * i]));
          xp[2 * i + 1] = add2(fma2(v23, nl2e, ahp[2 * i + 1]), fma2(v23, nl2elo, alp[2 * i + 1]));
          float p0, p1, q0, q1;
          upk2(xp[2 * i], p0, p1);
          upk2(xp[2 * i + 1], q0, q1);
          m0 = fmaxf(m0, fmaxf(p0, q0));
          m1 = fmaxf(m1, fmaxf(p1, q1));
        }
        m0 = fmaxf(m0, m1);
        if constexpr (LPS == 32) {
          m0 = warp_max_f32(m0);  // the whole warp holds the sample
        } else {
#pragma unroll
          for (int o = LPS / 2; o >= 1; o >>= 1) m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, o));
        }
        const unsigned long long nm = pk2(-m0, -m0);
        unsigned long long sp = 0ull;   // (sum over even entries, sum over odd entries)
        unsigned top = 0u;
        int nt = 0;
        if constexpr (EXACT) {
          // r = the sum of 2^(x - m) over the entries below the maximum; the
          // maximal entries (each exactly 1) are zeroed and marked in `top`
#pragma unroll
          for (int j = 0; j < E2; ++j) {
            float d0, d1;
            upk2(add2(xp[j], nm), d0, d1);
            const bool z0 = d0 == 0.f, z1 = d1 == 0.f;
            xp[j] = pk2(z0 ? 0.f : ex2_approx(d0), z1 ? 0.f : ex2_approx(d1));
            if (z0) top |= 1u << (2 * j);
            if (z1) top |= 2u << (2 * j);
            sp = add2(sp, xp[j]);
          }
          // the group's number of maximal entries: its lanes holding one,
          // counted exactly when some lane holds two or lanes tie
          const unsigned gm = LPS == 32 ? 0xffffffffu : ((1u << LPS) - 1u) << (grp * LPS);
          nt = __popc(__ballot_sync(0xffffffffu, top != 0u) & gm);
          if (__any_sync(0xffffffffu, (top & (top - 1u)) != 0u || nt > 1)) {
            nt = __popc(top);
#pragma unroll
            for (int o = LPS / 2; o >= 1; o >>= 1) nt += __shfl_xor_sync(0xffffffffu, nt, o);
          }
        } else {
#pragma unroll
          for (int j = 0; j < E2; ++j) {
            float d0, d1;
            upk2(add2(xp[j], nm), d0, d1);
            xp[j] = pk2(ex2_approx(d0), ex2_approx(d1));
            sp = add2(sp, xp[j]);
          }
        }
        float s0, s1;
        upk2(sp, s0, s1);
        s0 += s1;
#pragma unroll
        for (int o = LPS / 2; o >= 1; o >>= 1) s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        const float sum = EXACT ? static_cast<float>(nt) + s0 : s0;
        float w0 = 0.f, h0 = 0.f;
        if (v0) {
          const int64_t gn = n0 + j0;
          h0 = p.H ? static_cast<float>(p.H[gn]) : 1.f;
          w0 = h0 * rcp_approx(sum);
          if (p.logden != nullptr && lig == 0) static_cast<float*>(p.logden)[gn] = (m0 + __log2f(sum)) * kLn2;
        }
        const unsigned long long wp = pk2(w0, w0);
#pragma unroll
        for (int j = 0; j < E2; ++j) accp[j] = fma2(xp[j], wp, accp[j]);
        if (EXACT && top != 0u && w0 != 0.f) {
          // the maximal entries of this lane: a single maximum adds
          // -r / sum to its row and H to its count, tied maxima 1 / sum each
          const float add = nt == 1 ? -s0 * w0 : w0;
          do {
            const int e = __ffs(top) - 1;
            top &= top - 1u;
            const int k = 4 * (lig + LPS * (e >> 2)) + (e & 3);
            if constexpr (LPS == 32) {
              // one sample per warp: the row entry of state k is only ever
              // updated by this lane (here and in fold), so the count and
              // the remainder go into the unevaluated pair directly (TwoSum)
              float2 c = myrow[k];
              if (nt == 1) {
                const float sum1 = c.x + h0, b1 = sum1 - c.x;
                c.y += (c.x - (sum1 - b1)) + (h0 - b1);
                c.x = sum1;
              }
              const float sum2 = c.x + add, bv = sum2 - c.x;
              c.y += (c.x - (sum2 - bv)) + (add - bv);
              c.x = sum2;
              myrow[k] = c;
            } else {
              if (nt == 1) atomicAdd(&cnt[cw * Kp + k], static_cast<unsigned>(h0));
#pragma unroll
              for (int q = 0; q < E2; ++q)
                if (q == (e >> 1)) {
                  float lo, hi;
                  upk2(accp[q], lo, hi);
                  if (e & 1) hi += add; else lo += add;
                  accp[q] = pk2(lo, hi);
                }
            }
          } while (top != 0u);
        }
        if (++slots >= kSmFlush) {
          fold();
          slots = 0;
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
    fold();
  }

  // ---- per-CTA row sums: the compute warps' partials in warp order ----
  __syncthreads();
  double* out = p.partials + static_cast<size_t>(blockIdx.x) * K;
  for (int k = tid; k < K; k += NT) {
    double t = 0.0;
    for (int w = 0; w < NWC; ++w) {
      const float2 c = rows[static_cast<size_t>(w) * Kp + k];
      t += static_cast<double>(c.x) + static_cast<double>(c.y);
      if constexpr (LPS < 32) t += static_cast<double>(cnt[static_cast<size_t>(w) * Kp + k]);
    }
    out[k] = t;
  }
}

namespace {

// lanes per sample: as few as give every lane at most four float4 chunks
// (16 states), so the per-sample shuffles, reciprocal and logden write are
// spread over as many entries as the registers allow; 32 lanes (and more
// chunks per lane) from K = 256
void smaj_shape(int64_t K, int* lps, int* nk, int* nt) {
  const int64_t q = round_up(K, 4) / 4;
  int l = 1;
  while (l < 32 && l * 4 < q) l <<= 1;
  int c = static_cast<int>(ceil_div(q, static_cast<int64_t>(l)));
  if (l < 32 && c == 3) c = 4;
  *lps = l;
  *nk = c;
  *nt = c <= 4 ? 512 : 256;  // 15 or 7 compute warps + the producer warp
}

template <int LPS, int NK, int NT, bool EXACT>
void smaj_run_one(const LsePlan& pl, const float* vst, int Kp, const LseParams& prm, cudaStream_t st) {
  static bool init = false;
  {
    std::lock_guard<std::recursive_mutex> lock(init_mutex());
    if (!init) {
      int dev = 0, optin = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      cudaFuncSetAttribute(lse_smaj_kernel<LPS, NK, NT, EXACT>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
      init = true;
    }
  }
  lse_smaj_kernel<LPS, NK, NT, EXACT><<<pl.grid, NT, pl.smem, st>>>(vst, Kp, pl.C, pl.stages, prm);
}

template <int LPS, int NK, int NT>
void smaj_run(const LsePlan& pl, const float* vst, int Kp, const LseParams& prm, cudaStream_t st) {
  if (prm.exact_max) smaj_run_one<LPS, NK, NT, true>(pl, vst, Kp, prm, st);
  else smaj_run_one<LPS, NK, NT, false>(pl, vst, Kp, prm, st);
}

}  // namespace

LsePlan lse_smaj_plan(int64_t K, int64_t n) {
  int lps = 0, nk = 0, nt = 0, stage_bytes = 0;
  if (tuned_shape(kTuneSamples, K, n, &lps, &nk, &nt, &stage_bytes))
    return lse_smaj_plan_for(K, n, lps, nk, nt, stage_bytes);
  return lse_smaj_plan_rule(K, n);
}

LsePlan lse_smaj_plan_rule(int64_t K, int64_t n) {
  int lps = 0, nk = 0, nt = 0;
  smaj_shape(K, &lps, &nk, &nt);
  return lse_smaj_plan_for(K, n, lps, nk, nt, kSmStageBytes);
}

LsePlan lse_smaj_plan_for(int64_t K, int64_t n, int lps, int nk, int nt, int stage_bytes) {
  LsePlan pl{};
  const int64_t Kp = round_up(K, 4);
  const int spw = 32 / lps;
  // samples per stage: about stage_bytes (48 KB by the shape rule, also at
  // small K, where 32 KB stages measured 7 % slower), a multiple of 4
  // (16-byte aligned runs) and at least one sample slot per compute warp
  int64_t S = std::max<int64_t>(stage_bytes / (Kp * 4), 1);
  S = std::max<int64_t>(S, static_cast<int64_t>(spw) * (nt / 32 - 1));
  S = round_up(S, 4);
  const size_t sb = static_cast<size_t>(S) * Kp * 4;
  const size_t part = static_cast<size_t>(nt / 32 - 1) * Kp * 8;
  int stages = 6;
  while (stages > 2 && stages * sb + part > 200 * 1024) --stages;
  pl.variant = 2;
  pl.C = static_cast<int>(S);
  pl.stages = stages;
  pl.threads = nt;
  pl.J = nk;
  pl.H = lps;
  pl.num_strips = static_cast<int>(ceil_div(n, S));
  const size_t counts = lps < 32 ? static_cast<size_t>(nt / 32 - 1) * Kp * 4 : 0;
  pl.smem = stages * sb + part + 2 * stages * 8 + 16 + counts + 1024;
  static int optin = -1;
  {
    std::lock_guard<std::recursive_mutex> lock(init_mutex());
    if (optin < 0) {
      int dev = 0, v = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      cudaGetLastError();
      optin = v;
    }
  }
  pl.ok = optin > 0 && pl.smem <= static_cast<size_t>(optin);
  pl.grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(pl.num_strips, num_sms())));
  return pl;
}

bool lse_smaj_supported(int64_t K) { return K >= 1 && K <= 1024; }

// Where the sample-major pass beats the row-major FP32 kernels: everywhere
// it runs (measured on B300 at 1e9 entries, sample-major vs row-major: K =
// 16: 0.64 vs 3.03 ms; K = 50: 0.84 vs 1.29; K = 64: 0.69 vs 1.02; K = 128:
// 0.71 vs 1.06; K = 200: 0.86 vs 0.95; K = 500: 0.73 vs 0.87; K = 1000:
// 0.79 vs 1.82). Before lanes per sample were cut to give each lane up to
// 16 states, K = 64..128 measured 1.3-1.5 ms and the row-major kernel won.
bool lse_smaj_preferred(int64_t K) { return lse_smaj_supported(K); }

mbar_status lse_smaj_launch(const float* vst, const LsePlan& pl, LseParams prm, cudaStream_t st) {
  if (!pl.ok) {
    set_error("lse pass: %zu bytes of shared memory per CTA exceed the device limit", pl.smem);
    return MBAR_EUNSUPPORTED;
  }
  prm.nparts = pl.grid;
  prm.epi = prm.partials + static_cast<size_t>(pl.grid) * prm.K;
  const int Kp = static_cast<int>(round_up(prm.K, 4));
  const int lps = pl.H, nk = pl.J;
  // the instances the shape rule reaches: one lane per sample with 1, 2 or
  // 4 chunks; 2..16 lanes with 4 chunks; 32 lanes with 3..8 chunks
  bool ok = true;
  if (lps == 1 && nk == 1) smaj_run<1, 1, 512>(pl, vst, Kp, prm, st);
  else if (lps == 1 && nk == 2) smaj_run<1, 2, 512>(pl, vst, Kp, prm, st);
  else if (lps == 1 && nk == 4) smaj_run<1, 4, 512>(pl, vst, Kp, prm, st);
  else if (lps == 2 && nk == 4) smaj_run<2, 4, 512>(pl, vst, Kp, prm, st);
  else if (lps == 4 && nk == 4) smaj_run<4, 4, 512>(pl, vst, Kp, prm, st);
  else if (lps == 8 && nk == 4) smaj_run<8, 4, 512>(pl, vst, Kp, prm, st);
  else if (lps == 16 && nk == 4) smaj_run<16, 4, 512>(pl, vst, Kp, prm, st);
  else if (lps == 32) {
    switch (nk) {
      case 3: smaj_run<32, 3, 512>(pl, vst, Kp, prm, st); break;
      case 4: smaj_run<32, 4, 512>(pl, vst, Kp, prm, st); break;
      case 5: smaj_run<32, 5, 256>(pl, vst, Kp, prm, st); break;
      case 6: smaj_run<32, 6, 256>(pl, vst, Kp, prm, st); break;
      case 7: smaj_run<32, 7, 256>(pl, vst, Kp, prm, st); break;
      case 8: smaj_run<32, 8, 256>(pl, vst, Kp, prm, st); break;
      default: ok = false;
    }
  } else {
    ok = false;
  }
  if (!ok) {
    set_error("lse_smaj_launch: unsupported shape (%d lanes, %d chunks)", lps, nk);
    return MBAR_EUNSUPPORTED;
  }
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return lse_epilogue_launch(prm, st);
}

}  // namespace bumbar
