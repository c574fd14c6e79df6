// Fused paired-LSE pass (Eq. 1) over factorised reduced potentials
//     u_kp = a_k + b_k phi_p,
// the setting the paper starts from (u_kp = beta_k E_p: a = 0, b = beta,
// phi = the sample's energy). u is generated in registers from phi, so the
// pass reads 8 bytes per sample (12 with counts) instead of K * 4: it is
// bound by the SFU (one ex2 per entry) and the FP32 pipe, not by HBM.
// For every sample p
//     logden_p = log sum_j exp(f_j + log N_j - a_j - b_j phi_p),
//     Q_i     += H_p exp(f_i + log N_i - a_i - b_i phi_p - logden_p).
//
// Arithmetic: per state the FP64 constants c_k = (f_k + log N_k - a_k)
// log2(e) and b'_k = b_k log2(e) become unevaluated FP32 pairs (hi, lo), as
// does each phi_p. Each sample is taken relative to a reference state r(p)
// close to its largest exponent (a table of the maximising state at 4096
// points spread over the range of phi, built per pass by fact_ref_kernel):
//     x_kp - x_rp = [(c_hi,k - c_hi,r) - (b_hi,k - b_hi,r) p_hi]
//                 + [lo_k - lo_r],   lo_k = c_lo,k - b_lo,k p_hi - b_hi,k p_lo.
// Where c_k and c_r (b'_k and b'_r) lie within a factor of two of each other
// -- the states that carry weight, on large magnitudes -- both differences
// are exact (Sterbenz); elsewhere they round at their own magnitude. The
// bracket then rounds once, at the magnitude of x_kp - x_rp rather than of
// x_kp: u in the thousands or hundreds of thousands of kT (replica ladders
// u = beta_k E) keeps the accuracy of u near 0. The dropped b_lo p_lo term is
// 2^-48 of the product. That form costs three more FP32 operations per entry
// (measured 1.55x the pass time at K = 500), so it is taken only where it is
// needed: the table kernel bounds |x| by max|c| + max|b'| max|phi| and sets
// the table's `relative` flag above 2^12 (one FP32 ulp 2.4e-4); below it the
// pass forms x_kp itself, fma(-b_hi, p_hi, c_hi) + lo_k, rounded once at
// |x_kp|. The flag is the same for the whole grid (a uniform branch). The
// pairs of entries go through f32x2 instructions, then max, ex2, sum and one
// FMA into the row partial.
// Schedule: one CTA per SM, every warp computes. Warps take 32-sample chunks
// round robin over the grid; lane l loads phi (and H) of sample l of the
// chunk, and LPS-lane groups take the samples one after another (shuffles).
// A lane holds 4 NK states (LPS lanes cover Kp = K rounded up to 4; up to 16
// states per lane below K = 256, so at K <= 16 a lane owns whole samples),
// with the four constants of each in registers. Row partials as in the
// sample-major pass: FP32 per lane, folded every 64 samples into the warp's
// row of shared memory as an unevaluated FP32 sum (TwoSum), the rows added
// in warp order in FP64 at the end; lse_epilogue_kernel reduces the CTAs'
// rows.
#include <cmath>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace bumbar {

namespace {

constexpr int kFactFlush = 64;  // sample slots between folds of the FP32 partials

// FP64 -> FP32 pair (hi, lo), hi = RN32(x); lo = 0 when hi is not finite
__device__ __forceinline__ void split_pair(double x, float& hi, float& lo) {
  hi = static_cast<float>(x);
  lo = isfinite(hi) ? static_cast<float>(x - static_cast<double>(hi)) : 0.f;
}

// The same per sample with integer operations (the FP64 pipe of B300 is
// narrow, and this conversion sits on every sample's path); zero, tiny and
// huge values take the FP64 route.
__device__ __forceinline__ void split_pair_fast(double x, float& hi, float& lo) {
  if (!split_f64(x, hi, lo)) split_pair(x, hi, lo);
}

constexpr int kRangeParts = 256;  // partial (min, max) of phi for a pass without a known range
constexpr int kRefThreads = 256;

// Per-CTA min and max of phi (grid-stride), for passes given no range.
__global__ void __launch_bounds__(kRefThreads) fact_range_kernel(const double* __restrict__ phi, int64_t n,
                                                                 double* __restrict__ mins,
                                                                 double* __restrict__ maxs) {
  __shared__ double smin[kRefThreads], smax[kRefThreads];
  double lo = INFINITY, hi = -INFINITY;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * kRefThreads + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * kRefThreads) {
    const double v = phi[i];
    lo = fmin(lo, v);
    hi = fmax(hi, v);
  }
  smin[threadIdx.x] = lo;
  smax[threadIdx.x] = hi;
  __syncthreads();
  for (int o = kRefThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + o]);
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    mins[blockIdx.x] = smin[0];
    maxs[blockIdx.x] = smax[0];
  }
}

// The reference-state table of one pass: the range [lo, hi] of phi from
// `nparts` partial minima and maxima, then for grid point g (one thread) the
// state maximising c_k - b'_k phi_g, phi_g = lo + g (hi - lo) / (G - 1), in
// FP32 (a state within rounding of the maximum serves as well). States of
// weight zero (c_k = -inf) are never chosen while another state exists.
__global__ void __launch_bounds__(kRefThreads) fact_ref_kernel(const double* __restrict__ a,
                                                               const double* __restrict__ b, const double* f,
                                                               const double* logN, int K, const double* mins,
                                                               const double* maxs, int nparts, FactRef* out) {
  __shared__ float2 cb[1024];
  __shared__ double slo[kRefThreads], shi[kRefThreads];
  __shared__ float smc[kRefThreads], smb[kRefThreads];
  double lo = INFINITY, hi = -INFINITY;
  for (int i = threadIdx.x; i < nparts; i += kRefThreads) {
    lo = fmin(lo, mins[i]);
    hi = fmax(hi, maxs[i]);
  }
  slo[threadIdx.x] = lo;
  shi[threadIdx.x] = hi;
  float mc = 0.f, mb = 0.f;  // largest finite |c_k| and |b'_k|
  for (int k = threadIdx.x; k < K; k += kRefThreads) {
    const float2 v = make_float2(static_cast<float>((f[k] + logN[k] - a[k]) * 1.4426950408889634),
                                 static_cast<float>(b[k] * 1.4426950408889634));
    cb[k] = v;
    if (isfinite(v.x)) mc = fmaxf(mc, fabsf(v.x));
    mb = fmaxf(mb, fabsf(v.y));
  }
  smc[threadIdx.x] = mc;
  smb[threadIdx.x] = mb;
  __syncthreads();
  for (int o = kRefThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      slo[threadIdx.x] = fmin(slo[threadIdx.x], slo[threadIdx.x + o]);
      shi[threadIdx.x] = fmax(shi[threadIdx.x], shi[threadIdx.x + o]);
      smc[threadIdx.x] = fmaxf(smc[threadIdx.x], smc[threadIdx.x + o]);
      smb[threadIdx.x] = fmaxf(smb[threadIdx.x], smb[threadIdx.x + o]);
    }
    __syncthreads();
  }
  lo = slo[0];
  hi = shi[0];
  const bool spread = hi > lo;
  const double step = spread ? (hi - lo) / (kRefGrid - 1) : 0.0;
  const int g = blockIdx.x * kRefThreads + threadIdx.x;
  if (g < kRefGrid) {
    const float x = static_cast<float>(lo + step * g);
    int best = 0;
    float bv = -INFINITY;
    for (int k = 0; k < K; ++k) {
      const float2 c = cb[k];
      const float v = fmaf(-c.y, x, c.x);
      if (v > bv) {
        bv = v;
        best = k;
      }
    }
    out->state[g] = static_cast<int16_t>(best);
  }
  if (g == 0) {
    out->lo = static_cast<float>(lo);
    out->inv_step = spread ? static_cast<float>(1.0 / step) : 0.f;
    // a bound on |x_kp| = |c_k - b'_k phi_p|
    const double X = static_cast<double>(smc[0]) + static_cast<double>(smb[0]) * fmax(fabs(lo), fabs(hi));
    out->relative = X > 4096.0 ? 1 : 0;
  }
}

}  // namespace

// EXACT: the state(s) attaining a sample's maximum exponent contribute
// exactly 1 to its sum; with a single maximum its weight 1 / (1 + r) is
// accumulated as the exact count (into the warp's row pair with 32 lanes per
// sample, else a per-warp integer row in shared memory) plus the remainder
// -r / (1 + r), tied maxima 1 / sum each (as in the sample-major pass: FP32
// terms close to 1 lose their deficits r, which biases Q by up to ~6e-8 N).
template <int LPS, int NK, int NT, bool EXACT>
__global__ void __launch_bounds__(NT, 1) lse_fact_kernel(const double* __restrict__ a, const double* __restrict__ b,
                                                         const double* __restrict__ phi, int Kp,
                                                         const FactRef* __restrict__ ref, LseParams p) {
  constexpr int SPW = 32 / LPS;  // samples per warp at once
  constexpr int NW = NT / 32;
  constexpr int E = 4 * NK;      // states per lane
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* cst = reinterpret_cast<float4*>(smem_raw);   // [Kp] (c_hi, c_lo, b_hi, b_lo)
  float2* rows = reinterpret_cast<float2*>(cst + Kp);  // [NW][Kp] unevaluated sums hi + lo
  int16_t* tbl = reinterpret_cast<int16_t*>(rows + static_cast<size_t>(NW) * Kp);  // [kRefGrid] reference states
  unsigned* cnt = reinterpret_cast<unsigned*>(tbl + kRefGrid);  // [NW][Kp], EXACT, LPS < 32
  const int K = p.K;
  const int64_t n = p.n;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (lse_skip(p)) return;

  for (int k = tid; k < Kp; k += NT) {
    float4 c = make_float4(-INFINITY, 0.f, 0.f, 0.f);  // padding states: weight 0
    if (k < K) {
      split_pair((p.f[k] + p.logN[k] - a[k]) * 1.4426950408889634, c.x, c.y);  // N_k = 0: -inf
      split_pair(b[k] * 1.4426950408889634, c.z, c.w);
    }
    cst[k] = c;
  }
  for (int i = tid; i < NW * Kp; i += NT) rows[i] = make_float2(0.f, 0.f);
  for (int i = tid; i < kRefGrid / 8; i += NT)
    reinterpret_cast<int4*>(tbl)[i] = reinterpret_cast<const int4*>(ref->state)[i];
  if constexpr (EXACT && LPS < 32)
    for (int i = tid; i < NW * Kp; i += NT) cnt[i] = 0u;
  const float ref_lo = ref->lo, ref_inv = ref->inv_step;
  const bool rel = ref->relative != 0;  // the same for the whole grid
  __syncthreads();

  const int lig = lane % LPS;  // lane in group
  const int grp = lane / LPS;  // sample group within the warp
  // entries e and e + 1 of the lane side by side (f32x2): c_hi, c_lo, -b_hi, -b_lo
  unsigned long long ch2[E / 2], cl2[E / 2], nbh2[E / 2], nbl2[E / 2];
#pragma unroll
  for (int i = 0; i < NK; ++i)
#pragma unroll
    for (int t = 0; t < 4; t += 2) {
      const int k = 4 * (lig + LPS * i) + t;
      const float4 c0 = k < Kp ? cst[k] : make_float4(-INFINITY, 0.f, 0.f, 0.f);
      const float4 c1 = k + 1 < Kp ? cst[k + 1] : make_float4(-INFINITY, 0.f, 0.f, 0.f);
      const int q = (4 * i + t) / 2;
      ch2[q] = pk2(c0.x, c1.x);
      cl2[q] = pk2(c0.y, c1.y);
      nbh2[q] = pk2(-c0.z, -c1.z);
      nbl2[q] = pk2(-c0.w, -c1.w);
    }
  float acc[E];
#pragma unroll
  for (int e = 0; e < E; ++e) acc[e] = 0.f;
  float2* myrow = rows + static_cast<size_t>(warp) * Kp;
  auto fold = [&]() {
#pragma unroll
    for (int i = 0; i < NK; ++i)
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int e = 4 * i + t;
        float v = acc[e];
#pragma unroll
        for (int o = LPS; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        const int k = 4 * (lig + LPS * i) + t;
        if (grp == 0 && k < Kp) {
          // TwoSum (Knuth): hi + v = sum + err exactly
          const float2 c = myrow[k];
          const float sum = c.x + v, bv = sum - c.x;
          const float err = (c.x - (sum - bv)) + (v - bv);
          myrow[k] = make_float2(sum, c.y + err);
        }
        acc[e] = 0.f;
      }
  };

  int since = 0;
  const int64_t nchunks = (n + 31) / 32;
  for (int64_t chunk = static_cast<int64_t>(blockIdx.x) * NW + warp; chunk < nchunks;
       chunk += static_cast<int64_t>(gridDim.x) * NW) {
    const int64_t base = chunk * 32;
    const int nloc = static_cast<int>(n - base < 32 ? n - base : 32);
    float ph_l = 0.f, pl_l = 0.f, h_l = 0.f;
    if (lane < nloc) {
      split_pair_fast(phi[base + lane], ph_l, pl_l);
      h_l = p.H ? static_cast<float>(p.H[base + lane]) : 1.f;
    }
    // the lane's sample: reference state r from the table, its c_hi and b_hi,
    // and lo_r = c_lo,r - b_lo,r p_hi - b_hi,r p_lo
    float chr_l = 0.f, bhr_l = 0.f, lor_l = 0.f;
    if (rel) {
      const int g = min(max(__float2int_rn((ph_l - ref_lo) * ref_inv), 0), kRefGrid - 1);
      const float4 cr = cst[tbl[g]];
      chr_l = cr.x;
      bhr_l = cr.z;
      lor_l = fmaf(-cr.w, ph_l, fmaf(-cr.z, pl_l, cr.y));
    }
    float ld_mine = 0.f;  // logden of sample `lane` of the chunk, written once per chunk
    for (int j0 = 0; j0 < nloc; j0 += SPW) {
      const int j = j0 + grp;  // < 32: j0 is a multiple of SPW, grp < SPW
      const float ph = __shfl_sync(0xffffffffu, ph_l, j);
      const float pl = __shfl_sync(0xffffffffu, pl_l, j);
      const float hw = __shfl_sync(0xffffffffu, h_l, j);
      // the reference state's values: only the relative form uses them
      float chr = 0.f, bhr = 0.f, lor = 0.f;
      if (rel) {
        chr = __shfl_sync(0xffffffffu, chr_l, j);
        bhr = __shfl_sync(0xffffffffu, bhr_l, j);
        lor = __shfl_sync(0xffffffffu, lor_l, j);
      }
      const unsigned long long ph2 = pk2(ph, ph), pl2 = pk2(pl, pl);
      const unsigned long long nchr2 = pk2(-chr, -chr), bhr2 = pk2(bhr, bhr), nlor2 = pk2(-lor, -lor);
      float x[E];  // x_kp - x_rp, or x_kp (log2 units)
      float m0 = -INFINITY, m1 = -INFINITY;
      if (rel) {
#pragma unroll
        for (int q = 0; q < E / 2; ++q) {
          const unsigned long long dch = add2(ch2[q], nchr2);     // c_hi,k - c_hi,r (exact)
          const unsigned long long ndb = add2(nbh2[q], bhr2);     // -(b_hi,k - b_hi,r) (exact)
          const unsigned long long xh = fma2(ndb, ph2, dch);      // one rounding
          const unsigned long long lo = fma2(nbl2[q], ph2, fma2(nbh2[q], pl2, cl2[q]));
          upk2(add2(xh, add2(lo, nlor2)), x[2 * q], x[2 * q + 1]);
          m0 = fmaxf(m0, x[2 * q]);
          m1 = fmaxf(m1, x[2 * q + 1]);
        }
      } else {
        // |x| <= 2^12: x_kp itself, rounded once where c_k and b'_k phi_p cancel
#pragma unroll
        for (int q = 0; q < E / 2; ++q) {
          const unsigned long long xh = fma2(nbh2[q], ph2, ch2[q]);
          const unsigned long long lo = fma2(nbl2[q], ph2, fma2(nbh2[q], pl2, cl2[q]));
          upk2(add2(xh, lo), x[2 * q], x[2 * q + 1]);
          m0 = fmaxf(m0, x[2 * q]);
          m1 = fmaxf(m1, x[2 * q + 1]);
        }
      }
      float m = fmaxf(m0, m1);
      if constexpr (LPS == 32) {
        m = warp_max_f32(m);  // the whole warp holds one sample
      } else {
#pragma unroll
        for (int o = LPS / 2; o >= 1; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      }
      float s0 = 0.f, s1 = 0.f;
      unsigned top = 0u;
      int nt = 0;
      if constexpr (EXACT) {
#pragma unroll
        for (int e = 0; e < E; e += 2) {
          const float d0 = x[e] - m, d1 = x[e + 1] - m;
          const bool z0 = d0 == 0.f, z1 = d1 == 0.f;
          x[e] = z0 ? 0.f : ex2_approx(d0);
          x[e + 1] = z1 ? 0.f : ex2_approx(d1);
          if (z0) top |= 1u << e;
          if (z1) top |= 2u << e;
          s0 += x[e];
          s1 += x[e + 1];
        }
        const unsigned gm = LPS == 32 ? 0xffffffffu : ((1u << LPS) - 1u) << (grp * LPS);
        nt = __popc(__ballot_sync(0xffffffffu, top != 0u) & gm);
        if (__any_sync(0xffffffffu, (top & (top - 1u)) != 0u || nt > 1)) {
          nt = __popc(top);
#pragma unroll
          for (int o = LPS / 2; o >= 1; o >>= 1) nt += __shfl_xor_sync(0xffffffffu, nt, o);
        }
      } else {
#pragma unroll
        for (int e = 0; e < E; e += 2) {
          x[e] = ex2_approx(x[e] - m);
          x[e + 1] = ex2_approx(x[e + 1] - m);
          s0 += x[e];
          s1 += x[e + 1];
        }
      }
      float r = s0 + s1;
#pragma unroll
      for (int o = LPS / 2; o >= 1; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
      const float s = EXACT ? static_cast<float>(nt) + r : r;
      const float w = j < nloc ? hw * rcp_approx(s) : 0.f;
      // every lane of a group holds its sample's m and s: lane l takes the
      // logden of sample l from the group that holds it in this exchange step
      // logden_p = (x_rp + m + log2 s) ln 2, x_rp = c_r - b'_r phi_p (0 in the absolute form)
      const float xr = rel ? fmaf(-bhr, ph, chr) + lor : 0.f;
      const float lv = (xr + (m + __log2f(s))) * kLn2;
      const float lv_l = __shfl_sync(0xffffffffu, lv, ((lane - j0) & (SPW - 1)) * LPS);
      if (lane >= j0 && lane < j0 + SPW) ld_mine = lv_l;
#pragma unroll
      for (int e = 0; e < E; ++e) acc[e] = fmaf(x[e], w, acc[e]);
      if (EXACT && top != 0u && w != 0.f) {
        const float add = nt == 1 ? -r * w : w;
        do {
          const int e = __ffs(top) - 1;
          top &= top - 1u;
          const int k = 4 * (lig + LPS * (e >> 2)) + (e & 3);
          if constexpr (LPS == 32) {
            // this lane is the only writer of the row entry of state k
            float2 c = myrow[k];
            if (nt == 1) {
              const float sum1 = c.x + hw, b1 = sum1 - c.x;
              c.y += (c.x - (sum1 - b1)) + (hw - b1);
              c.x = sum1;
            }
            const float sum2 = c.x + add, bv = sum2 - c.x;
            c.y += (c.x - (sum2 - bv)) + (add - bv);
            c.x = sum2;
            myrow[k] = c;
          } else {
            if (nt == 1) atomicAdd(&cnt[warp * Kp + k], static_cast<unsigned>(hw));
#pragma unroll
            for (int q = 0; q < E; ++q)
              if (q == e) acc[q] += add;
          }
        } while (top != 0u);
      }
      if (++since >= kFactFlush) {
        fold();
        since = 0;
      }
    }
    // one coalesced store of the chunk's logden (FP64 built with integer
    // operations: a conversion per sample on the FP64 pipe stalled the warp)
    if (p.logden != nullptr && lane < nloc) static_cast<double*>(p.logden)[base + lane] = f32_to_f64_bits(ld_mine);
  }
  fold();

  // ---- per-CTA row sums: the warps' partials in warp order ----
  __syncthreads();
  double* out = p.partials + static_cast<size_t>(blockIdx.x) * K;
  for (int k = tid; k < K; k += NT) {
    double t = 0.0;
    for (int w = 0; w < NW; ++w) {
      const float2 c = rows[static_cast<size_t>(w) * Kp + k];
      t += static_cast<double>(c.x) + static_cast<double>(c.y);
      if constexpr (EXACT && LPS < 32) t += static_cast<double>(cnt[static_cast<size_t>(w) * Kp + k]);
    }
    out[k] = t;
  }
}

namespace {

template <int LPS, int NK, int NT, bool EXACT>
void fact_run_one(const LsePlan& pl, const double* a, const double* b, const double* phi, int Kp, const FactRef* ref,
                  const LseParams& prm, cudaStream_t st) {
  static bool init = false;
  {
    std::lock_guard<std::recursive_mutex> lock(init_mutex());
    if (!init) {
      // the device maximum once, so every K of this instantiation fits
      int dev = 0, optin = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      cudaFuncSetAttribute(lse_fact_kernel<LPS, NK, NT, EXACT>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
      init = true;
    }
  }
  lse_fact_kernel<LPS, NK, NT, EXACT><<<pl.grid, NT, pl.smem, st>>>(a, b, phi, Kp, ref, prm);
}

template <int LPS, int NK, int NT>
void fact_run(const LsePlan& pl, const double* a, const double* b, const double* phi, int Kp, const FactRef* ref,
              const LseParams& prm, cudaStream_t st) {
  if (prm.exact_max) fact_run_one<LPS, NK, NT, true>(pl, a, b, phi, Kp, ref, prm, st);
  else fact_run_one<LPS, NK, NT, false>(pl, a, b, phi, Kp, ref, prm, st);
}

}  // namespace

// Threads of the compiled factorised instance with `nk` chunks per lane:
// four FP32 constants per state in registers, 512 threads (128 registers)
// up to 12 states per lane, 384 at 16 (512 spilled), 256 beyond.
int fact_threads(int nk) { return nk <= 3 ? 512 : (nk == 4 ? 384 : 256); }

LsePlan lse_fact_plan(int64_t K, int64_t n) {
  int lps = 0, nk = 0, nt = 0, unused = 0;
  if (tuned_shape(kTuneFactorised, K, n, &lps, &nk, &nt, &unused)) return lse_fact_plan_for(K, n, lps, nk);
  return lse_fact_plan_rule(K, n);
}

LsePlan lse_fact_plan_rule(int64_t K, int64_t n) {
  int lps = 0, nk = 0;
  // lanes per sample: as few as give every lane at most 16 states (four
  // float4 groups), so the per-sample shuffles, reciprocal and logden write
  // are spread over as many entries as the registers allow; 32 lanes (and up
  // to 32 states each) from K = 256
  const int64_t q = round_up(K, 4) / 4;
  lps = 1;
  while (lps < 32 && lps * 4 < q) lps <<= 1;
  nk = static_cast<int>(ceil_div(q, static_cast<int64_t>(lps)));
  if (lps < 32 && nk == 3) nk = 4;
  return lse_fact_plan_for(K, n, lps, nk);
}

LsePlan lse_fact_plan_for(int64_t K, int64_t n, int lps, int nk) {
  LsePlan pl{};
  const int nt = fact_threads(nk);
  const int64_t Kp = round_up(K, 4);
  pl.variant = 3;
  pl.threads = nt;
  pl.J = nk;
  pl.H = lps;
  pl.C = 32;
  pl.num_strips = static_cast<int>(ceil_div(n, 32));
  // + the per-warp counts of the exact split below 32 lanes per sample
  pl.smem = static_cast<size_t>(Kp) * 16 + static_cast<size_t>(nt / 32) * Kp * (lps < 32 ? 12 : 8) +
            static_cast<size_t>(kRefGrid) * sizeof(int16_t);
  pl.ok = K >= 1 && K <= 1024;
  // every warp of every CTA gets at least one chunk where n allows
  pl.grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(ceil_div(pl.num_strips, nt / 32), num_sms())));
  return pl;
}

size_t lse_fact_ref_bytes() {
  return round_up(static_cast<int64_t>(sizeof(FactRef)), 256) + 2 * kRangeParts * sizeof(double);
}

mbar_status lse_fact_launch(const double* a, const double* b, const double* phi, const LsePlan& pl, LseParams prm,
                            const double* phi_min, const double* phi_max, int nparts, void* ref_buf,
                            cudaStream_t st) {
  if (!pl.ok) {
    set_error("factorised lse pass: unsupported K=%d", prm.K);
    return MBAR_EUNSUPPORTED;
  }
  if (!ref_buf || (reinterpret_cast<uintptr_t>(ref_buf) & 15) != 0) {
    set_error("factorised lse pass: the reference-table buffer must be 16-byte aligned");
    return MBAR_EINVAL;
  }
  FactRef* ref = static_cast<FactRef*>(ref_buf);
  {
    // a pass its guard skips still builds the table (it only reads f)
    if (!phi_min) {
      double* mins = reinterpret_cast<double*>(static_cast<unsigned char*>(ref_buf) +
                                               round_up(static_cast<int64_t>(sizeof(FactRef)), 256));
      double* maxs = mins + kRangeParts;
      const int g = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(kRangeParts, ceil_div(prm.n, 4096))));
      fact_range_kernel<<<g, kRefThreads, 0, st>>>(phi, prm.n, mins, maxs);
      phi_min = mins;
      phi_max = maxs;
      nparts = g;
      count_launches(1);
    }
    fact_ref_kernel<<<kRefGrid / kRefThreads, kRefThreads, 0, st>>>(a, b, prm.f, prm.logN, prm.K, phi_min, phi_max,
                                                                     nparts, ref);
    count_launches(1);
  }
  prm.nparts = pl.grid;
  prm.epi = prm.partials + static_cast<size_t>(pl.grid) * prm.K;
  const int Kp = static_cast<int>(round_up(prm.K, 4));
  const int lps = pl.H, nk = pl.J;
  // the instances the shape rule reaches: one lane per sample with 1, 2 or
  // 4 chunks; 2..16 lanes with 4 chunks; 32 lanes with 3..8 chunks
  bool ok = true;
  if (lps == 1 && nk == 1) fact_run<1, 1, 512>(pl, a, b, phi, Kp, ref, prm, st);
  else if (lps == 1 && nk == 2) fact_run<1, 2, 512>(pl, a, b, phi, Kp, ref, prm, st);
  else if (lps == 1 && nk == 4) fact_run<1, 4, 384>(pl, a, b, phi, Kp, ref, prm, st);
  else if (lps == 2 && nk == 4) fact_run<2, 4, 384>(pl, a, b, phi, Kp, ref, prm, st);
  else if (lps == 4 && nk == 4) fact_run<4, 4, 384>(pl, a, b, phi, Kp, ref, prm, st);
  else if (lps == 8 && nk == 4) fact_run<8, 4, 384>(pl, a, b, phi, Kp, ref, prm, st);
  else if (lps == 16 && nk == 4) fact_run<16, 4, 384>(pl, a, b, phi, Kp, ref, prm, st);
  else if (lps == 32) {
    switch (nk) {
      case 3: fact_run<32, 3, 512>(pl, a, b, phi, Kp, ref, prm, st); break;
      case 4: fact_run<32, 4, 384>(pl, a, b, phi, Kp, ref, prm, st); break;
      case 5: fact_run<32, 5, 256>(pl, a, b, phi, Kp, ref, prm, st); break;
      case 6: fact_run<32, 6, 256>(pl, a, b, phi, Kp, ref, prm, st); break;
      case 7: fact_run<32, 7, 256>(pl, a, b, phi, Kp, ref, prm, st); break;
      case 8: fact_run<32, 8, 256>(pl, a, b, phi, Kp, ref, prm, st); break;
      default: ok = false;
    }
  } else {
    ok = false;
  }
  if (!ok) {
    set_error("lse_fact_launch: unsupported shape (%d lanes, %d chunks)", lps, nk);
    return MBAR_EUNSUPPORTED;
  }
  count_launches(1);
  BUMBAR_CUDA(cudaGetLastError());
  return lse_epilogue_launch(prm, st);
}

}  // namespace bumbar
