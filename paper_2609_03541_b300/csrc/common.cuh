// Shared device/host helpers of the BU-MBAR library (sm_103a).
#pragma once

#include <mutex>

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bumbar.h"

namespace bumbar {

constexpr int kThreads = 256;           // CTA size of the streaming kernels
constexpr float kLog2e = 1.4426950408889634f;
// log2(e) - kLog2e: with it, v log2(e) = v kLog2e + v kLog2eLo carries no
// systematic relative error of 1.3e-8 (which, multiplied by energies of
// hundreds of kT, would bias free energies at the 1e-5 kT level)
constexpr float kLog2eLo = static_cast<float>(1.4426950408889634 - static_cast<double>(kLog2e));
constexpr float kLn2 = 0.6931471805599453f;

// ---------------------------------------------------------------------------
// error plumbing (host)
// ---------------------------------------------------------------------------
void set_error(const char* fmt, ...);
mbar_status cuda_status(cudaError_t e, const char* where);

#define BUMBAR_CUDA(call)                                              \
  do {                                                                 \
    cudaError_t _e = (call);                                           \
    if (_e != cudaSuccess) return ::bumbar::cuda_status(_e, #call);    \
  } while (0)

#define BUMBAR_TRY(call)                                               \
  do {                                                                 \
    mbar_status _s = (call);                                           \
    if (_s != MBAR_OK) return _s;                                      \
  } while (0)

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
inline int64_t ceil_div(int64_t x, int64_t m) { return (x + m - 1) / m; }

int num_sms();

// Process-wide count of kernels launched by this library.
// Guards the one-time caches (occupancy, shared-memory limits, plans) that
// concurrent solves on several host threads may fill at the same time.
std::recursive_mutex& init_mutex();
void count_launches(int n);
int64_t launches_so_far();

// ---------------------------------------------------------------------------
// device helpers: mbarrier + TMA (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase. Gives up after ~max_spins polls and
// returns false (the caller records a timeout and stops cleanly).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t max_spins) {
  for (uint32_t i = 0; i < max_spins; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
  }
  return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// 1-D bulk copy global -> shared memory (both 16-byte aligned, bytes a
// multiple of 16), completion on `bar` (complete_tx).
__device__ __forceinline__ void bulk_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 2-D tiled TMA load of one box into shared memory, completion on `bar`.
// Coordinates: c0 = innermost (column) element index, c1 = row index.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
      : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// 2^x on the SFU (MUFU.EX2), flushing denormal results to zero.
// 1/x to within 1 ulp, denormals flushed (callers pass sums whose largest
// term is 1); the IEEE division takes about ten instructions
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// max over the 32 lanes of the warp in one instruction (NaN inputs ignored)
__device__ __forceinline__ float warp_max_f32(float v) {
  float r;
  asm volatile("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
  return r;
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Two FP32 values in one 64-bit register for the f32x2 instructions of
// sm_100-family GPUs: one issue slot does the add or FMA of both halves,
// each rounded exactly as the scalar instruction would round it.
__device__ __forceinline__ unsigned long long pk2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk2(unsigned long long v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// Byte offset of 16-byte chunk `chunk` of 128-byte row `row` inside a tile
// written by TMA with CU_TENSOR_MAP_SWIZZLE_128B (tile base 1024-aligned):
// chunk index is XORed with row % 8.
__device__ __forceinline__ uint32_t swz128(uint32_t row, uint32_t chunk) {
  return row * 128u + ((chunk ^ (row & 7u)) << 4);
}

// ---------------------------------------------------------------------------
// host: tensor-map encoding through the driver entry point
// ---------------------------------------------------------------------------
// Encodes a 2-D row-major tensor (rows x cols, row pitch `ld` elements) with
// a box of (box_cols x box_rows) elements and 128-byte swizzle.
mbar_status make_tmap_2d(CUtensorMap* map, const void* base, CUtensorMapDataType dtype, int elem_bytes,
                         int64_t rows, int64_t cols, int64_t ld, int box_cols, int box_rows);
// The same with the 128-byte swizzle optional (false: boxes land in shared
// memory as plain row-major tiles; inner extent up to 256 elements).
mbar_status make_tmap_2d_swz(CUtensorMap* map, const void* base, CUtensorMapDataType dtype, int elem_bytes,
                             int64_t rows, int64_t cols, int64_t ld, int box_cols, int box_rows, bool swizzle128);

// Splits a binary64 x into hi = RN32(x) and lo = RN32(x - hi) with integer
// operations only: the residual is (dropped 29 fraction bits - the rounding
// increment) x 2^(E - 1075), formed as an int -> float conversion and a
// power-of-two scale. False when hi or the scale would leave the normal
// binary32 range (the caller then uses FP64 arithmetic).
__device__ __forceinline__ bool split_f64(double x, float& hi, float& lo) {
  const unsigned long long d = static_cast<unsigned long long>(__double_as_longlong(x));
  const unsigned int dh = static_cast<unsigned int>(d >> 32), dl = static_cast<unsigned int>(d);
  const int E = static_cast<int>((dh >> 20) & 0x7FFu);
  const int e = E - 1023 + 127;
  const int s = E - 1075;  // weight of the last binary64 fraction bit
  if (e <= 0 || e >= 254 || s < -126) return false;
  const unsigned int sign = dh & 0x80000000u;
  const unsigned int mant = ((dh & 0xFFFFFu) << 3) | (dl >> 29);
  const unsigned int rest = dl & 0x1FFFFFFFu;
  const unsigned int half = 0x10000000u;
  const unsigned int up = (rest > half || (rest == half && (mant & 1u))) ? 1u : 0u;
  hi = __uint_as_float(sign | (((static_cast<unsigned int>(e) << 23) | mant) + up));
  const int r = static_cast<int>(rest) - (up ? (1 << 29) : 0);
  const float scale = __uint_as_float(static_cast<unsigned int>(s + 127) << 23);
  lo = __uint_as_float(sign ^ __float_as_uint(__int2float_rn(r) * scale));
  return true;
}

// binary32 -> binary64 with integer operations only (exact: widen the
// exponent, shift the fraction); subnormal inputs take the hardware
// conversion, which runs on the FP64 pipe.
__device__ __forceinline__ double f32_to_f64_bits(float x) {
  const unsigned int u = __float_as_uint(x);
  const unsigned int sign = u & 0x80000000u, e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  unsigned int hi;
  if (e == 0u) {
    if (m != 0u) return static_cast<double>(x);
    hi = sign;  // +-0
  } else if (e == 0xFFu) {
    hi = sign | 0x7FF00000u | (m >> 3);  // inf / nan
  } else {
    hi = sign | ((e + 896u) << 20) | (m >> 3);
  }
  const unsigned long long bits = (static_cast<unsigned long long>(hi) << 32) | (static_cast<unsigned long long>(m) << 29);
  return __longlong_as_double(static_cast<long long>(bits));
}

}  // namespace bumbar
