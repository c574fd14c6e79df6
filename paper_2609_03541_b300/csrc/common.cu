// Host-side helpers: error strings, device properties, tensor-map encoding.
#include <cudaTypedefs.h>

#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "common.cuh"

namespace bumbar {

static thread_local char g_last_error[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
}

const char* last_error() { return g_last_error; }

mbar_status cuda_status(cudaError_t e, const char* where) {
  set_error("CUDA error %d (%s) in %s", static_cast<int>(e), cudaGetErrorString(e), where);
  if (e == cudaErrorMemoryAllocation) return MBAR_ENOMEM;
  return MBAR_ECUDA;
}

static std::atomic<int64_t> g_launches{0};
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

int num_sms() {
  static const int sms = [] {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
  }();
  return sms;
}

std::recursive_mutex& init_mutex() {
  static std::recursive_mutex m;
  return m;
}

static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

mbar_status make_tmap_2d(CUtensorMap* map, const void* base, CUtensorMapDataType dtype, int elem_bytes,
                         int64_t rows, int64_t cols, int64_t ld, int box_cols, int box_rows) {
  return make_tmap_2d_swz(map, base, dtype, elem_bytes, rows, cols, ld, box_cols, box_rows, true);
}

mbar_status make_tmap_2d_swz(CUtensorMap* map, const void* base, CUtensorMapDataType dtype, int elem_bytes,
                             int64_t rows, int64_t cols, int64_t ld, int box_cols, int box_rows, bool swizzle128) {
  auto encode = get_encode();
  if (!encode) {
    set_error("cuTensorMapEncodeTiled unavailable from the driver");
    return MBAR_ECUDA;
  }
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (ld * elem_bytes) % 16 != 0) {
    set_error("tensor map: base must be 16-byte aligned and the row pitch a multiple of 16 bytes");
    return MBAR_EINVAL;
  }
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld * elem_bytes)};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(box_cols), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(map, dtype, 2, const_cast<void*>(base), dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d): rows=%lld cols=%lld ld=%lld box=%dx%d", static_cast<int>(r),
              static_cast<long long>(rows), static_cast<long long>(cols), static_cast<long long>(ld), box_cols,
              box_rows);
    return MBAR_ECUDA;
  }
  return MBAR_OK;
}

}  // namespace bumbar
