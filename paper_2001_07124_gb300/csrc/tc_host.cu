// Host-side helpers shared by the tensor-core kernels: TMA tensor-map encoding
// through the driver entry point, and the SM count used to size persistent grids.
#include <cuda_runtime.h>

#include <atomic>

#include "tc_common.cuh"

namespace rhosvd {
namespace tc {

namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Looked up once per process; the initialisation of a function-local static
// is thread-safe, so concurrent first calls all see the finished lookup.
EncodeTiledFn encode_fn() {
  static const EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeTiledFn>(p);
    return static_cast<EncodeTiledFn>(nullptr);
  }();
  return fn;
}

}  // namespace

bool make_tmap_f32(CUtensorMap* m, const float* base, int rank, const uint64_t* dims, const uint64_t* strides,
                   const uint32_t* box, CUtensorMapSwizzle sw) {
  EncodeTiledFn fn = encode_fn();
  if (fn == nullptr || rank < 1 || rank > 3) return false;
  cuuint64_t d[3], g[2];
  cuuint32_t b[3], e[3] = {1, 1, 1};
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    b[i] = box[i];
    if (dims[i] == 0 || box[i] == 0 || box[i] > 256) return false;
  }
  for (int i = 0; i + 1 < rank; ++i) {
    if (strides[i] % 4 != 0) return false;
    g[i] = strides[i] * sizeof(float);
  }
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<float*>(base), d, g, b, e,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_tmap_u(CUtensorMap* m, const void* base, int elem_bytes, int rank, const uint64_t* dims,
                 const uint64_t* strides, const uint32_t* box, CUtensorMapSwizzle sw) {
  EncodeTiledFn fn = encode_fn();
  if (fn == nullptr || rank < 1 || rank > 3 || (elem_bytes != 1 && elem_bytes != 2)) return false;
  cuuint64_t d[3], g[2];
  cuuint32_t b[3], e[3] = {1, 1, 1};
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    b[i] = box[i];
    if (dims[i] == 0 || box[i] == 0 || box[i] > 256) return false;
  }
  if ((box[0] * (uint32_t)elem_bytes) % 16 != 0) return false;        // inner box extent: 16-byte multiple
  for (int i = 0; i + 1 < rank; ++i) {
    g[i] = strides[i] * (uint64_t)elem_bytes;
    if (g[i] % 16 != 0) return false;
  }
  const CUtensorMapDataType t = elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8;
  return fn(m, t, (cuuint32_t)rank, const_cast<void*>(base), d, g, b, e, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// SM count of the current device, cached per device (atomics: any host thread
// may be first to ask).
int device_sms() {
  constexpr int kMaxDev = 64;
  static std::atomic<int> cache[kMaxDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  const bool cached = dev >= 0 && dev < kMaxDev;
  int n = cached ? cache[dev].load(std::memory_order_relaxed) : 0;
  if (n > 0) return n;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
  if (cached) cache[dev].store(n, std::memory_order_relaxed);
  return n;
}

}  // namespace tc
}  // namespace rhosvd
