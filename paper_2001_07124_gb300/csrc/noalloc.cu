// rhosvd_sketch_noalloc: the mode-n sketch Y = X_(n) Omega with its split-K
// scratch in a fixed device array instead of a caller workspace.
//
// Some callers cannot allocate device memory at the point where they need a
// sketch: code running inside another framework's memory pool that forbids
// foreign cudaMalloc calls, plug-ins that are handed only input and output
// buffers, or latency-critical loops where an allocation (and the implicit
// synchronisation cudaMalloc/cudaFree can cause) is not allowed.  For them this
// entry point keeps the partial sums in `g_sketch_scratch`, a file-scope
// __device__ array that exists once per device for as long as the library is
// loaded.  The call itself allocates nothing.
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace rhosvd {
namespace {

// Scratch for the split-K partial sums: 2^20 floats (4 MiB) per device.
constexpr int64_t kScratchFloats = int64_t(1) << 20;
static __device__ __align__(256) float g_sketch_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
float* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_sketch_scratch on the current device.  In host code the
// symbol names a host-side stand-in, not device memory, so the address has to
// be looked up once per device with that device current.
cudaError_t scratch_for_current_device(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sketch_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace rhosvd

using namespace rhosvd;

extern "C" rhosvd_status rhosvd_sketch_noalloc(const float* X, const rhosvd_shape* shape, int32_t mode,
                                               int32_t K, const float* Omega, float* Y, void* stream) {
  if (shape == nullptr || shape->N < 1 || shape->N > RHOSVD_MAX_MODES) return RHOSVD_EINVAL;
  if (X == nullptr || Omega == nullptr || Y == nullptr || mode < 0 || mode >= shape->N || K < 1 ||
      K > RHOSVD_MAX_K)
    return RHOSVD_EINVAL;
  // same shape rules as every other entry point: each size in [1, 2^40] and
  // the element count below 2^62, so that no product of sizes overflows
  int64_t L = 1, Rt = 1, tot = 1;
  for (int k = 0; k < shape->N; ++k) {
    const int64_t d = shape->dims[k];
    if (d < 1 || d > (int64_t(1) << 40)) return RHOSVD_EINVAL;
    if (tot > (int64_t(1) << 62) / d) return RHOSVD_EINVAL;
    tot *= d;
    if (k < mode) L *= d;
    if (k > mode) Rt *= d;
  }
  const int64_t I = shape->dims[mode];
  // one split needs I*K floats of scratch; larger sketches are rejected
  if (I * (int64_t)K > kScratchFloats) return RHOSVD_EINVAL;
  float* scratch = nullptr;
  if (scratch_for_current_device(&scratch) != cudaSuccess) return RHOSVD_ECUDA;
  View x;
  x.p = X;
  x.L = L;
  x.I = I;
  x.Rt = Rt;
  x.s_i = L;
  x.s_r = L * I;
  WView w{Omega, L, L * Rt};
  const int max_splits = (int)(kScratchFloats / (I * (int64_t)K));
  // every partial the reduction reads is written by this call first, so the
  // scratch needs no clearing between calls
  cudaError_t e = launch_sketch_capped(x, w, K, Y, I, scratch, max_splits, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? RHOSVD_OK : RHOSVD_ECUDA;
}
