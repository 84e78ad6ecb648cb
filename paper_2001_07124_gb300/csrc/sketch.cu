// SIMT contraction kernels on strided unfoldings (Sec. 2):
//   sketch  Y(i,k) = sum_j X_(n)(i,j) W(j,k)   (the sketches of Alg. 1, Alg. 6
//           and Alg. 9; also the Gram A^T A of a tall matrix)
//   ttm     T(j,k) = sum_i X_(n)(i,j) M(i,k)    (n-mode product, power step
//           Z = X_(n)^T Q, projection B = Q^T X_(n), core chain, Y <- Y R^-1)
// The unfolding is never materialised: column j = l + L*r of X_(n) is read at
// X[l + i*s_i + r*s_r].  The sketch splits the long contraction j over CTAs
// and reduces the per-CTA partials in a fixed order (deterministic results).
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace rhosvd {

namespace {

constexpr int SK_BJ = 16;    // contraction step
constexpr int SK_THREADS = 256;
constexpr int TARGET_CTAS = 608;   // 4 CTAs per SM on 152 SMs

template <bool DF>
struct Acc;
template <>
struct Acc<false> {
  float v = 0.f;
  __device__ __forceinline__ void fma(float a, float b) { v = fmaf(a, b, v); }
  __device__ __forceinline__ float out() const { return v; }
};
template <>
struct Acc<true> {
  df64 v{0.f, 0.f};
  __device__ __forceinline__ void fma(float a, float b) { df64_fma(v, a, b); }
  __device__ __forceinline__ double out() const { return df64_to_double(v); }
};

// Output tile of 16 TU x 16 TU per CTA (TU values per thread in each dimension):
// TU = 4 in general, TU = 2 when I and K are both at most 64, where one 64 x 64
// tile would leave the GPU idle and spend its (double-float) multiply-adds on
// padding.
template <bool DF, typename OutT, int TU>
__global__ void __launch_bounds__(SK_THREADS)
sketch_partial_kernel(View x, WView w, int K, int64_t jchunk, OutT* __restrict__ part) {
  constexpr int SK_BI = 16 * TU, SK_BK = 16 * TU;
  __shared__ float Xs[SK_BJ][SK_BI + 1];
  __shared__ float Ws[SK_BJ][SK_BK + 1];
  __shared__ int64_t xoff[SK_BJ];
  __shared__ int64_t woff[SK_BJ];

  const int tid = threadIdx.x;
  const int64_t J = x.L * x.Rt;
  const int64_t i0 = (int64_t)blockIdx.x * SK_BI;
  const int k0 = blockIdx.y * SK_BK;
  const int64_t jb = (int64_t)blockIdx.z * jchunk;
  const int64_t je = min(J, jb + jchunk);
  const int tx = tid & 15, ty = tid >> 4;
  const bool x_i_fast = (x.s_i == 1);
  const bool w_k_fast = (w.w_k == 1);

  Acc<DF> acc[TU][TU];

  for (int64_t jt = jb; jt < je; jt += SK_BJ) {
    if (tid < SK_BJ) {
      int64_t j = jt + tid;
      if (j < je) {
        int64_t r = j / x.L, l = j - r * x.L;
        xoff[tid] = l + r * x.s_r;
        woff[tid] = l + r * w.w_r;
      } else {
        xoff[tid] = -1;
        woff[tid] = -1;
      }
    }
    __syncthreads();
    for (int e = tid; e < SK_BJ * SK_BI; e += SK_THREADS) {
      int jj, ii;
      if (x_i_fast) { ii = e % SK_BI; jj = e / SK_BI; } else { jj = e % SK_BJ; ii = e / SK_BJ; }
      const int64_t i = i0 + ii;
      const int64_t off = xoff[jj];
      Xs[jj][ii] = (off >= 0 && i < x.I) ? __ldg(x.p + off + i * x.s_i) : 0.f;
    }
    for (int e = tid; e < SK_BJ * SK_BK; e += SK_THREADS) {
      int jj, kk;
      if (w_k_fast) { kk = e % SK_BK; jj = e / SK_BK; } else { jj = e % SK_BJ; kk = e / SK_BJ; }
      const int k = k0 + kk;
      const int64_t off = woff[jj];
      Ws[jj][kk] = (off >= 0 && k < K) ? __ldg(w.p + off + (int64_t)k * w.w_k) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int jj = 0; jj < SK_BJ; ++jj) {
      float a[TU], b[TU];
#pragma unroll
      for (int u = 0; u < TU; ++u) {
        a[u] = Xs[jj][tx + 16 * u];
        b[u] = Ws[jj][ty + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < TU; ++u)
#pragma unroll
        for (int v = 0; v < TU; ++v) acc[u][v].fma(a[u], b[v]);
    }
    __syncthreads();
  }
  OutT* dst = part + (int64_t)blockIdx.z * x.I * K;
#pragma unroll
  for (int u = 0; u < TU; ++u) {
    const int64_t i = i0 + tx + 16 * u;
#pragma unroll
    for (int v = 0; v < TU; ++v) {
      const int k = k0 + ty + 16 * v;
      if (i < x.I && k < K) dst[(int64_t)k * x.I + i] = (OutT)acc[u][v].out();
    }
  }
}

// Fixed-order reduction over splits: out(e) = sum_s part[s*n + e].  A CTA
// owns 32 consecutive outputs; its 8 warps each sum every 8th split for those
// outputs, then the 8 partial sums are added in warp order.  The order depends
// only on (splits, n), so results are bitwise reproducible.
constexpr int RD_ROWS = 8;
template <typename T, typename OutT>
__global__ void __launch_bounds__(32 * RD_ROWS)
reduce_partials_kernel(const T* __restrict__ part, int splits, int64_t I, int K, OutT* __restrict__ y,
                       int64_t ldy) {
  __shared__ T acc[RD_ROWS][32];
  const int lane = threadIdx.x & 31, row = threadIdx.x >> 5;
  const int64_t n = I * K;
  const int64_t e = (int64_t)blockIdx.x * 32 + lane;
  T s = 0;
  if (e < n)
#pragma unroll 4
    for (int t = row; t < splits; t += RD_ROWS) s += part[(int64_t)t * n + e];
  acc[row][lane] = s;
  __syncthreads();
  if (row == 0 && e < n) {
    T tot = acc[0][lane];
#pragma unroll
    for (int r = 1; r < RD_ROWS; ++r) tot += acc[r][lane];
    const int64_t k = e / I, i = e - k * I;
    y[i + k * ldy] = (OutT)tot;
  }
}

__global__ void __launch_bounds__(32 * RD_ROWS)
reduce_d_kernel(const double* __restrict__ part, int splits, int64_t n, double* __restrict__ out) {
  __shared__ double acc[RD_ROWS][32];
  const int lane = threadIdx.x & 31, row = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * 32 + lane;
  double s = 0;
  if (e < n)
#pragma unroll 4
    for (int t = row; t < splits; t += RD_ROWS) s += part[(int64_t)t * n + e];
  acc[row][lane] = s;
  __syncthreads();
  if (row == 0 && e < n) {
    double tot = acc[0][lane];
#pragma unroll
    for (int r = 1; r < RD_ROWS; ++r) tot += acc[r][lane];
    out[e] = tot;
  }
}

// ---------------------------------------------------------------- TTM
constexpr int TT_MAX_BJ = 128;
constexpr int TT_BI = 16;
constexpr int TT_THREADS = 256;

template <int UJ, int KT>   // rows per CTA = 16*UJ, output columns per CTA = 16*KT
__global__ void __launch_bounds__(TT_THREADS)
ttm_kernel(View x, const float* __restrict__ M, int64_t m_i, int64_t m_k, int K, OView out,
           const DevStatus* skip) {
  if (skip != nullptr && skip->orth_fail) return;
  constexpr int BK = 16 * KT;
  constexpr int TT_BJ = 16 * UJ;
  __shared__ float Xs[TT_BI][TT_BJ + 1];
  __shared__ float Ms[TT_BI][BK + 1];
  __shared__ int64_t xoff[TT_BJ];
  __shared__ int64_t ooff[TT_BJ];

  const int tid = threadIdx.x;
  const int64_t J = x.L * x.Rt;
  const int64_t j0 = (int64_t)blockIdx.x * TT_BJ;
  const int k0 = blockIdx.y * BK;
  const int tj = tid & 15, tk = tid >> 4;

  if (tid < TT_BJ) {
    const int64_t j = j0 + tid;
    if (j < J) {
      const int64_t r = j / x.L, l = j - r * x.L;
      const int64_t oL = out.o_L > 0 ? out.o_L : x.L;
      const int64_t ro = j / oL;
      xoff[tid] = l + r * x.s_r;
      ooff[tid] = (j - ro * oL) + ro * out.o_r;
    } else {
      xoff[tid] = -1;
      ooff[tid] = -1;
    }
  }
  __syncthreads();

  float acc[UJ][KT];
#pragma unroll
  for (int u = 0; u < UJ; ++u)
#pragma unroll
    for (int v = 0; v < KT; ++v) acc[u][v] = 0.f;

  const bool x_i_fast = (x.s_i == 1);
  const bool m_i_fast = (m_i == 1);
  for (int64_t it = 0; it < x.I; it += TT_BI) {
    for (int e = tid; e < TT_BI * TT_BJ; e += TT_THREADS) {
      int ii, jj;
      if (x_i_fast) { ii = e % TT_BI; jj = e / TT_BI; } else { jj = e % TT_BJ; ii = e / TT_BJ; }
      const int64_t i = it + ii;
      const int64_t off = xoff[jj];
      Xs[ii][jj] = (off >= 0 && i < x.I) ? x.p[off + i * x.s_i] : 0.f;
    }
    for (int e = tid; e < TT_BI * BK; e += TT_THREADS) {
      int ii, kk;
      if (m_i_fast) { ii = e % TT_BI; kk = e / TT_BI; } else { kk = e % BK; ii = e / BK; }
      const int64_t i = it + ii;
      const int k = k0 + kk;
      Ms[ii][kk] = (i < x.I && k < K) ? __ldg(M + i * m_i + (int64_t)k * m_k) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int ii = 0; ii < TT_BI; ++ii) {
      float a[UJ], b[KT];
#pragma unroll
      for (int u = 0; u < UJ; ++u) a[u] = Xs[ii][tj + 16 * u];
#pragma unroll
      for (int v = 0; v < KT; ++v) b[v] = Ms[ii][tk + 16 * v];
#pragma unroll
      for (int u = 0; u < UJ; ++u)
#pragma unroll
        for (int v = 0; v < KT; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < UJ; ++u) {
    const int64_t off = ooff[tj + 16 * u];
    if (off < 0) continue;
#pragma unroll
    for (int v = 0; v < KT; ++v) {
      const int k = k0 + tk + 16 * v;
      if (k < K) out.p[off + (int64_t)k * out.o_k] = acc[u][v];
    }
  }
}

template <bool DF, typename OutT>
void launch_partials(const SketchPlan& pl, const View& x, const WView& w, int K, OutT* part, cudaStream_t st) {
  const dim3 grid(pl.tiles_i, pl.tiles_k, pl.splits);
  if (pl.tu == 2)
    sketch_partial_kernel<DF, OutT, 2><<<grid, SK_THREADS, 0, st>>>(x, w, K, pl.jchunk, part);
  else
    sketch_partial_kernel<DF, OutT, 4><<<grid, SK_THREADS, 0, st>>>(x, w, K, pl.jchunk, part);
}

}  // namespace

cudaError_t allow_dynamic_smem(const void* kernel, size_t bytes) {
  // The largest limit set so far per (device, kernel) pair; the attribute is
  // raised whenever a launch needs more (a kernel whose shared memory depends
  // on its arguments asks for different sizes).  The table is shared by every
  // host thread, so it is read and written under a lock.
  constexpr int kMaxDev = 64, kMaxKern = 64;
  static std::mutex mu;
  static const void* kernels[kMaxKern] = {nullptr};
  static size_t set_bytes[kMaxKern][kMaxDev] = {{0}};
  static int nk = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  int slot = -1;
  for (int i = 0; i < nk; ++i)
    if (kernels[i] == kernel) slot = i;
  if (slot < 0 && nk < kMaxKern) {
    slot = nk++;
    kernels[slot] = kernel;
  }
  if (slot >= 0 && dev < kMaxDev && set_bytes[slot][dev] >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess && slot >= 0 && dev < kMaxDev) set_bytes[slot][dev] = bytes;
  return e;
}

SketchPlan plan_sketch(int64_t I, int K, int64_t J) {
  SketchPlan pl;
  pl.tu = (I <= 64 && K <= 64) ? 2 : 4;         // small outputs: four times the CTAs, less padding
  const int tile = 16 * pl.tu;
  pl.tiles_i = (int)((I + tile - 1) / tile);
  pl.tiles_k = (K + tile - 1) / tile;
  const int64_t tiles = (int64_t)pl.tiles_i * pl.tiles_k;
  int64_t want = std::max<int64_t>(1, TARGET_CTAS / std::max<int64_t>(1, tiles));
  int64_t chunk = (J + want - 1) / want;
  chunk = ((chunk + SK_BJ - 1) / SK_BJ) * SK_BJ;
  chunk = std::max<int64_t>(chunk, (J > 4096 ? 4 : 1) * SK_BJ);   // short contractions: one step per CTA
  pl.jchunk = chunk;
  pl.splits = (int)std::max<int64_t>(1, (J + chunk - 1) / chunk);
  return pl;
}

size_t sketch_partial_floats(const SketchPlan& pl, int64_t I, int K) {
  return (size_t)pl.splits * (size_t)I * (size_t)K;
}

cudaError_t launch_sketch(const View& x, const WView& w, int K, float* Y, int64_t ldy, float* ws_part,
                          cudaStream_t st) {
  const int64_t J = x.L * x.Rt;
  SketchPlan pl = plan_sketch(x.I, K, J);
  launch_partials<false, float>(pl, x, w, K, ws_part, st);
  const int64_t n = x.I * K;
  reduce_partials_kernel<float, float><<<(unsigned)((n + 31) / 32), 32 * RD_ROWS, 0, st>>>(
      ws_part, pl.splits, x.I, K, Y, ldy);
  return cudaGetLastError();
}

cudaError_t launch_reduce_partials_f(const float* part, int splits, int64_t I, int K, float* Y, int64_t ldy,
                                     cudaStream_t st) {
  const int64_t n = I * K;
  reduce_partials_kernel<float, float><<<(unsigned)((n + 31) / 32), 32 * RD_ROWS, 0, st>>>(part, splits, I, K, Y,
                                                                                          ldy);
  return cudaGetLastError();
}

size_t sketch_scratch_floats(int64_t I, int K, int64_t J) {
  const size_t simt = sketch_partial_floats(plan_sketch(I, K, J), I, K);
  const TcSketchPlan tp = plan_tc_sketch(I, K, J);
  return std::max(simt, (size_t)tp.splits * (size_t)I * (size_t)K);
}

cudaError_t launch_sketch_auto(const View& x, const WView& w, int K, float* Y, int64_t ldy, float* part,
                               DevStatus* st, cudaStream_t stream) {
  if (st != nullptr && tc_sketch_supported(x, w, K)) {
    cudaError_t e = launch_tc_sketch(x, w, K, Y, ldy, part, st, stream);
    if (e != cudaErrorNotSupported) return e;
  }
  return launch_sketch(x, w, K, Y, ldy, part, stream);
}

cudaError_t launch_ttm_auto(const View& x, const float* Mp, int64_t m_i, int64_t m_k, int K, const OView& out,
                            const DevStatus* skip, DevStatus* st, cudaStream_t stream) {
  if (st != nullptr && tc_ttm_supported(x, m_i, m_k, K, out)) {
    cudaError_t e = launch_tc_ttm(x, Mp, m_k, K, out, skip, st, stream);
    if (e != cudaErrorNotSupported) return e;
  }
  return launch_ttm(x, Mp, m_i, m_k, K, out, skip, stream);
}

cudaError_t launch_sketch_capped(const View& x, const WView& w, int K, float* Y, int64_t ldy, float* part,
                                 int max_splits, cudaStream_t st) {
  const int64_t J = x.L * x.Rt;
  SketchPlan pl = plan_sketch(x.I, K, J);
  if (pl.splits > max_splits) {
    // widen the per-CTA contraction chunk until the partial sums fit
    int64_t chunk = (J + max_splits - 1) / max_splits;
    pl.jchunk = ((chunk + SK_BJ - 1) / SK_BJ) * SK_BJ;
    pl.splits = (int)std::max<int64_t>(1, (J + pl.jchunk - 1) / pl.jchunk);
  }
  launch_partials<false, float>(pl, x, w, K, part, st);
  const int64_t n = x.I * K;
  reduce_partials_kernel<float, float><<<(unsigned)((n + 31) / 32), 32 * RD_ROWS, 0, st>>>(
      part, pl.splits, x.I, K, Y, ldy);
  return cudaGetLastError();
}

cudaError_t launch_sketch_df(const View& x, const WView& w, int K, double* Gd, int64_t ldg,
                             double* ws_part, cudaStream_t st) {
  const int64_t J = x.L * x.Rt;
  SketchPlan pl = plan_sketch(x.I, K, J);
  launch_partials<true, double>(pl, x, w, K, ws_part, st);
  const int64_t n = x.I * K;
  reduce_partials_kernel<double, double><<<(unsigned)((n + 31) / 32), 32 * RD_ROWS, 0, st>>>(
      ws_part, pl.splits, x.I, K, Gd, ldg);
  return cudaGetLastError();
}

cudaError_t launch_reduce_d(const double* part, int splits, int64_t n, double* out, cudaStream_t st) {
  reduce_d_kernel<<<(unsigned)((n + 31) / 32), 32 * RD_ROWS, 0, st>>>(part, splits, n, out);
  return cudaGetLastError();
}

cudaError_t launch_ttm(const View& x, const float* Mp, int64_t m_i, int64_t m_k, int K, const OView& out,
                       const DevStatus* skip, cudaStream_t st) {
  const int64_t J = x.L * x.Rt;
  if (J == 0 || K == 0) return cudaSuccess;
  // 128-row tiles when there are enough of them to fill the GPU, 32-row tiles otherwise
  const bool wide = (J + TT_MAX_BJ - 1) / TT_MAX_BJ >= 296;
  const int bj = wide ? 128 : 32;
  const unsigned gx = (unsigned)((J + bj - 1) / bj);
  if (K <= 16) {
    if (wide) ttm_kernel<8, 1><<<dim3(gx, 1), TT_THREADS, 0, st>>>(x, Mp, m_i, m_k, K, out, skip);
    else ttm_kernel<2, 1><<<dim3(gx, 1), TT_THREADS, 0, st>>>(x, Mp, m_i, m_k, K, out, skip);
  } else if (K <= 64) {
    if (wide) ttm_kernel<8, 4><<<dim3(gx, 1), TT_THREADS, 0, st>>>(x, Mp, m_i, m_k, K, out, skip);
    else ttm_kernel<2, 4><<<dim3(gx, 1), TT_THREADS, 0, st>>>(x, Mp, m_i, m_k, K, out, skip);
  } else {
    const dim3 grid(gx, (unsigned)((K + 127) / 128));
    if (wide) ttm_kernel<8, 8><<<grid, TT_THREADS, 0, st>>>(x, Mp, m_i, m_k, K, out, skip);
    else ttm_kernel<2, 8><<<grid, TT_THREADS, 0, st>>>(x, Mp, m_i, m_k, K, out, skip);
  }
  return cudaGetLastError();
}

}  // namespace rhosvd
