// Gram matrix G = A^T A of a tall column-major matrix A (m x K, leading
// dimension ld), reduced to FP64: the "small Gram" of CholeskyQR2 (the orthonormal
// basis of Alg. 1) and of the truncation (B B^T, the SVD of B in Alg. 1).
//
// Only the upper triangle a <= b is accumulated (K(K+1)/2 pairs per row); each
// CTA owns a contiguous block of rows, stages 64-row tiles in shared memory and
// writes its partial K x K Gram (both triangles) in FP64; partials are summed in
// a fixed order (reduce_d_kernel), so results are bitwise reproducible.
//
// Two accumulation modes:
//  * EXACT: every product a*b is split exactly by an FMA (TwoProd) and added
//    with TwoSum into a double-float accumulator (Ogita, Rump, Oishi 2005,
//    "Accurate sum and dot product"), so the Gram is FP64-accurate even when
//    cond(A) is ~1e6 (first CholeskyQR pass).  Up to K = 64 it runs
//    register-blocked (gram_dw_kernel, 2 x 2 column-pair blocks).
//  * CHUNKED: products are summed in FP32 over four 64-row tiles and those sums
//    are added in FP64; enough when A is close to orthonormal (second pass).
//    Register-blocked: a thread owns a 4 x 4 block of column pairs and reads
//    the tile as float4 row quads, 2 shared loads per 16 FMAs per row.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace rhosvd {
namespace {

constexpr int GR_THREADS = 256;
constexpr int GR_TILE = 64;                      // rows per shared-memory tile
constexpr int GR_TARGET_CTAS = 296;              // 2 per SM on 148-152 SMs

template <bool EXACT, int PT>                    // PT = max pairs per thread
__global__ void __launch_bounds__(GR_THREADS)
gram_kernel(const float* __restrict__ A, int64_t m, int K, int64_t ld, int64_t rows_per_cta,
            double* __restrict__ part) {
  extern __shared__ float tile[];                // [K][GR_TILE + 1]
  const int tid = threadIdx.x;
  const int P = K * (K + 1) / 2;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r1 = min(m, r0 + rows_per_cta);
  constexpr int LD = GR_TILE + 1;

  int pab[PT];                                    // a | b << 16
  double dacc[PT];
  df64 xacc[PT];
#pragma unroll
  for (int t = 0; t < PT; ++t) {
    const int p = tid + t * GR_THREADS;
    int b = (int)((sqrtf(8.f * (float)p + 1.f) - 1.f) * 0.5f);
    while (b > 0 && b * (b + 1) / 2 > p) --b;
    while ((b + 1) * (b + 2) / 2 <= p) ++b;
    pab[t] = (p < P) ? ((p - b * (b + 1) / 2) | (b << 16)) : 0;
    dacc[t] = 0.0;
    xacc[t] = df64{0.f, 0.f};
  }
  for (int64_t rt = r0; rt < r1; rt += GR_TILE) {
    const int nrow = (r1 - rt < GR_TILE) ? (int)(r1 - rt) : GR_TILE;
    __syncthreads();
        for (int e = tid; e < K * GR_TILE; e += GR_THREADS) {
      const int c = e / GR_TILE, r = e % GR_TILE;
      tile[c * LD + r] = (r < nrow) ? __ldg(A + (rt + r) + (int64_t)c * ld) : 0.f;
    }
    __syncthreads();
    const int nr8 = (nrow + 7) & ~7;              // rows past nrow are zero in the tile
#pragma unroll
    for (int t = 0; t < PT; ++t) {
      if (tid + t * GR_THREADS >= P) break;
      const float* ca = tile + (pab[t] & 0xffff) * LD;
      const float* cb = tile + (pab[t] >> 16) * LD;
      if (EXACT) {
        df64 acc = xacc[t];
        if (nrow == GR_TILE) {                      // full tile: compile-time trip count
#pragma unroll 8
          for (int r = 0; r < GR_TILE; ++r) df64_fma(acc, ca[r], cb[r]);
        } else {
#pragma unroll 8
          for (int r = 0; r < nr8; ++r) df64_fma(acc, ca[r], cb[r]);
        }
        xacc[t] = acc;
      } else {
        float s = 0.f;
#pragma unroll 8
        for (int r = 0; r < nr8; ++r) s = fmaf(ca[r], cb[r], s);
        dacc[t] += (double)s;
      }
    }
  }
  double* dst = part + (int64_t)blockIdx.x * K * K;
#pragma unroll
  for (int t = 0; t < PT; ++t) {
    if (tid + t * GR_THREADS >= P) break;
    const double v = EXACT ? df64_to_double(xacc[t]) : dacc[t];
    const int a = pab[t] & 0xffff, b = pab[t] >> 16;
    dst[a + b * K] = v;
    dst[b + a * K] = v;
  }
}

// ---------------------------------------------------------------- chunked, register-blocked
constexpr int GF_LD = GR_TILE + 4;               // column pitch of the tile (== 4 mod 32)
constexpr int GF_FLUSH = 4;                      // tiles summed in FP32 before the FP64 add

__device__ __forceinline__ void pair_blocks(int p, int& bi, int& bj) {   // p -> (bi <= bj), column-major upper
  int b = (int)((sqrtf(8.f * (float)p + 1.f) - 1.f) * 0.5f);
  while (b > 0 && b * (b + 1) / 2 > p) --b;
  while ((b + 1) * (b + 2) / 2 <= p) ++b;
  bi = p - b * (b + 1) / 2;
  bj = b;
}

template <int PT>                                // block pairs per thread (npairs <= PT * GR_THREADS)
__global__ void __launch_bounds__(GR_THREADS)
gram_f32_kernel(const float* __restrict__ A, int64_t m, int K, int64_t ld, int64_t rows_per_cta,
                double* __restrict__ part) {
  extern __shared__ __align__(16) float gf_smem[];   // tile [4*nb][GF_LD]; later the phase partials
  const int tid = threadIdx.x;
  const int nb = (K + 3) / 4, npairs = nb * (nb + 1) / 2;
  const int phases = npairs >= GR_THREADS ? 1 : GR_THREADS / npairs;
  const int phase = npairs >= GR_THREADS ? 0 : tid / npairs;
  const bool active = npairs >= GR_THREADS ? true : tid < phases * npairs;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r1 = min(m, r0 + rows_per_cta);

  int bi[PT], bj[PT];
  bool own[PT];
  float acc[PT][16];
  double dacc[PT][16];
#pragma unroll
  for (int t = 0; t < PT; ++t) {
    const int p = (npairs >= GR_THREADS) ? tid + t * GR_THREADS : (t == 0 ? tid % npairs : npairs);
    own[t] = active && p < npairs;
    pair_blocks(own[t] ? p : 0, bi[t], bj[t]);
#pragma unroll
    for (int e = 0; e < 16; ++e) { acc[t][e] = 0.f; dacc[t][e] = 0.0; }
  }
  int ntile = 0;
  for (int64_t rt = r0; rt < r1; rt += GR_TILE, ++ntile) {
    const int nrow = (r1 - rt < GR_TILE) ? (int)(r1 - rt) : GR_TILE;
    __syncthreads();
#pragma unroll 8
    for (int e = tid; e < 4 * nb * GR_TILE; e += GR_THREADS) {
      const int c = e / GR_TILE, r = e % GR_TILE;
      gf_smem[c * GF_LD + r] = (r < nrow && c < K) ? __ldg(A + (rt + r) + (int64_t)c * ld) : 0.f;
    }
    __syncthreads();
    for (int q = phase; q < GR_TILE / 4; q += phases) {
#pragma unroll
      for (int t = 0; t < PT; ++t) {
        if (!own[t]) continue;
        float4 a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          a[u] = *reinterpret_cast<const float4*>(gf_smem + (4 * bi[t] + u) * GF_LD + 4 * q);
          b[u] = *reinterpret_cast<const float4*>(gf_smem + (4 * bj[t] + u) * GF_LD + 4 * q);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            float x = acc[t][4 * u + v];
            x = fmaf(a[u].x, b[v].x, x);
            x = fmaf(a[u].y, b[v].y, x);
            x = fmaf(a[u].z, b[v].z, x);
            x = fmaf(a[u].w, b[v].w, x);
            acc[t][4 * u + v] = x;
          }
      }
    }
    if ((ntile + 1) % GF_FLUSH == 0) {
#pragma unroll
      for (int t = 0; t < PT; ++t)
#pragma unroll
        for (int e = 0; e < 16; ++e) { dacc[t][e] += (double)acc[t][e]; acc[t][e] = 0.f; }
    }
  }
#pragma unroll
  for (int t = 0; t < PT; ++t)
#pragma unroll
    for (int e = 0; e < 16; ++e) dacc[t][e] += (double)acc[t][e];
  double* dst = part + (int64_t)blockIdx.x * K * K;
  if (phases == 1) {
#pragma unroll
    for (int t = 0; t < PT; ++t) {
      if (!own[t]) continue;
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int a = 4 * bi[t] + e / 4, b = 4 * bj[t] + e % 4;
        if (a < K && b < K) { dst[a + b * K] = dacc[t][e]; dst[b + a * K] = dacc[t][e]; }
      }
    }
    return;
  }
  // several row phases per pair block: sum them in a fixed order through shared memory
  __syncthreads();
  double* red = reinterpret_cast<double*>(gf_smem);   // [phase][pair][16]
  if (own[0])
#pragma unroll
    for (int e = 0; e < 16; ++e) red[((size_t)phase * npairs + tid % npairs) * 16 + e] = dacc[0][e];
  __syncthreads();
  for (int w = tid; w < npairs * 16; w += GR_THREADS) {
    const int p = w / 16, e = w % 16;
    double v = 0.0;
    for (int ph = 0; ph < phases; ++ph) v += red[((size_t)ph * npairs + p) * 16 + e];
    int pi, pj;
    pair_blocks(p, pi, pj);
    const int a = 4 * pi + e / 4, b = 4 * pj + e % 4;
    if (a < K && b < K) { dst[a + b * K] = v; dst[b + a * K] = v; }
  }
}

// ---------------------------------------------------------------- double-float, register-blocked
// The EXACT accumulation of gram_kernel with a thread owning a 2 x 2 block of
// column pairs: per row quad it reads 4 float4 (two columns of each side) for
// 16 double-float multiply-adds, where the scalar form reads two floats per
// multiply-add; the threads take the row quads of a tile in phases when the
// block pairs are fewer.  The 64-row tiles are double-buffered: cp.async copies the next
// tile in while the current one is used.  Each CTA's partial Gram is the sum
// over its rows in row order per accumulator (deterministic).
constexpr int GD_LD = GR_TILE + 4;               // column pitch of a tile (== 4 mod 32)
constexpr int GD_THREADS = 512;                  // two CTAs per SM (256 threads measured the same)

__device__ __forceinline__ void gd_cp_async(float* dst, const float* src, bool valid) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}

// start copying rows rt..rt+nrow-1 of A (all 2 nb columns, zeros past K and nrow)
__device__ __forceinline__ void gd_stage(const float* A, int64_t rt, int nrow, int K, int ncol, int64_t ld,
                                         float* tile) {
  for (int e = threadIdx.x; e < ncol * GR_TILE; e += GD_THREADS) {
    const int c = e / GR_TILE, r = e - c * GR_TILE;
    const bool ok = r < nrow && c < K;
    gd_cp_async(tile + c * GD_LD + r, ok ? A + (rt + r) + (int64_t)c * ld : A, ok);
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int PT>                                // block pairs per thread (npairs <= PT * GD_THREADS)
__global__ void __launch_bounds__(GD_THREADS, 2)
gram_dw_kernel(const float* __restrict__ A, int64_t m, int K, int64_t ld, int64_t rows_per_cta,
               double* __restrict__ part) {
  extern __shared__ __align__(16) float gd_smem[];   // two tiles [2 nb][GD_LD]; later the phase partials
  const int tid = threadIdx.x;
  const int nb = (K + 1) / 2, npairs = nb * (nb + 1) / 2, ncol = 2 * nb;
  const int phases = npairs >= GD_THREADS ? 1 : GD_THREADS / npairs;
  const int phase = npairs >= GD_THREADS ? 0 : tid / npairs;
  const bool active = npairs >= GD_THREADS ? true : tid < phases * npairs;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r1 = min(m, r0 + rows_per_cta);
  const int tile_floats = ncol * GD_LD;

  int bi[PT], bj[PT];
  bool own[PT];
  df64 acc[PT][4];
#pragma unroll
  for (int t = 0; t < PT; ++t) {
    const int p = (npairs >= GD_THREADS) ? tid + t * GD_THREADS : (t == 0 ? tid % npairs : npairs);
    own[t] = active && p < npairs;
    pair_blocks(own[t] ? p : 0, bi[t], bj[t]);
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[t][e] = df64{0.f, 0.f};
  }
  const int ntiles = r1 > r0 ? (int)((r1 - r0 + GR_TILE - 1) / GR_TILE) : 0;
  if (ntiles > 0) gd_stage(A, r0, (int)(r1 - r0 < GR_TILE ? r1 - r0 : GR_TILE), K, ncol, ld, gd_smem);
  for (int it = 0; it < ntiles; ++it) {
    const int64_t rt = r0 + (int64_t)it * GR_TILE;
    const int nrow = (r1 - rt < GR_TILE) ? (int)(r1 - rt) : GR_TILE;
    const float* tile = gd_smem + (it & 1) * tile_floats;
    if (it + 1 < ntiles) {
      const int64_t rn = rt + GR_TILE;
      gd_stage(A, rn, (int)(r1 - rn < GR_TILE ? r1 - rn : GR_TILE), K, ncol, ld, gd_smem + ((it + 1) & 1) * tile_floats);
    } else {
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    __syncthreads();
    const int nq = (nrow + 3) / 4;               // rows past nrow are zero in the tile
    for (int q = phase; q < nq; q += phases) {
#pragma unroll
      for (int t = 0; t < PT; ++t) {
        if (!own[t]) continue;
        const float4 a0 = *reinterpret_cast<const float4*>(tile + (2 * bi[t]) * GD_LD + 4 * q);
        const float4 a1 = *reinterpret_cast<const float4*>(tile + (2 * bi[t] + 1) * GD_LD + 4 * q);
        const float4 b0 = *reinterpret_cast<const float4*>(tile + (2 * bj[t]) * GD_LD + 4 * q);
        const float4 b1 = *reinterpret_cast<const float4*>(tile + (2 * bj[t] + 1) * GD_LD + 4 * q);
        df64_fma(acc[t][0], a0.x, b0.x);
        df64_fma(acc[t][1], a0.x, b1.x);
        df64_fma(acc[t][2], a1.x, b0.x);
        df64_fma(acc[t][3], a1.x, b1.x);
        df64_fma(acc[t][0], a0.y, b0.y);
        df64_fma(acc[t][1], a0.y, b1.y);
        df64_fma(acc[t][2], a1.y, b0.y);
        df64_fma(acc[t][3], a1.y, b1.y);
        df64_fma(acc[t][0], a0.z, b0.z);
        df64_fma(acc[t][1], a0.z, b1.z);
        df64_fma(acc[t][2], a1.z, b0.z);
        df64_fma(acc[t][3], a1.z, b1.z);
        df64_fma(acc[t][0], a0.w, b0.w);
        df64_fma(acc[t][1], a0.w, b1.w);
        df64_fma(acc[t][2], a1.w, b0.w);
        df64_fma(acc[t][3], a1.w, b1.w);
      }
    }
    __syncthreads();                             // the tile may be refilled
  }
  double* dst = part + (int64_t)blockIdx.x * K * K;
  if (phases == 1) {
#pragma unroll
    for (int t = 0; t < PT; ++t) {
      if (!own[t]) continue;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int a = 2 * bi[t] + e / 2, b = 2 * bj[t] + e % 2;
        const double v = df64_to_double(acc[t][e]);
        if (a < K && b < K) { dst[a + b * K] = v; dst[b + a * K] = v; }
      }
    }
    return;
  }
  // several row phases per pair block: sum them in a fixed order through shared memory
  double* red = reinterpret_cast<double*>(gd_smem);   // [phase][pair][4]
  if (own[0])
#pragma unroll
    for (int e = 0; e < 4; ++e) red[((size_t)phase * npairs + tid % npairs) * 4 + e] = df64_to_double(acc[0][e]);
  __syncthreads();
  for (int w = tid; w < npairs * 4; w += GD_THREADS) {
    const int p = w / 4, e = w % 4;
    double v = 0.0;
    for (int ph = 0; ph < phases; ++ph) v += red[((size_t)ph * npairs + p) * 4 + e];
    int pi, pj;
    pair_blocks(p, pi, pj);
    const int a = 2 * pi + e / 2, b = 2 * pj + e % 2;
    if (a < K && b < K) { dst[a + b * K] = v; dst[b + a * K] = v; }
  }
}

cudaError_t launch_gram_dw(const float* A, int64_t m, int K, int64_t ld, double* G, double* part, int ctas,
                           int64_t rows, cudaStream_t st) {
  const int nb = (K + 1) / 2, npairs = nb * (nb + 1) / 2;
  const int phases = npairs >= GD_THREADS ? 1 : GD_THREADS / npairs;
  const size_t tiles = (size_t)2 * (2 * nb) * GD_LD * sizeof(float);
  const size_t red = phases > 1 ? (size_t)phases * npairs * 4 * sizeof(double) : 0;
  const size_t smem = tiles > red ? tiles : red;
  cudaError_t e;
  if (npairs <= GD_THREADS) {
    if ((e = allow_dynamic_smem((const void*)gram_dw_kernel<1>, smem)) != cudaSuccess) return e;
    gram_dw_kernel<1><<<ctas, GD_THREADS, smem, st>>>(A, m, K, ld, rows, part);
  } else if (npairs <= 2 * GD_THREADS) {
    if ((e = allow_dynamic_smem((const void*)gram_dw_kernel<2>, smem)) != cudaSuccess) return e;
    gram_dw_kernel<2><<<ctas, GD_THREADS, smem, st>>>(A, m, K, ld, rows, part);
  } else {
    if ((e = allow_dynamic_smem((const void*)gram_dw_kernel<3>, smem)) != cudaSuccess) return e;
    gram_dw_kernel<3><<<ctas, GD_THREADS, smem, st>>>(A, m, K, ld, rows, part);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return launch_reduce_d(part, ctas, (int64_t)K * K, G, st);
}

cudaError_t launch_gram_f32(const float* A, int64_t m, int K, int64_t ld, double* G, double* part, int ctas,
                            int64_t rows, cudaStream_t st) {
  const int nb = (K + 3) / 4, npairs = nb * (nb + 1) / 2;
  const int phases = npairs >= GR_THREADS ? 1 : GR_THREADS / npairs;
  const size_t tile = (size_t)4 * nb * GF_LD * sizeof(float);
  const size_t red = phases > 1 ? (size_t)phases * npairs * 16 * sizeof(double) : 0;   // <= 32 KB
  const size_t smem = tile > red ? tile : red;
  cudaError_t e;
  if (npairs <= GR_THREADS) {
    if ((e = allow_dynamic_smem((const void*)gram_f32_kernel<1>, 64 * 1024)) != cudaSuccess) return e;
    gram_f32_kernel<1><<<ctas, GR_THREADS, smem, st>>>(A, m, K, ld, rows, part);
  } else if (npairs <= 2 * GR_THREADS) {
    if ((e = allow_dynamic_smem((const void*)gram_f32_kernel<2>, 64 * 1024)) != cudaSuccess) return e;
    gram_f32_kernel<2><<<ctas, GR_THREADS, smem, st>>>(A, m, K, ld, rows, part);
  } else {
    if ((e = allow_dynamic_smem((const void*)gram_f32_kernel<3>, 64 * 1024)) != cudaSuccess) return e;
    gram_f32_kernel<3><<<ctas, GR_THREADS, smem, st>>>(A, m, K, ld, rows, part);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return launch_reduce_d(part, ctas, (int64_t)K * K, G, st);
}

template <bool EXACT>
cudaError_t launch_gram_t(const float* A, int64_t m, int K, int64_t ld, double* G, double* part, int ctas,
                          int64_t rows, cudaStream_t st) {
  const int P = K * (K + 1) / 2;
  const int pt = (P + GR_THREADS - 1) / GR_THREADS;
  const size_t smem = (size_t)K * (GR_TILE + 1) * sizeof(float);
  if (pt <= 4) gram_kernel<EXACT, 4><<<ctas, GR_THREADS, smem, st>>>(A, m, K, ld, rows, part);
  else if (pt <= 8) gram_kernel<EXACT, 8><<<ctas, GR_THREADS, smem, st>>>(A, m, K, ld, rows, part);
  else if (pt <= 16) gram_kernel<EXACT, 16><<<ctas, GR_THREADS, smem, st>>>(A, m, K, ld, rows, part);
  else gram_kernel<EXACT, 33><<<ctas, GR_THREADS, smem, st>>>(A, m, K, ld, rows, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_reduce_d(part, ctas, (int64_t)K * K, G, st);
}

}  // namespace

GramPlan plan_gram(int64_t m, int K, bool exact) {
  GramPlan pl;
  // enough rows per CTA that the pair bookkeeping amortises, at most ~2 CTAs per SM;
  // the double-float path, whose cost is its arithmetic, goes down to 16-row
  // CTAs on short matrices (a 512-row basis is then spread over 32 SMs, not 8)
  const int64_t step = (exact && m < (int64_t)GR_TARGET_CTAS * GR_TILE) ? 16 : GR_TILE;
  int64_t rows = (m + GR_TARGET_CTAS - 1) / GR_TARGET_CTAS;
  rows = std::max<int64_t>(step, ((rows + step - 1) / step) * step);
  pl.rows_per_cta = rows;
  pl.ctas = (int)std::max<int64_t>(1, (m + rows - 1) / rows);
  (void)K;
  return pl;
}

cudaError_t launch_gram(const float* A, int64_t m, int K, int64_t ld, double* G, double* part, bool exact,
                        cudaStream_t st) {
  GramPlan pl = plan_gram(m, K, exact);
  if (!exact) return launch_gram_f32(A, m, K, ld, G, part, pl.ctas, pl.rows_per_cta, st);
  // register-blocked double-float form up to K = 64 (at most three block pairs per thread)
  if (K <= 64) return launch_gram_dw(A, m, K, ld, G, part, pl.ctas, pl.rows_per_cta, st);
  return launch_gram_t<true>(A, m, K, ld, G, part, pl.ctas, pl.rows_per_cta, st);
}

}  // namespace rhosvd
