// Tensor-core (tcgen05) mode-1 sketch Y = X_(1) W for an X whose first mode
// is contiguous (L = 1): Y(i,k) = sum_j X[i + I*j] W[j + J*k] (Alg. 1 step 2,
// Alg. 6 line 3, Alg. 9 line 1 for n = 1; the dominant pass of R-STHOSVD).
//
// The contraction over j is split over CTAs (one CTA per SM, persistent); each
// CTA owns up to 512 rows i (four 128-row MMA tiles) and a contiguous range of
// j, and writes its partial I x K block for the fixed-order reducer.
//
// Data path per 16-column block of j (two MMA K steps of kind::tf32):
//   * TMA copies the X tile (16 x 512 FP32, two 256-wide boxes) and the raw W
//     tile (16 x 64) into a 4-stage shared-memory ring (producer warp 8).
//   * Eight transform warps (two warpgroups; warp w owns TMEM lane quadrant
//     w % 4, warpgroup g the 128-row tiles 2g and 2g+1) read X rows from
//     shared memory, split every value into TF32 hi + lo (3xTF32) and store
//     both into tensor memory as the A operand (tcgen05.st), so the skinny
//     N <= 64 GEMM never re-reads A from shared memory; they also split the W
//     tile into hi/lo B tiles in the canonical no-swizzle K-major layout.
//   * One thread of warp 9 issues, per 128-row tile and K step, the three MMAs
//     A_hi*B_hi + A_hi*B_lo + A_lo*B_hi into FP32 accumulators in TMEM.
//   * At the end the transform warps read the accumulators (tcgen05.ld) and
//     write the partial sums.
// Requirements (checked by the launcher, which otherwise declines): I % 4 == 0,
// J % 4 == 0 (TMA strides), K <= 64.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace rhosvd {
namespace {

using namespace tc;

constexpr int BJ = 16;                    // j per stage (two tf32 MMA K steps of 8)
constexpr int X_STAGES = 5;
constexpr int A_STAGES = 2;
constexpr int ROWS = 512;                 // rows i per CTA (4 MMA tiles)
constexpr int BOXW = 256;                 // TMA box width in i
constexpr int NUM_XFORM = 256;            // warps 0-7
constexpr int NUM_THREADS = NUM_XFORM + 64;   // + warp 8 producer, warp 9 MMA issuer
constexpr uint32_t TMEM_COLS = 512;
constexpr int D_COLS = 64;                // accumulator columns reserved per tile
constexpr int A_COL0 = 4 * D_COLS;        // first TMEM column of the A stages
constexpr int A_STAGE_COLS = 128;         // per stage: 4 tiles x (16 hi + 16 lo)
constexpr int B_TILE = 64 * BJ;           // floats per B tile (N <= 64)

struct __align__(1024) SketchSmem {
  float x[X_STAGES][ROWS / BOXW][BJ * BOXW];   // TMA boxes: [box][jj][256]
  float wraw[X_STAGES][B_TILE];                // TMA box [n][jj], rows n >= K are zero-filled
  float b[A_STAGES][2][B_TILE];                // hi / lo B tiles, canonical K-major layout
  uint64_t full_x[X_STAGES], empty_x[X_STAGES];
  uint64_t full_a[A_STAGES], empty_a[A_STAGES];
  uint64_t done;
  uint32_t tmem_base;
  int abort_flag;
};

// B tiles (N x 16 K elements, K-major, no swizzle): element (n, kk) sits at
// byte (n >> 3) * 512 + (kk >> 2) * 128 + (n & 7) * 16 + (kk & 3) * 4, i.e.
// 8-row x 16-byte core matrices with LBO = 128 (K direction) and SBO = 512
// (N direction); the second MMA K step starts 256 bytes in.

template <int NPAD>
__global__ void __launch_bounds__(NUM_THREADS, 1)
tc_sketch_m1_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmW, int I,
                    int64_t J, int K, int64_t jchunk, float* __restrict__ part, DevStatus* st) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  SketchSmem& sm = *reinterpret_cast<SketchSmem*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int split = blockIdx.x;
  const int i0 = blockIdx.y * ROWS;
  const int rows = min(ROWS, I - i0);
  const int mt = (rows + 127) / 128;                 // MMA tiles in this CTA
  const int nbox = (rows + BOXW - 1) / BOXW;
  const int64_t jb = (int64_t)split * jchunk;
  const int64_t je = min(J, jb + jchunk);
  const int nkb = (int)((je - jb + BJ - 1) / BJ);
  constexpr uint32_t idesc = idesc_tf32(128, NPAD);

  if (tid == 0) {
    for (int s = 0; s < X_STAGES; ++s) {
      mbar_init(&sm.full_x[s], 1);
      mbar_init(&sm.empty_x[s], NUM_XFORM);
    }
    for (int a = 0; a < A_STAGES; ++a) {
      mbar_init(&sm.full_a[a], NUM_XFORM);
      mbar_init(&sm.empty_a[a], 1);
    }
    mbar_init(&sm.done, 1);
    sm.abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == 9) {
    tmem_alloc(&sm.tmem_base, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm.tmem_base;
  volatile int* abort_flag = &sm.abort_flag;
  bool ok = true;

  if (warp == 8) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      const uint32_t bytes = (uint32_t)(nbox * BJ * BOXW * 4 + B_TILE * 4);
      for (int kb = 0; kb < nkb && ok; ++kb) {
        const int s = kb % X_STAGES;
        const uint32_t ph = (uint32_t)(kb / X_STAGES) & 1u;
        if (!mbar_wait(&sm.empty_x[s], ph ^ 1u, abort_flag)) { ok = false; break; }
        mbar_arrive_expect_tx(&sm.full_x[s], bytes);
        const int jt = (int)(jb + (int64_t)kb * BJ);
        for (int bx = 0; bx < nbox; ++bx) tma_load_2d(sm.x[s][bx], &tmX, i0 + bx * BOXW, jt, &sm.full_x[s]);
        tma_load_2d(sm.wraw[s], &tmW, jt, 0, &sm.full_x[s]);
      }
    }
  } else if (warp == 9) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      for (int kb = 0; kb < nkb && ok; ++kb) {
        const int a = kb % A_STAGES;
        const uint32_t ph = (uint32_t)(kb / A_STAGES) & 1u;
        if (!mbar_wait(&sm.full_a[a], ph, abort_flag)) { ok = false; break; }
        tc_fence_after();
        const uint32_t bhi = smem_u32(sm.b[a][0]), blo = smem_u32(sm.b[a][1]);
        for (int t = 0; t < mt; ++t) {
          const uint32_t d = tmem + (uint32_t)(t * D_COLS);
          const uint32_t ahi = tmem + (uint32_t)(A_COL0 + a * A_STAGE_COLS + t * 32);
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            const uint64_t dbh = smem_desc_kmajor_nosw(bhi + ks * 256, 128, 512);
            const uint64_t dbl = smem_desc_kmajor_nosw(blo + ks * 256, 128, 512);
            mma_tf32_ts(d, ahi + ks * 8, dbh, idesc, (kb > 0 || ks > 0) ? 1u : 0u);
            mma_tf32_ts(d, ahi + ks * 8, dbl, idesc, 1u);
            mma_tf32_ts(d, ahi + 16 + ks * 8, dbh, idesc, 1u);
          }
        }
        mma_commit(&sm.empty_a[a]);
      }
      mma_commit(&sm.done);
    }
  } else {
    // ------------------------------------------------------------ transform (warps 0-7)
    const int quad = warp & 3, wg = warp >> 2;
    const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
    const int row_in_tile = quad * 32 + lane;
    for (int kb = 0; kb < nkb && ok; ++kb) {
      const int s = kb % X_STAGES, a = kb % A_STAGES;
      const uint32_t phx = (uint32_t)(kb / X_STAGES) & 1u, pha = (uint32_t)(kb / A_STAGES) & 1u;
      const int64_t rem = je - (jb + (int64_t)kb * BJ);
      const int valid = rem < BJ ? (int)rem : BJ;
      if (!mbar_wait(&sm.full_x[s], phx, abort_flag)) { ok = false; break; }
      if (!mbar_wait(&sm.empty_a[a], pha ^ 1u, abort_flag)) { ok = false; break; }
      tc_fence_after();
#pragma unroll
      for (int tt = 0; tt < 2; ++tt) {
        const int t = 2 * wg + tt;
        if (t < mt) {
          const int r = t * 128 + row_in_tile;       // row within the CTA's block
          const float* xb = sm.x[s][r / BOXW] + (r % BOXW);
          uint32_t hi[16], lo[16];
#pragma unroll
          for (int jj = 0; jj < BJ; ++jj) {
            const float v = (jj < valid && r < rows) ? xb[jj * BOXW] : 0.f;
            split_tf32(v, hi[jj], lo[jj]);
          }
          const uint32_t col = tmem + (uint32_t)(A_COL0 + a * A_STAGE_COLS + t * 32);
          tmem_st_x16(col + lane_base, hi);
          tmem_st_x16(col + 16 + lane_base, lo);
        }
      }
      // B tiles: element (n, jj) of W, split into hi / lo.  Threads walk the
      // canonical layout word by word (conflict-free stores): word w holds
      // n = 8 (w >> 7) + ((w >> 2) & 7), jj = 4 ((w >> 5) & 3) + (w & 3).
#pragma unroll
      for (int u = 0; u < NPAD * BJ / NUM_XFORM; ++u) {
        const int w = tid + u * NUM_XFORM;
        const int n = 8 * (w >> 7) + ((w >> 2) & 7), jj = 4 * ((w >> 5) & 3) + (w & 3);
        const float v = (jj < valid && n < K) ? sm.wraw[s][n * BJ + jj] : 0.f;
        uint32_t h, l;
        split_tf32(v, h, l);
        reinterpret_cast<uint32_t*>(sm.b[a][0])[w] = h;
        reinterpret_cast<uint32_t*>(sm.b[a][1])[w] = l;
      }
      fence_proxy_async_smem();
      tmem_wait_st();
      tc_fence_before();
      mbar_arrive(&sm.full_a[a]);
      mbar_arrive(&sm.empty_x[s]);
    }
    // ------------------------------------------------------------ epilogue
    if (ok && nkb > 0) ok = mbar_wait(&sm.done, 0, abort_flag);
    if (ok) {
      tc_fence_after();
#pragma unroll
      for (int tt = 0; tt < 2; ++tt) {
        const int t = 2 * wg + tt;
        if (t >= mt) continue;
        const int64_t i = i0 + t * 128 + row_in_tile;
#pragma unroll
        for (int c0 = 0; c0 < NPAD; c0 += 16) {
          uint32_t v[16];
          tmem_ld_x16(tmem + lane_base + (uint32_t)(t * D_COLS + c0), v);
          tmem_wait_ld();
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            const int k = c0 + c;
            if (k < K && i < I) part[((int64_t)split * K + k) * I + i] = (nkb > 0) ? __uint_as_float(v[c]) : 0.f;
          }
        }
      }
    }
  }
  if (!ok) {
    *abort_flag = 1;
    set_error(st, RHOSVD_ETIMEOUT);
  }
  // teardown: every role is past its last wait (all waits are bounded); let
  // in-flight MMAs drain before TMEM is released
  __syncthreads();
  if (warp == 9) {
    if (sm.abort_flag && lane == 0) {
      const uint64_t t0 = globaltimer_ns();
      while (!mbar_try_wait(&sm.done, 0) && globaltimer_ns() - t0 < kWaitLimitNs) {
      }
    }
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// ---------------------------------------------------------------- host side
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2-D FP32 tensor map: inner dimension contiguous, outer stride in elements.
bool make_tmap_2d(CUtensorMap* m, const float* base, uint64_t inner, uint64_t outer, uint64_t outer_stride,
                  uint32_t box_inner, uint32_t box_outer) {
  EncodeTiledFn fn = encode_fn();
  if (fn == nullptr) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {outer_stride * sizeof(float)};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

}  // namespace

bool tc_sketch_supported(const View& x, const WView& w, int K) {
  if (x.L != 1 || x.s_i != 1 || x.s_r != x.I) return false;           // mode-1 layout
  const int64_t J = x.Rt;
  if (w.w_r != 1 || w.w_k != J) return false;                          // W is J x K, ld J
  if (K < 1 || K > 64 || x.I % 4 != 0 || J % 4 != 0 || x.I > (int64_t(1) << 30)) return false;
  if ((reinterpret_cast<uintptr_t>(x.p) & 15) || (reinterpret_cast<uintptr_t>(w.p) & 15)) return false;
  return J >= 1024 && encode_fn() != nullptr;
}

TcSketchPlan plan_tc_sketch(int64_t I, int K, int64_t J) {
  TcSketchPlan pl;
  pl.mgroups = (int)((I + ROWS - 1) / ROWS);
  int64_t splits = std::max<int64_t>(1, num_sms() / pl.mgroups);
  int64_t chunk = (J + splits - 1) / splits;
  chunk = ((chunk + BJ - 1) / BJ) * BJ;
  pl.jchunk = chunk;
  pl.splits = (int)((J + chunk - 1) / chunk);
  (void)K;
  return pl;
}

cudaError_t launch_tc_sketch(const View& x, const WView& w, int K, float* Y, int64_t ldy, float* part,
                             DevStatus* st, cudaStream_t stream) {
  const int64_t I = x.I, J = x.Rt;
  TcSketchPlan pl = plan_tc_sketch(I, K, J);
  CUtensorMap tmX, tmW;
  if (!make_tmap_2d(&tmX, x.p, (uint64_t)I, (uint64_t)J, (uint64_t)I, BOXW, BJ)) return cudaErrorNotSupported;
  if (!make_tmap_2d(&tmW, w.p, (uint64_t)J, (uint64_t)K, (uint64_t)J, BJ, 64)) return cudaErrorNotSupported;
  const size_t smem = sizeof(SketchSmem) + 1024;
  const dim3 grid((unsigned)pl.splits, (unsigned)pl.mgroups);
  cudaError_t e;
  const int npad = ((K + 15) / 16) * 16;
  switch (npad) {
    case 16:
      if ((e = allow_dynamic_smem((const void*)tc_sketch_m1_kernel<16>, smem)) != cudaSuccess) return e;
      tc_sketch_m1_kernel<16><<<grid, NUM_THREADS, smem, stream>>>(tmX, tmW, (int)I, J, K, pl.jchunk, part, st);
      break;
    case 32:
      if ((e = allow_dynamic_smem((const void*)tc_sketch_m1_kernel<32>, smem)) != cudaSuccess) return e;
      tc_sketch_m1_kernel<32><<<grid, NUM_THREADS, smem, stream>>>(tmX, tmW, (int)I, J, K, pl.jchunk, part, st);
      break;
    case 48:
      if ((e = allow_dynamic_smem((const void*)tc_sketch_m1_kernel<48>, smem)) != cudaSuccess) return e;
      tc_sketch_m1_kernel<48><<<grid, NUM_THREADS, smem, stream>>>(tmX, tmW, (int)I, J, K, pl.jchunk, part, st);
      break;
    default:
      if ((e = allow_dynamic_smem((const void*)tc_sketch_m1_kernel<64>, smem)) != cudaSuccess) return e;
      tc_sketch_m1_kernel<64><<<grid, NUM_THREADS, smem, stream>>>(tmX, tmW, (int)I, J, K, pl.jchunk, part, st);
      break;
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return launch_reduce_partials_f(part, pl.splits, I, K, Y, ldy, stream);
}

}  // namespace rhosvd
