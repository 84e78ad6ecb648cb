// Tensor-core (tcgen05) n-mode product on a strided unfolding:
//   Out(j, k) = sum_i X_(n)(i, j) M(i, k),   M(i, k) = Mp[i + ldm*k],
//   X_(n)(i, j = l + L*r) = X[l + s_i*i + s_r*r]   (Sec. 2, Eq. for the n-mode product)
// i.e. Z = X_(n)^T Q (the power-iteration TTM of Alg. 1), B^T = X_(n)^T Q
// (the projection B = Q^T X_(n) of Alg. 1) and, with X a tall matrix seen
// as L = rows, Y R^-1 (the CholeskyQR apply) and the refold Ubar^T B.
// Out(j, k) is written at Out[l + r*o_r + k*o_k] with j = l + o_L*r (o_L
// defaults to the input's L).
//
// Tile layouts of the 128 j x 32 i stage:
//   * mode 1 (L = 1, i contiguous): one 2-D box {32 i, 128 j} with 128B swizzle,
//     each j row holding 32 consecutive i;
//   * strided, L a multiple of 128 (or a single r): a 3-D box {128 l, 32 i, 1 r}
//     over [L, I, Rt], smem [i][l'], tiles of 128 consecutive j;
//   * strided, L < 128 (several r): slab tiles, a box {L l, 32 i, TR r} with
//     TR = floor(128 / L) whole r-slabs, smem [r'][i][l'], the tile's L * TR
//     rows again consecutive in j (the remaining TMEM lanes idle);
//   * strided, L > 128 not a multiple of 128 (several r): per-r tiles, see below.
// In every strided layout the 32 lanes of a warp (consecutive j) read nearly
// consecutive words for every i.
//
// Persistent, warp-specialised: each CTA takes 128-row tiles of j in turn and
// contracts over all of i in stages of 32:
//   * warp 12 (producer): TMA copies the X tile (128 rows j x 32 floats i, 128B
//     swizzle) and the raw M tile (NPAD x 32) of a stage into a 7- or 8-stage ring;
//   * warps 0-7 (two transform warpgroups, alternating stages): split X into
//     TF32 hi/lo and store it in tensor memory as the A operand (thread = row j
//     = TMEM lane), split M into hi/lo B tiles in the canonical K-major layout;
//   * warp 13 (one thread): per stage, four K steps of two MMAs (the stacked
//     3xTF32 form below) into an FP32 TMEM accumulator; every SEG stages of a
//     tile form a segment with its own accumulator buffer (buffers in turn),
//     committed when the segment's last stage is issued;
//   * warps 8-11 (epilogue): read each finished segment (tcgen05.ld), add it
//     into FP32 registers, hand the buffer back, and write the rows of Out
//     once the tile's last segment is in.
// Requirements (checked by tc_ttm_supported): 16-byte aligned X and M, strides
// multiple of 4 elements, ldm % 4 == 0, K <= 64, L % 4 == 0.  When 128
// consecutive j would straddle r with L > 128 (L not a multiple of 128, Rt > 1)
// the tiles are laid out per r: ceil(L / 128) tiles of 128 l for each r, the
// rows past L zero-filled by TMA and not written.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace rhosvd {
namespace {

using namespace tc;

constexpr int BI = 32;                    // contraction elements per stage (4 MMA K steps)
constexpr int TILE_J = 128;               // rows j per tile (one MMA M)
constexpr int A_STAGES = 2;              // one A slot per transform warpgroup
constexpr int NUM_XFORM = 256;            // warps 0-7
constexpr int NUM_EPI = 128;              // warps 8-11
constexpr int PRODUCER_WARP = 12, MMA_WARP = 13;
constexpr int NUM_THREADS = NUM_XFORM + NUM_EPI + 64;   // + the producer and MMA warps
constexpr uint32_t TMEM_COLS = 512;
constexpr int A_STAGE_COLS = 2 * BI;      // 32 hi + 32 lo columns
constexpr int A_COL0 = 0;                 // A stages first, then the accumulator buffers
constexpr int D_COL0 = A_STAGES * A_STAGE_COLS;
// The tensor core rounds its FP32 accumulation toward zero, so a long
// accumulation in tensor memory drifts toward zero by about half an ulp per
// MMA (measured -1e-5 relative over a 512^3 sketch).  Each output tile is
// therefore accumulated in tensor memory only over segments of SEG stages
// (SEG * 4 K steps, 3 MMAs each); the epilogue adds the segments in FP32
// registers with round-to-nearest, in segment order (deterministic).
constexpr int SEG = 2;

// Products in 3xTF32: X_hi M_hi + X_hi M_lo + X_lo M_hi.  The B operand of a
// stage is the stacked [M_hi; M_lo] (N = 2 NPAD rows), so each K step takes two
// MMAs, D[:, 0:2NPAD) += X_hi [M_hi M_lo] and D[:, 0:NPAD) += X_lo M_hi, and
// the product is D[:, 0:NPAD) + D[:, NPAD:2NPAD).  An accumulator buffer holds
// both halves; as many buffers as tensor memory allows (at most four) cycle
// over the segments.
template <int NPAD>
struct TtmAcc {
  static constexpr int D_COLS = 2 * NPAD;
  static constexpr int FIT = (512 - D_COL0) / D_COLS;
  static constexpr int NBUF = FIT < 4 ? FIT : 4;
};

// The M and B tiles hold NPAD rows (K padded to 16), and the X ring is as deep
// as 227 KB allows.  The pace is set by the MMA stream (12 skinny MMAs per
// stage), not by the TMA copies: the X tiles arrive before they are needed.
template <int NPAD>
struct TtmGeo {
  static constexpr int M_TILE = NPAD * BI;                  // floats per M / B tile
  static constexpr int X_STAGES = NPAD <= 48 ? 8 : 7;
};

template <int NPAD>
struct __align__(1024) TtmSmem {
  static constexpr int X_STAGES = TtmGeo<NPAD>::X_STAGES, M_TILE = TtmGeo<NPAD>::M_TILE;
  float x[X_STAGES][TILE_J * BI];          // TMA tile: mode 1 [j][i] swizzled, strided [r'][i][l']
  float mraw[X_STAGES][M_TILE];            // TMA tile [k][i] (128B swizzle), rows k >= K zero-filled
  float b[A_STAGES][2][M_TILE];            // hi / lo B tiles, canonical K-major layout
  float ostage[4][32 * 17];                // per epilogue warp: 32 rows x 16 columns (+1 pad)
  uint64_t full_x[X_STAGES], empty_x[X_STAGES];
  uint64_t full_a[A_STAGES], empty_a[A_STAGES];
  uint64_t d_full[TtmAcc<NPAD>::NBUF], d_empty[TtmAcc<NPAD>::NBUF];
  uint64_t drain;                          // arrives when every MMA this CTA issued has completed
  uint32_t tmem_base;
  int abort_flag;
};

// B tile with 32 K elements: element (n, kk) at byte (n >> 3) * 1024 +
// (kk >> 2) * 128 + (n & 7) * 16 + (kk & 3) * 4 (LBO = 128, SBO = 1024); MMA
// K step ks starts 256 * ks bytes in.  Word w of the tile holds
// n = 8 (w >> 8) + ((w >> 2) & 7), kk = 4 ((w >> 5) & 7) + (w & 3).

template <int NPAD, bool M1>
__global__ void __launch_bounds__(NUM_THREADS, 1)
tc_ttm_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmM, int I,
              int64_t L, int64_t J, int bl, int tr, int tpr, int K, float* __restrict__ out, int64_t o_k,
              int64_t o_r, int64_t o_L, const DevStatus* skip, DevStatus* st) {
  if (skip != nullptr && skip->orth_fail) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  constexpr int X_STAGES = TtmGeo<NPAD>::X_STAGES, M_TILE = TtmGeo<NPAD>::M_TILE;
  constexpr int NBUF = TtmAcc<NPAD>::NBUF, D_COLS = TtmAcc<NPAD>::D_COLS;
  TtmSmem<NPAD>& sm = *reinterpret_cast<TtmSmem<NPAD>*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // tpr > 0: tiles never straddle r (tpr tiles of 128 l per r, rows l >= L are
  // zero-filled by TMA and not written); slab tiles of tr whole r when L < 128
  // (rows = L * tr consecutive j); otherwise tiles of 128 consecutive j
  const int64_t Rt = J / L;
  const bool slab = !M1 && tpr == 0 && bl < TILE_J;   // tiles of tr whole r-slabs of L < 128 rows each
  const int ntiles = tpr > 0 ? (int)(tpr * Rt) : slab ? (int)((Rt + tr - 1) / tr) : (int)((J + TILE_J - 1) / TILE_J);
  const int tile_rows = slab ? bl * tr : TILE_J;     // TMEM lanes holding data
  const uint32_t xbytes = (uint32_t)((M1 ? TILE_J : bl * tr) * BI * 4);
  const int nst = (I + BI - 1) / BI;                  // stages per tile
  const int nseg = (nst + SEG - 1) / SEG;             // accumulation segments per tile
  constexpr uint32_t idesc2 = idesc_tf32(128, 2 * NPAD), idesc1 = idesc_tf32(128, NPAD);

  if (tid == 0) {
    for (int s = 0; s < X_STAGES; ++s) {
      mbar_init(&sm.full_x[s], 1);
      mbar_init(&sm.empty_x[s], 128);
    }
    for (int a = 0; a < A_STAGES; ++a) {
      mbar_init(&sm.full_a[a], 128);
      mbar_init(&sm.empty_a[a], 1);
    }
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(&sm.d_full[b], 1);
      mbar_init(&sm.d_empty[b], NUM_EPI);
    }
    mbar_init(&sm.drain, 1);
    sm.abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == MMA_WARP) {
    tmem_alloc(&sm.tmem_base, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm.tmem_base;
  volatile int* abort_flag = &sm.abort_flag;
  bool ok = true;
  // tiles of this CTA: blockIdx.x, blockIdx.x + gridDim.x, ...
  const int my_tiles = (ntiles > (int)blockIdx.x) ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int total = my_tiles * nst;                   // stages of this CTA

  int issued = 0;                                     // stages the producer has put in flight
  if (warp == PRODUCER_WARP) {
    if (lane == 0) {
      const uint32_t bytes = xbytes + (uint32_t)(M_TILE * 4);
      for (int g = 0; g < total && ok; ++g) {
        const int s = g % X_STAGES;
        const uint32_t ph = (uint32_t)(g / X_STAGES) & 1u;
        if (!mbar_wait(&sm.empty_x[s], ph ^ 1u, abort_flag)) { ok = false; break; }
        const int tile = (int)blockIdx.x + (g / nst) * (int)gridDim.x;
        const int ib = (g % nst) * BI;
        issued = g + 1;
        mbar_arrive_expect_tx(&sm.full_x[s], bytes);
        if (M1) {
          tma_load_2d(sm.x[s], &tmX, ib, tile * TILE_J, &sm.full_x[s]);
        } else if (tpr > 0) {
          tma_load_3d(sm.x[s], &tmX, (tile % tpr) * TILE_J, ib, tile / tpr, &sm.full_x[s]);
        } else if (slab) {                            // r past Rt in the last slab tile reads zeros
          tma_load_3d(sm.x[s], &tmX, 0, ib, tile * tr, &sm.full_x[s]);
        } else {
          const int64_t j0 = (int64_t)tile * TILE_J, r0 = j0 / L;
          tma_load_3d(sm.x[s], &tmX, (int)(j0 - r0 * L), ib, (int)r0, &sm.full_x[s]);
        }
        tma_load_2d(sm.mraw[s], &tmM, ib, 0, &sm.full_x[s]);
      }
    }
  } else if (warp == MMA_WARP) {
    if (lane == 0) {
      int ks0 = 0, gs = 0;                             // stage within the tile, segment over the CTA
      for (int g = 0; g < total && ok; ++g) {
        const int buf = gs % NBUF;
        const bool seg_first = (ks0 % SEG) == 0, seg_last = (ks0 % SEG) == SEG - 1 || ks0 == nst - 1;
        if (seg_first) {                               // the segment's buffer must have been drained
          if (!mbar_wait_fast(&sm.d_empty[buf], ((uint32_t)(gs / NBUF) & 1u) ^ 1u, abort_flag)) { ok = false; break; }
        }
        const int a = g % A_STAGES;
        if (!mbar_wait_fast(&sm.full_a[a], (uint32_t)(g / A_STAGES) & 1u, abort_flag)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(D_COL0 + buf * D_COLS);
        const uint32_t ahi = tmem + (uint32_t)(A_COL0 + a * A_STAGE_COLS);
        const uint32_t bhl = smem_u32(sm.b[a][0]);   // the lo tile follows: rows NPAD.. of the stacked operand
#pragma unroll
        for (int ks = 0; ks < BI / 8; ++ks) {
          const uint64_t db = smem_desc_kmajor_nosw(bhl + ks * 256, 128, 1024);
          mma_tf32_ts(d, ahi + ks * 8, db, idesc2, (!seg_first || ks > 0) ? 1u : 0u);
          mma_tf32_ts(d, ahi + BI + ks * 8, db, idesc1, 1u);
        }
        mma_commit(&sm.empty_a[a]);
        if (seg_last) {
          mma_commit(&sm.d_full[buf]);
          ++gs;
        }
        if (++ks0 == nst) ks0 = 0;
      }
      mma_commit(&sm.drain);
    }
  } else if (warp < 8) {
    // ------------------------------------------------------------ transform
    const int wg = warp >> 2, quad = warp & 3;
    const int row = quad * 32 + lane;                 // j within the tile = TMEM lane
    const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
    const int xt = tid & 127;                         // thread index within the warpgroup
    const int xoff = M1 ? 0 : (row / bl) * BI * bl + row % bl;   // strided: row = l' + bl r' -> [r'][0][l']
    for (int g = wg; g < total && ok; g += 2) {
      const int s = g % X_STAGES, a = g % A_STAGES;
      if (!mbar_wait(&sm.full_x[s], (uint32_t)(g / X_STAGES) & 1u, abort_flag)) { ok = false; break; }
      if (!mbar_wait(&sm.empty_a[a], ((uint32_t)(g / A_STAGES) & 1u) ^ 1u, abort_flag)) { ok = false; break; }
      tc_fence_after();
      uint32_t hi[32], lo[32];
      if (M1) {
        // row `row` of the swizzled X tile: logical 16-byte chunk c sits at chunk c ^ (row & 7)
        const float4* xr = reinterpret_cast<const float4*>(sm.x[s] + row * BI);
#pragma unroll
        for (int c = 0; c < BI / 4; ++c) {
          const float4 v = xr[c ^ (row & 7)];
          split_tf32(v.x, hi[4 * c + 0], lo[4 * c + 0]);
          split_tf32(v.y, hi[4 * c + 1], lo[4 * c + 1]);
          split_tf32(v.z, hi[4 * c + 2], lo[4 * c + 2]);
          split_tf32(v.w, hi[4 * c + 3], lo[4 * c + 3]);
        }
      } else if (row < tile_rows) {
        // strided tile [r'][i][l']
        const float* xr = sm.x[s] + xoff;
#pragma unroll
        for (int i = 0; i < BI; ++i) split_tf32(xr[i * bl], hi[i], lo[i]);
      } else {
#pragma unroll
        for (int i = 0; i < BI; ++i) hi[i] = lo[i] = 0u;   // idle lane of a slab tile
      }
      const uint32_t col = tmem + (uint32_t)(A_COL0 + a * A_STAGE_COLS) + lane_base;
      uint32_t h16[16], l16[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) { h16[q] = hi[q]; l16[q] = lo[q]; }
      tmem_st_x16(col, h16);
      tmem_st_x16(col + BI, l16);
#pragma unroll
      for (int q = 0; q < 16; ++q) { h16[q] = hi[16 + q]; l16[q] = lo[16 + q]; }
      tmem_st_x16(col + 16, h16);
      tmem_st_x16(col + BI + 16, l16);
      // B tiles: M(i, k) for the stage, element (n = k, kk = i offset)
#pragma unroll
      for (int u = 0; u < NPAD * BI / 128; ++u) {
        const int w = xt + u * 128;
        const int n = 8 * (w >> 8) + ((w >> 2) & 7), kk = 4 * ((w >> 5) & 7) + (w & 3);
        // raw M tile rows are 128-byte swizzled: 16-byte chunk c of row n sits at c ^ (n & 7)
        const float v = (n < K) ? sm.mraw[s][n * BI + (((kk >> 2) ^ (n & 7)) << 2) + (kk & 3)] : 0.f;
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
  } else if (warp < 12) {
    // ------------------------------------------------------------ epilogue
    const int quad = warp & 3;
    const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
    for (int tl = 0; tl < my_tiles && ok; ++tl) {
      // the tile's segments, summed in FP32 registers in segment order
      float acc[NPAD];
#pragma unroll
      for (int c = 0; c < NPAD; ++c) acc[c] = 0.f;
      for (int sg = 0; sg < nseg && ok; ++sg) {
        const int gs = tl * nseg + sg, buf = gs % NBUF;
        if (!mbar_wait(&sm.d_full[buf], (uint32_t)(gs / NBUF) & 1u, abort_flag)) { ok = false; break; }
        tc_fence_after();
#pragma unroll
        for (int c0 = 0; c0 < NPAD / 16; ++c0) {
          uint32_t vh[16], vl[16];
          const uint32_t dcol = tmem + lane_base + (uint32_t)(D_COL0 + buf * D_COLS + 16 * c0);
          tmem_ld_x16(dcol, vh);
          tmem_ld_x16(dcol + NPAD, vl);
          tmem_wait_ld();
#pragma unroll
          for (int c = 0; c < 16; ++c) acc[16 * c0 + c] += __uint_as_float(vh[c]) + __uint_as_float(vl[c]);
        }
        tc_fence_before();
        mbar_arrive(&sm.d_empty[buf]);
      }
      if (!ok) break;
      const int tile = (int)blockIdx.x + tl * (int)gridDim.x;
      const int64_t tj0 = slab ? (int64_t)tile * tr * L : (int64_t)tile * TILE_J;   // first j of the tile
      int64_t j = tj0 + quad * 32 + lane;
      if (quad * 32 + lane >= tile_rows) j = J;
      if (tpr > 0) {                                   // row l of this r's tile; l >= L is padding
        const int64_t l = (int64_t)(tile % tpr) * TILE_J + quad * 32 + lane;
        j = (l < L) ? l + L * (int64_t)(tile / tpr) : J;
      }
      const int64_t rj = j / o_L;
      float* orow = out + (j - rj * o_L) + rj * o_r;
      if (o_k == 1 && o_L == 1 && tpr == 0) {
        // rows of the output are contiguous in k (row j at out + j*o_r): stage 32 rows x
        // 16 columns per warp and store two 64-byte row segments per instruction
        float* stg = sm.ostage[quad];
        const int64_t jw = tj0 + quad * 32;                       // first row of this warp
#pragma unroll
        for (int c0 = 0; c0 < NPAD; c0 += 16) {
#pragma unroll
          for (int c = 0; c < 16; ++c) stg[lane * 17 + c] = acc[c0 + c];
          __syncwarp();
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int rr = 2 * q + (lane >> 4), cc = lane & 15;
            const int64_t jr = jw + rr;
            if (c0 + cc < K && jr < J && quad * 32 + rr < tile_rows) out[jr * o_r + c0 + cc] = stg[rr * 17 + cc];
          }
          __syncwarp();
        }
      } else {
#pragma unroll
        for (int k = 0; k < NPAD; ++k)
          if (k < K && j < J) orow[(int64_t)k * o_k] = acc[k];
      }
    }
  }
  if (!ok) {
    *abort_flag = 1;
    set_error(st, RHOSVD_ETIMEOUT);
  }
  __syncthreads();
  if (sm.abort_flag && warp == PRODUCER_WARP && lane == 0) {
    // copies the producer issued may still be writing into the ring: wait
    // (bounded) for the last phase of every stage it used before the CTA exits
    for (int s = 0; s < X_STAGES && s < issued; ++s) {
      const int g_last = s + X_STAGES * ((issued - 1 - s) / X_STAGES);
      const uint64_t t0 = globaltimer_ns();
      while (!mbar_try_wait(&sm.full_x[s], (uint32_t)(g_last / X_STAGES) & 1u) &&
             globaltimer_ns() - t0 < kWaitLimitNs) {
      }
    }
  }
  if (warp == MMA_WARP) {
    if (sm.abort_flag && lane == 0) {
      // MMAs already issued must finish before tensor memory is released
      const uint64_t t0 = globaltimer_ns();
      while (!mbar_try_wait(&sm.drain, 0) && globaltimer_ns() - t0 < kWaitLimitNs) {
      }
    }
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// ---------------------------------------------------------------- host side
// Tile geometry of a strided view: the box's l extent (0 if unsupported; below
// 128 it selects slab tiles, when L < 128 and Rt > 1), the r-slabs per tile
// tr = floor(128 / L) of slab tiles, and tpr > 0 when
// tiles are laid out per r (tpr = ceil(L / 128) tiles of 128 l for each r, the
// last one partial) because 128 consecutive j would straddle r.
int strided_bl(const View& x, int* tr, int* tpr) {
  *tpr = 0;
  *tr = 1;
  if (x.L < 4 || x.L % 4 != 0) return 0;
  if (x.Rt == 1 && x.L >= 128) return 128;
  if (x.L % 128 == 0) return 128;
  if (x.L < 128) {
    *tr = (int)(128 / x.L);
    return (int)x.L;
  }
  *tpr = (int)((x.L + TILE_J - 1) / TILE_J);
  return 128;
}

template <int NPAD, bool M1>
cudaError_t launch_npad(const CUtensorMap& tmX, const CUtensorMap& tmM, int I, int64_t L, int64_t J, int bl, int tr,
                        int tpr, int K, const OView& out, const DevStatus* skip, DevStatus* st, cudaStream_t stream) {
  const size_t smem = sizeof(TtmSmem<NPAD>) + 1024;
  static_assert(sizeof(TtmSmem<NPAD>) + 1024 <= 232448, "TTM stages exceed shared memory");
  cudaError_t e = allow_dynamic_smem((const void*)tc_ttm_kernel<NPAD, M1>, smem);
  if (e != cudaSuccess) return e;
  const int64_t Rt = J / L;
  const bool slab = !M1 && tpr == 0 && bl < TILE_J;
  const int ntiles = tpr > 0 ? (int)(tpr * Rt) : slab ? (int)((Rt + tr - 1) / tr) : (int)((J + TILE_J - 1) / TILE_J);
  const int grid = std::min(ntiles, device_sms());
  const int64_t o_L = out.o_L > 0 ? out.o_L : L;
  tc_ttm_kernel<NPAD, M1><<<grid, NUM_THREADS, smem, stream>>>(tmX, tmM, I, L, J, bl, tr, tpr, K, out.p,
                                                                out.o_k, out.o_r, o_L, skip, st);
  return cudaGetLastError();
}

template <bool M1>
cudaError_t launch_m(const CUtensorMap& tmX, const CUtensorMap& tmM, int I, int64_t L, int64_t J, int bl, int tr,
                     int tpr, int K, const OView& out, const DevStatus* skip, DevStatus* st, cudaStream_t stream) {
  switch (((K + 15) / 16) * 16) {
    case 16: return launch_npad<16, M1>(tmX, tmM, I, L, J, bl, tr, tpr, K, out, skip, st, stream);
    case 32: return launch_npad<32, M1>(tmX, tmM, I, L, J, bl, tr, tpr, K, out, skip, st, stream);
    case 48: return launch_npad<48, M1>(tmX, tmM, I, L, J, bl, tr, tpr, K, out, skip, st, stream);
    default: return launch_npad<64, M1>(tmX, tmM, I, L, J, bl, tr, tpr, K, out, skip, st, stream);
  }
}

}  // namespace

bool tc_ttm_supported(const View& x, int64_t m_i, int64_t m_k, int K, const OView& out) {
  if (m_i != 1 || m_k < x.I || m_k % 4 != 0) return false;     // M column-major, ld multiple of 4
  if (K < 1 || K > 64 || x.I < 1 || x.I > (int64_t(1) << 30)) return false;
  const int64_t J = x.L * x.Rt;
  if (J < TILE_J || J > (int64_t(1) << 40)) return false;
  if (x.L == 1) return x.s_i == 1 && x.s_r == x.I && x.I % 4 == 0;   // X(i, j) = X[i + I*j]
  int tr = 1, tpr = 0;
  if (strided_bl(x, &tr, &tpr) == 0 || x.s_i % 4 != 0 || (x.Rt > 1 && x.s_r % 4 != 0)) return false;
  if (tpr > 0 && out.o_L > 0 && out.o_L != x.L) return false;     // per-r tiles split j by the input's L
  if (tpr > 0 && (int64_t)tpr * x.Rt >= (int64_t(1) << 31)) return false;
  return x.Rt < (int64_t(1) << 31) && x.L < (int64_t(1) << 31);
}

cudaError_t launch_tc_ttm(const View& x, const float* Mp, int64_t m_k, int K, const OView& out,
                          const DevStatus* skip, DevStatus* st, cudaStream_t stream) {
  if ((reinterpret_cast<uintptr_t>(x.p) & 15) || (reinterpret_cast<uintptr_t>(Mp) & 15)) return cudaErrorNotSupported;
  const int64_t I = x.I, J = x.L * x.Rt;
  CUtensorMap tmX, tmM;
  {
    const uint64_t dims[2] = {(uint64_t)I, (uint64_t)K};
    const uint64_t strides[1] = {(uint64_t)m_k};
    const uint32_t box[2] = {BI, (uint32_t)(((K + 15) / 16) * 16)};   // NPAD rows, k >= K zero-filled
    if (!make_tmap_f32(&tmM, Mp, 2, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_128B)) return cudaErrorNotSupported;
  }
  if (x.L == 1) {
    const uint64_t dims[2] = {(uint64_t)I, (uint64_t)J};
    const uint64_t strides[1] = {(uint64_t)I};
    const uint32_t box[2] = {BI, TILE_J};
    if (!make_tmap_f32(&tmX, x.p, 2, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_128B)) return cudaErrorNotSupported;
    return launch_m<true>(tmX, tmM, (int)I, 1, J, 0, 1, 0, K, out, skip, st, stream);
  }
  int tr = 1, tpr = 0;
  const int bl = strided_bl(x, &tr, &tpr);
  if (bl == 0) return cudaErrorNotSupported;
  // always rank 3 (the producer issues 3-D copies); a matrix view gets a unit r extent
  const uint64_t dims[3] = {(uint64_t)x.L, (uint64_t)I, (uint64_t)x.Rt};
  const uint64_t strides[2] = {(uint64_t)x.s_i, x.Rt > 1 ? (uint64_t)x.s_r : (uint64_t)x.s_i * (uint64_t)I};
  const uint32_t box[3] = {(uint32_t)bl, BI, (uint32_t)tr};
  const bool okmap = make_tmap_f32(&tmX, x.p, 3, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_NONE);
  if (!okmap) return cudaErrorNotSupported;
  return launch_m<false>(tmX, tmM, (int)I, x.L, J, bl, tr, tpr, K, out, skip, st, stream);
}

}  // namespace rhosvd
