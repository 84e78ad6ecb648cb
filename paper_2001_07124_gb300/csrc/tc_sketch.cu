// Tensor-core (tcgen05) sketch Y = X_(n) W on a strided unfolding:
// Y(i,k) = sum_j X_(n)(i,j) W[j + J*k], X_(n)(i, j = l + L*r) = X[l + s_i*i + s_r*r]
// (the sketches of Alg. 1, Alg. 6 and Alg. 9; for n = 1 the dominant pass of
// R-STHOSVD).  A stage holds 32 KB of X: 32 j x 256 rows i (two 128-row MMA
// tiles, two 16-j chunks) for modes with I > 128, 64 j x 128 rows (one tile,
// four chunks) for short modes.  Layouts in shared memory:
//   * mode 1 (L = 1): one 2-D box {rows i, stage j}, smem [jj][rows];
//   * strided (L % 16 == 0): one 3-D box {16 l, rows i, 1 r} per 16-j chunk
//     over [L, I, Rt] with 64-byte swizzle, smem [chunk][i][16 l], each lane
//     reading its own 64-byte row as four float4 (16-byte piece q of row i
//     sits at piece q ^ ((i >> 1) & 3)).
//
// The contraction over j is split over CTAs (one CTA per SM, persistent); each
// CTA owns up to 256 rows i and every gridDim.x-th stage-sized block of j, and
// writes its partial I x K block for the fixed-order reducer.  Interleaving
// the blocks keeps the CTAs' concurrent reads within one window of each row
// of X_(n), and CTAs of different row groups read the same W block at about
// the same time (its second read comes from L2).
//
// Products in 3xTF32 (each FP32 value split into a TF32 part hi and an exact
// remainder lo, Ootomo & Yokota 2022): X_hi W_hi + X_hi W_lo + X_lo W_hi.  The
// B operand of a chunk is the stacked [W_hi; W_lo] (N = 2 NPAD rows), so each
// K step of a tile takes two MMAs instead of three skinny ones:
//   D[:, 0:2NPAD)  += X_hi [W_hi W_lo]     (N = 2 NPAD)
//   D[:, 0:NPAD)   += X_lo W_hi            (N = NPAD)
// and Y = D[:, 0:NPAD) + D[:, NPAD:2NPAD).  Roles:
//   * TMA producer (warp 8): the X tile and the raw W tiles (16 x NPAD per
//     chunk) of a stage into a shared-memory ring;
//   * eight transform warps (two warpgroups; warp w owns TMEM lane quadrant
//     w % 4; warpgroup g fills A slots 2g and 2g+1, slot u = (tile u / NC,
//     chunk u % NC)) split X into hi and lo and store both into tensor memory
//     as the A operand (tcgen05.st), and build the hi/lo B tiles in the
//     canonical no-swizzle K-major layout;
//   * one thread of warp 9 issues the MMAs into FP32 accumulators in TMEM;
//   * at the end the transform warps read the accumulators (tcgen05.ld), add
//     the two halves and write the partial sums.
// Requirements (checked by tc_sketch_supported): K <= 64, J >= 1024, W a
// plain J x K matrix with J % 4 == 0, 16-byte aligned pointers; mode 1 needs
// I % 4 == 0, a strided view L % 16 == 0 and strides that are multiples of 4.
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace rhosvd {
namespace {

using namespace tc;

constexpr int BJ = 16;                    // j per MMA chunk (two tf32 MMA K steps of 8)
constexpr int A_STAGES = 2;
constexpr int NUM_XFORM = 256;            // warps 0-7
constexpr int NUM_THREADS = NUM_XFORM + 64;   // + warp 8 producer, warp 9 MMA issuer
constexpr uint32_t TMEM_COLS = 512;
constexpr int D_COLS = 128;               // accumulator columns per tile: the hi and lo halves (<= 64 each)
constexpr int A_STAGE_COLS = 128;         // per stage: 4 slots x (16 hi + 16 lo)
constexpr int STAGE_FLOATS = 8192;        // X floats per stage (32 KB)
constexpr size_t kSmemLimit = 232448;     // dynamic shared memory per CTA (227 KB)

// Stage geometry, NC = chunks of 16 j per stage: NC = 2 stages 32 j x 256 rows
// (two 128-row tiles), NC = 4 stages 64 j x 128 rows (one tile) for short modes
// (I <= 128).  The four TMEM A slots of a stage hold (tile, chunk) pairs.  The W
// and B tiles hold only NPAD rows (K padded to 16) and the rest of shared memory
// deepens the X ring.
template <int NPAD, int NC>
struct Geo {
  static constexpr int TILES = 4 / NC;                    // 128-row tiles per CTA
  static constexpr int ROWS = 128 * TILES;                // rows i per CTA (one TMA box)
  static constexpr int SBJ = BJ * NC;                     // j per stage
  static constexpr int W_TILE = NPAD * BJ;                // floats per W / B tile
  static constexpr int A_COL0 = TILES * D_COLS;           // first TMEM column of the A stages
  static constexpr size_t FIXED = (size_t)A_STAGES * NC * 2 * W_TILE * 4 + 2048;
  static constexpr size_t PER_STAGE = (size_t)STAGE_FLOATS * 4 + (size_t)NC * W_TILE * 4;
  static constexpr int X_STAGES_FIT = (int)((kSmemLimit - 1024 - FIXED) / PER_STAGE);
  static constexpr int X_STAGES = X_STAGES_FIT < 6 ? X_STAGES_FIT : 6;
  static_assert(A_COL0 + A_STAGES * A_STAGE_COLS <= (int)TMEM_COLS, "tensor memory overflow");
  static_assert(2 * NPAD <= D_COLS, "accumulator halves exceed the tile's columns");
};

template <int NPAD, int NC>
struct __align__(1024) SketchSmem {
  using G = Geo<NPAD, NC>;
  float x[G::X_STAGES][STAGE_FLOATS];        // mode 1: [jj][rows]; strided: [chunk][i][16]
  float wraw[G::X_STAGES][NC][G::W_TILE];    // TMA boxes [n][jj] (64B swizzle), rows n >= K zero-filled
  float b[A_STAGES][NC][2][G::W_TILE];       // per chunk the hi tile, then the lo tile (one N = 2 NPAD operand)
  uint64_t full_x[G::X_STAGES], empty_x[G::X_STAGES];
  uint64_t full_a[A_STAGES], empty_a[A_STAGES];
  uint64_t done;
  uint32_t tmem_base;
  int abort_flag;
};

// B tiles (N x 16 K elements, K-major, no swizzle): element (n, kk) sits at
// byte (n >> 3) * 512 + (kk >> 2) * 128 + (n & 7) * 16 + (kk & 3) * 4, i.e.
// 8-row x 16-byte core matrices with LBO = 128 (K direction) and SBO = 512
// (N direction); the second MMA K step starts 256 bytes in.  The lo tile
// follows the hi tile directly, so rows NPAD.. of the stacked operand are lo.

// GEN: W is the seeded Gaussian test matrix Omega(j, k) of (seed, stream),
// computed in the transform warps from the counter-based generator (the same
// function the omega kernel evaluates, so the values are identical) instead of
// being read from memory.
template <int NPAD, bool M1, int NC, bool GEN>
__global__ void __launch_bounds__(NUM_THREADS, 1)
tc_sketch_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmW, int I,
                 int64_t L, int64_t J, int K, float* __restrict__ part, uint64_t seed,
                 uint32_t stream_id, DevStatus* st) {
  using G = Geo<NPAD, NC>;
  constexpr int X_STAGES = G::X_STAGES, ROWS = G::ROWS, SBJ = G::SBJ, A_COL0 = G::A_COL0;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  SketchSmem<NPAD, NC>& sm = *reinterpret_cast<SketchSmem<NPAD, NC>*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int split = blockIdx.x;
  const int i0 = blockIdx.y * ROWS;
  const int rows = min(ROWS, I - i0);
  const int mt = (rows + 127) / 128;                 // MMA tiles in this CTA
  // stage kb of this CTA covers j in [(split + kb * nsplit) * SBJ, ... + SBJ) clipped to J
  const int64_t nblk = (J + SBJ - 1) / SBJ, nsplit = gridDim.x;
  const int nkb = nblk > split ? (int)((nblk - 1 - split) / nsplit + 1) : 0;
  auto stage_j = [&](int kb) -> int64_t { return ((int64_t)split + (int64_t)kb * nsplit) * SBJ; };
  constexpr uint32_t idesc2 = idesc_tf32(128, 2 * NPAD), idesc1 = idesc_tf32(128, NPAD);

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
  int issued = 0;                                    // stages the producer has put in flight

  if (warp == 8) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      const uint32_t bytes = (uint32_t)(STAGE_FLOATS * 4) + (GEN ? 0u : (uint32_t)(NC * G::W_TILE * 4));
      for (int kb = 0; kb < nkb && ok; ++kb) {
        const int s = kb % X_STAGES;
        const uint32_t ph = (uint32_t)(kb / X_STAGES) & 1u;
        if (!mbar_wait(&sm.empty_x[s], ph ^ 1u, abort_flag)) { ok = false; break; }
        issued = kb + 1;
        mbar_arrive_expect_tx(&sm.full_x[s], bytes);
        const int jt = (int)stage_j(kb);
        if (M1) {
          tma_load_2d(sm.x[s], &tmX, i0, jt, &sm.full_x[s]);
        } else {
          // one box per 16-j chunk; a chunk never crosses r since L % 16 == 0
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            const int64_t jc = (int64_t)jt + BJ * c, rc = jc / L;
            tma_load_3d(sm.x[s] + c * BJ * ROWS, &tmX, (int)(jc - rc * L), i0, (int)rc, &sm.full_x[s]);
          }
        }
        if (!GEN)
#pragma unroll
          for (int c = 0; c < NC; ++c) tma_load_2d(sm.wraw[s][c], &tmW, jt + BJ * c, 0, &sm.full_x[s]);
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
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int t = u / NC, c = u % NC;
          if (t >= mt) continue;
          const uint32_t d = tmem + (uint32_t)(t * D_COLS);
          const uint32_t ahi = tmem + (uint32_t)(A_COL0 + a * A_STAGE_COLS + u * 32);
          const uint32_t bhl = smem_u32(sm.b[a][c][0]);
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            const uint64_t db = smem_desc_kmajor_nosw(bhl + ks * 256, 128, 512);
            mma_tf32_ts(d, ahi + ks * 8, db, idesc2, (kb > 0 || c > 0 || ks > 0) ? 1u : 0u);
            mma_tf32_ts(d, ahi + 16 + ks * 8, db, idesc1, 1u);
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
      const int64_t rem = J - stage_j(kb);
      const int valid = rem < SBJ ? (int)rem : SBJ;   // valid j of this stage
      if (!mbar_wait(&sm.empty_a[a], pha ^ 1u, abort_flag)) { ok = false; break; }
      tc_fence_after();
      // Generated B tiles need no data from X: they are built before waiting for
      // the stage's X tile, in the shadow of its TMA copy.
      if (GEN) {
        // Omega(j, 4g..4g+3) from one generator call; thread = (jj, g) of a chunk
        constexpr int NQ = NPAD / 4;
        const int64_t jt = stage_j(kb);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int vc = valid - BJ * c;
          for (int q = tid; q < BJ * NQ; q += NUM_XFORM) {
            const int jj = q % BJ, g = q / BJ;
            float z[4] = {0.f, 0.f, 0.f, 0.f};
            if (jj < vc && 4 * g < K) omega_quad(seed, stream_id, (uint64_t)(jt + BJ * c + jj), (uint32_t)g, z);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int n = 4 * g + e;
              const int w = (n >> 3) * 128 + (jj >> 2) * 32 + (n & 7) * 4 + (jj & 3);
              uint32_t h, l;
              split_tf32(n < K ? z[e] : 0.f, h, l);
              reinterpret_cast<uint32_t*>(sm.b[a][c][0])[w] = h;
              reinterpret_cast<uint32_t*>(sm.b[a][c][1])[w] = l;
            }
          }
        }
      }
      if (!mbar_wait(&sm.full_x[s], phx, abort_flag)) { ok = false; break; }
#pragma unroll
      for (int uu = 0; uu < 2; ++uu) {
        const int u = 2 * wg + uu;                    // A slot: (tile, chunk)
        const int t = u / NC, c = u % NC;
        if (t < mt) {
          const int r = t * 128 + row_in_tile;       // row within the CTA's block
          const int vc = valid - BJ * c;              // valid j of this chunk (may be <= 0)
          uint32_t hi[16], lo[16];
          if (M1) {
            const float* xb = sm.x[s] + BJ * c * ROWS + r;
#pragma unroll
            for (int jj = 0; jj < BJ; ++jj) {
              const float v = (jj < vc && r < rows) ? xb[jj * ROWS] : 0.f;
              split_tf32(v, hi[jj], lo[jj]);
            }
          } else {
            const float4* xr = reinterpret_cast<const float4*>(sm.x[s] + c * BJ * ROWS + r * BJ);
#pragma unroll
            for (int q = 0; q < BJ / 4; ++q) {
              float4 v = xr[q ^ ((r >> 1) & 3)];
              if (r >= rows) v = make_float4(0.f, 0.f, 0.f, 0.f);
              const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
              for (int w = 0; w < 4; ++w) split_tf32((4 * q + w < vc) ? e[w] : 0.f, hi[4 * q + w], lo[4 * q + w]);
            }
          }
          const uint32_t col = tmem + (uint32_t)(A_COL0 + a * A_STAGE_COLS + u * 32);
          tmem_st_x16(col + lane_base, hi);
          tmem_st_x16(col + 16 + lane_base, lo);
        }
      }
      // B tiles from memory: element (n, jj) of W, split into hi / lo.  Threads walk
      // the canonical layout word by word (conflict-free stores): word w holds
      // n = 8 (w >> 7) + ((w >> 2) & 7), jj = 4 ((w >> 5) & 3) + (w & 3).
#pragma unroll
      for (int c = 0; c < (GEN ? 0 : NC); ++c) {
        const int vc = valid - BJ * c;
#pragma unroll
        for (int u = 0; u < NPAD * BJ / NUM_XFORM; ++u) {
          const int w = tid + u * NUM_XFORM;
          const int n = 8 * (w >> 7) + ((w >> 2) & 7), jj = 4 * ((w >> 5) & 3) + (w & 3);
          // raw W tile rows are 64-byte swizzled: 16-byte piece q of row n sits at q ^ ((n >> 1) & 3)
          const float v =
              (jj < vc && n < K) ? sm.wraw[s][c][n * BJ + (((jj >> 2) ^ ((n >> 1) & 3)) << 2) + (jj & 3)] : 0.f;
          uint32_t h, l;
          split_tf32(v, h, l);
          reinterpret_cast<uint32_t*>(sm.b[a][c][0])[w] = h;
          reinterpret_cast<uint32_t*>(sm.b[a][c][1])[w] = l;
        }
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
      for (int t = wg; t < mt; t += 2) {
        const int64_t i = i0 + t * 128 + row_in_tile;
#pragma unroll
        for (int c0 = 0; c0 < NPAD; c0 += 16) {
          uint32_t vh[16], vl[16];
          tmem_ld_x16(tmem + lane_base + (uint32_t)(t * D_COLS + c0), vh);
          tmem_ld_x16(tmem + lane_base + (uint32_t)(t * D_COLS + NPAD + c0), vl);
          tmem_wait_ld();
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            const int k = c0 + c;
            if (k < K && i < I)
              part[((int64_t)split * K + k) * I + i] =
                  (nkb > 0) ? __uint_as_float(vh[c]) + __uint_as_float(vl[c]) : 0.f;
          }
        }
      }
    }
  }
  if (!ok) {
    *abort_flag = 1;
    set_error(st, RHOSVD_ETIMEOUT);
  }
  // teardown: every role is past its last wait (all waits are bounded); on the
  // abort path let copies and MMAs in flight drain before the CTA releases
  // tensor memory and exits
  __syncthreads();
  if (sm.abort_flag && warp == 8 && lane == 0) {
    for (int s = 0; s < X_STAGES && s < issued; ++s) {
      const int kb_last = s + X_STAGES * ((issued - 1 - s) / X_STAGES);
      const uint64_t t0 = globaltimer_ns();
      while (!mbar_try_wait(&sm.full_x[s], (uint32_t)(kb_last / X_STAGES) & 1u) &&
             globaltimer_ns() - t0 < kWaitLimitNs) {
      }
    }
  }
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
struct Gen {
  bool on;
  uint64_t seed;
  uint32_t stream;
};

template <int NPAD, bool M1, int NC, bool GEN>
cudaError_t launch_k(const CUtensorMap& tmX, const CUtensorMap& tmW, int I, int64_t L, int64_t J, int K,
                     const TcSketchPlan& pl, float* part, const Gen& gen, DevStatus* st, cudaStream_t stream) {
  const size_t smem = sizeof(SketchSmem<NPAD, NC>) + 1024;
  static_assert(sizeof(SketchSmem<NPAD, NC>) + 1024 <= kSmemLimit, "sketch stages exceed shared memory");
  cudaError_t e = allow_dynamic_smem((const void*)tc_sketch_kernel<NPAD, M1, NC, GEN>, smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)pl.splits, (unsigned)pl.mgroups);
  tc_sketch_kernel<NPAD, M1, NC, GEN><<<grid, NUM_THREADS, smem, stream>>>(tmX, tmW, I, L, J, K, part, gen.seed,
                                                                          gen.stream, st);
  return cudaGetLastError();
}

template <bool M1, int NC, bool GEN>
cudaError_t launch_g(const CUtensorMap& tmX, const CUtensorMap& tmW, int I, int64_t L, int64_t J, int K,
                     const TcSketchPlan& pl, float* part, const Gen& gen, DevStatus* st, cudaStream_t stream) {
  switch (((K + 15) / 16) * 16) {
    case 16: return launch_k<16, M1, NC, GEN>(tmX, tmW, I, L, J, K, pl, part, gen, st, stream);
    case 32: return launch_k<32, M1, NC, GEN>(tmX, tmW, I, L, J, K, pl, part, gen, st, stream);
    case 48: return launch_k<48, M1, NC, GEN>(tmX, tmW, I, L, J, K, pl, part, gen, st, stream);
    default: return launch_k<64, M1, NC, GEN>(tmX, tmW, I, L, J, K, pl, part, gen, st, stream);
  }
}

template <bool M1, int NC>
cudaError_t launch_m(const CUtensorMap& tmX, const CUtensorMap& tmW, int I, int64_t L, int64_t J, int K,
                     const TcSketchPlan& pl, float* part, const Gen& gen, DevStatus* st, cudaStream_t stream) {
  return gen.on ? launch_g<M1, NC, true>(tmX, tmW, I, L, J, K, pl, part, gen, st, stream)
                : launch_g<M1, NC, false>(tmX, tmW, I, L, J, K, pl, part, gen, st, stream);
}

// Chunks per stage for a view: 4 (64 j x 128 rows, one tile) for short modes,
// else 2 (32 j x 256 rows, two tiles).
int chunks_for(const View& x) { return x.I > 128 ? 2 : 4; }

}  // namespace

bool tc_sketch_supported(const View& x, const WView& w, int K) {
  const int64_t J = x.L * x.Rt;
  if (w.w_r != x.L || w.w_k != J || J % 4 != 0) return false;      // W is a plain J x K matrix
  if (K < 1 || K > 64 || x.I < 1 || x.I > (int64_t(1) << 30) || J < 1024 || J >= (int64_t(1) << 31)) return false;
  if ((reinterpret_cast<uintptr_t>(x.p) & 15) || (reinterpret_cast<uintptr_t>(w.p) & 15)) return false;
  if (x.L == 1) return x.s_i == 1 && x.s_r == x.I && x.I % 4 == 0;  // mode-1 layout
  if (x.L % BJ != 0 || x.s_i % 4 != 0 || (x.Rt > 1 && x.s_r % 4 != 0)) return false;
  return x.L < (int64_t(1) << 31) && x.Rt < (int64_t(1) << 31);
}

static TcSketchPlan plan_nc(int64_t I, int64_t J, int nc) {
  TcSketchPlan pl;
  const int rows = 512 / nc, sbj = BJ * nc;          // 256 rows for nc = 2, 128 for nc = 4
  pl.mgroups = (int)((I + rows - 1) / rows);
  const int64_t nblk = (J + sbj - 1) / sbj;            // stage-sized blocks of j, dealt round-robin
  pl.splits = (int)std::min<int64_t>(std::max<int64_t>(1, device_sms() / pl.mgroups), nblk);
  pl.jchunk = sbj;
  return pl;
}

TcSketchPlan plan_tc_sketch(int64_t I, int K, int64_t J) {
  (void)K;
  // the larger of the two possible split counts sizes the partial sums
  const TcSketchPlan a = plan_nc(I, J, 2), b = plan_nc(I, J, 4);
  return (a.splits * a.mgroups >= b.splits * b.mgroups) ? a : b;
}

static cudaError_t tc_sketch_impl(const View& x, const WView& w, int K, float* Y, int64_t ldy, float* part,
                                  const Gen& gen, DevStatus* st, cudaStream_t stream) {
  const int64_t I = x.I, J = x.L * x.Rt;
  const int nc = chunks_for(x);
  const TcSketchPlan pl = plan_nc(I, J, nc);
  CUtensorMap tmX, tmW;
  memset(&tmW, 0, sizeof(tmW));
  if (!gen.on) {
    const uint64_t dims[2] = {(uint64_t)J, (uint64_t)K};
    const uint64_t strides[1] = {(uint64_t)J};
    const uint32_t box[2] = {BJ, (uint32_t)(((K + 15) / 16) * 16)};   // NPAD rows, k >= K zero-filled
    if (!make_tmap_f32(&tmW, w.p, 2, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_64B)) return cudaErrorNotSupported;
  }
  cudaError_t e;
  const uint32_t boxw = nc == 2 ? 256u : 128u;          // rows per CTA (one TMA box)
  if (x.L == 1) {
    const uint64_t dims[2] = {(uint64_t)I, (uint64_t)J};
    const uint64_t strides[1] = {(uint64_t)I};
    const uint32_t box[2] = {boxw, (uint32_t)(BJ * nc)};
    if (!make_tmap_f32(&tmX, x.p, 2, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_NONE)) return cudaErrorNotSupported;
    e = nc == 2 ? launch_m<true, 2>(tmX, tmW, (int)I, 1, J, K, pl, part, gen, st, stream)
                : launch_m<true, 4>(tmX, tmW, (int)I, 1, J, K, pl, part, gen, st, stream);
  } else {
    const uint64_t dims[3] = {(uint64_t)x.L, (uint64_t)I, (uint64_t)x.Rt};
    const uint64_t strides[2] = {(uint64_t)x.s_i, x.Rt > 1 ? (uint64_t)x.s_r : (uint64_t)x.s_i * (uint64_t)I};
    const uint32_t box[3] = {BJ, boxw, 1};
    if (!make_tmap_f32(&tmX, x.p, 3, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_64B)) return cudaErrorNotSupported;
    e = nc == 2 ? launch_m<false, 2>(tmX, tmW, (int)I, x.L, J, K, pl, part, gen, st, stream)
                : launch_m<false, 4>(tmX, tmW, (int)I, x.L, J, K, pl, part, gen, st, stream);
  }
  if (e != cudaSuccess) return e;
  return launch_reduce_partials_f(part, pl.splits, I, K, Y, ldy, stream);
}

cudaError_t launch_tc_sketch(const View& x, const WView& w, int K, float* Y, int64_t ldy, float* part,
                             DevStatus* st, cudaStream_t stream) {
  return tc_sketch_impl(x, w, K, Y, ldy, part, Gen{false, 0, 0}, st, stream);
}

// Where the test matrix is generated in-kernel: the transform warps evaluate the
// generator for every stage, and with two row groups per j block (or 64-j
// stages for short modes) each W tile is generated more than once per SM's
// worth of X.  Measured on GB300 with the stacked-operand kernel: 512^3 mode 1,
// 174 us generated in-kernel against 28 + 105 us for drawing Omega first and
// sketching from memory; 128^4 mode 1, 335 against 126 + 194 us.  Omega is
// therefore drawn first, except where the stream of X is itself slow: rows of
// X_(n) 4 MB or more apart (the last mode of a large tensor), where the TMA
// copies, not the generator, set the pace.
bool tc_sketch_seeded_supported(const View& x, int K) {
  const int64_t J = x.L * x.Rt;
  if (!tc_sketch_supported(x, WView{nullptr, x.L, J}, K)) return false;
  return x.s_i >= (int64_t(1) << 20);
}

cudaError_t launch_tc_sketch_seeded(const View& x, int K, uint64_t seed, uint32_t stream_id, float* Y, int64_t ldy,
                                    float* part, DevStatus* st, cudaStream_t stream) {
  const int64_t J = x.L * x.Rt;
  if (st == nullptr || !tc_sketch_seeded_supported(x, K)) return cudaErrorNotSupported;
  return tc_sketch_impl(x, WView{nullptr, x.L, J}, K, Y, ldy, part, Gen{true, seed, stream_id}, st, stream);
}

}  // namespace rhosvd
