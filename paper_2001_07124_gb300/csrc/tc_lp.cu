// Reduced-precision form of the sketch contractions: X kept in BF16 or in FP8
// e4m3 with per-slice scales, tensor-core products with FP32 accumulation.
//
// Formats (the paper leaves the arithmetic open; these are the ones the
// tensor cores take): BF16 (.kind::f16 MMAs, K = 16 per instruction) and
// e4m3 (.kind::f8f6f4, K = 32), A and B of one MMA always of the same type.
// Round to nearest even, e4m3 saturating at +-448.
//
// Per-slice scales: X is cut into the frontal slices of its last mode; e4m3
// slice k is stored as e4m3(X[..., k] / s_k) with s_k the smallest power of
// two that brings the slice's largest magnitude to at most 448, so that
// s_k * value is exact in FP32.  BF16 has the exponent range of FP32 and is
// stored unscaled (s_k = 1).  The scale of an element of the mode-n unfolding
// depends on the column j (n < N: slice = j / (J / I_N)) or on the row
// (n = N); the kernels apply it to FP32 partial sums: a sketch accumulates
// each slice's contribution in tensor memory and scales it when the slice
// ends, a TTM scales its output rows.
//
// The other operand (the test matrix Omega, a basis Q or Z) arrives in FP32
// and is split into a hi part in the format and a lo part for the remainder;
// stacked as [W_hi; W_lo] along N it takes one MMA per K step and
// Y = D[:, 0:NPAD) + D[:, NPAD:2NPAD).  A test matrix drawn for a
// reduced-precision run is rounded to the format beforehand, so its lo part is
// zero and the product X_q Omega is exact apart from the FP32 accumulation.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cstring>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace rhosvd {
namespace {

using namespace tc;

constexpr float kE4m3Max = 448.f;

// ---------------------------------------------------------------- format conversions
__device__ __forceinline__ uint32_t to_bf16_bits(float x) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x));
}
__device__ __forceinline__ float bf16_bits_to_float(uint32_t b) { return __uint_as_float(b << 16); }
__device__ __forceinline__ uint32_t to_e4m3_bits(float x) {
  return (uint32_t)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
}
__device__ __forceinline__ float e4m3_bits_to_float(uint32_t b) {
  __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)b, __NV_E4M3);
  return __half2float(__half(h));
}
// The element type of a reduced-precision copy, as a policy: EB bytes per
// element, the bit pattern of an FP32 value rounded to nearest, its value.
template <int EB>
struct Fmt;
template <>
struct Fmt<2> {
  __device__ static uint32_t bits(float x) { return to_bf16_bits(x); }
  __device__ static float value(uint32_t b) { return bf16_bits_to_float(b); }
};
template <>
struct Fmt<1> {
  __device__ static uint32_t bits(float x) { return to_e4m3_bits(x); }
  __device__ static float value(uint32_t b) { return e4m3_bits_to_float(b); }
};

// ---------------------------------------------------------------- quantisation of X
// amax[k] = max |X[.., k]| over frontal slice k (slice_len elements); the float
// bits of non-negative values order like unsigned integers.
__global__ void slice_amax_kernel(const float* __restrict__ x, int64_t slice_len, int64_t nslices,
                                  unsigned int* __restrict__ amax_bits) {
  for (int64_t slice = blockIdx.y; slice < nslices; slice += gridDim.y) {
    float m = 0.f;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < slice_len;
         e += (int64_t)gridDim.x * blockDim.x)
      m = fmaxf(m, fabsf(x[slice * slice_len + e]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(&amax_bits[slice], __float_as_uint(m));
  }
}

// s_k = smallest power of two with amax_k / s_k <= 448 (1 for an all-zero slice);
// non-finite slices keep their amax (the sketches then report the non-finite input).
__global__ void slice_scale_kernel(const unsigned int* __restrict__ amax_bits, int64_t nslices,
                                   float* __restrict__ scale) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nslices) return;
  const float a = __uint_as_float(amax_bits[k]);
  float s = 1.f;
  if (a > 0.f && isfinite(a)) {
    int e;
    frexpf(a / kE4m3Max, &e);              // a / 448 = f 2^e with f in [0.5, 1): 2^e >= a / 448
    s = ldexpf(1.f, e);
    if (a / ldexpf(1.f, e - 1) <= kE4m3Max) s = ldexpf(1.f, e - 1);   // a / 448 exactly a power of two
  }
  scale[k] = s;
}

// X_q = format(X / s_slice), 16 consecutive elements per thread.
template <int EB>
__global__ void quantize_kernel(const float* __restrict__ x, int64_t n, int64_t slice_len,
                                const float* __restrict__ scale, unsigned char* __restrict__ xq) {
  const int64_t e0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 16;
  if (e0 >= n) return;
  uint32_t b[16];
  if (e0 + 16 <= n && (e0 / slice_len) == ((e0 + 15) / slice_len)) {
    const float inv = scale != nullptr ? 1.f / scale[e0 / slice_len] : 1.f;   // a power of two: exact
    const float4* p = reinterpret_cast<const float4*>(x + e0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 v = p[q];
      b[4 * q + 0] = Fmt<EB>::bits(v.x * inv);
      b[4 * q + 1] = Fmt<EB>::bits(v.y * inv);
      b[4 * q + 2] = Fmt<EB>::bits(v.z * inv);
      b[4 * q + 3] = Fmt<EB>::bits(v.w * inv);
    }
  } else {
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      const int64_t e = e0 + t;
      const float inv = (scale != nullptr && e < n) ? 1.f / scale[e / slice_len] : 1.f;
      b[t] = (e < n) ? Fmt<EB>::bits(x[e] * inv) : 0u;
    }
  }
  if (e0 + 16 <= n) {
    if (EB == 2) {
      uint4* o = reinterpret_cast<uint4*>(xq + e0 * 2);
      o[0] = make_uint4(b[0] | (b[1] << 16), b[2] | (b[3] << 16), b[4] | (b[5] << 16), b[6] | (b[7] << 16));
      o[1] = make_uint4(b[8] | (b[9] << 16), b[10] | (b[11] << 16), b[12] | (b[13] << 16), b[14] | (b[15] << 16));
    } else {
      uint4* o = reinterpret_cast<uint4*>(xq + e0);
      uint32_t w[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) w[q] = b[4 * q] | (b[4 * q + 1] << 8) | (b[4 * q + 2] << 16) | (b[4 * q + 3] << 24);
      o[0] = make_uint4(w[0], w[1], w[2], w[3]);
    }
  } else {
    for (int t = 0; t < 16 && e0 + t < n; ++t) {
      if (EB == 2) reinterpret_cast<uint16_t*>(xq)[e0 + t] = (uint16_t)b[t];
      else xq[e0 + t] = (unsigned char)b[t];
    }
  }
}

// a[i] <- the nearest value of the format (in place, FP32 storage): the test
// matrices of a reduced-precision run.
template <int EB>
__global__ void round_to_format_kernel(float* __restrict__ a, int64_t n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) a[e] = Fmt<EB>::value(Fmt<EB>::bits(a[e]));
}

// The seeded Gaussian test matrix (the omega kernel's values) rounded to the
// format on store: one thread per (row j, group of four columns).
template <int EB>
__global__ void omega_rounded_kernel(uint64_t seed, uint32_t stream_id, int64_t rows, int cols,
                                     float* __restrict__ out, int64_t ld) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int g = blockIdx.y;
  if (j >= rows) return;
  float z[4];
  omega_quad(seed, stream_id, (uint64_t)j, (uint32_t)g, z);
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int k = 4 * g + t;
    if (k < cols) out[j + (int64_t)k * ld] = Fmt<EB>::value(Fmt<EB>::bits(z[t]));
  }
}

// ---------------------------------------------------------------- sketch Y = X_q,(n) W
// Stage: ROWS rows x NKS K-step chunks of 32 bytes per row of X_q (KJ = 32 / EB
// elements of j per chunk: 16 BF16 or 32 e4m3): 32 KB with ROWS = 256 (two
// 128-row tiles, 4 chunks) for modes with I > 128, and for short modes
// ROWS = 128 (one tile) with 8 chunks (32 KB) in BF16, 4 chunks (16 KB) in
// e4m3, whose per-slice scales need slices of whole stages (a 4-chunk stage,
// 128 j, divides every slice length that is a multiple of 128).  Layouts in shared memory: mode 1 (L = 1) one 2-D box
// {ROWS i, SBJ j}, smem [jj][ROWS]; strided views one 3-D box {KJ l, ROWS i, 1 r}
// per chunk, smem [chunk][i][32 bytes].  The transform warps pack each row's
// chunk into eight 32-bit words (element order = K order) and store them into
// tensor memory as the A operand; they also build the stacked [W_hi; W_lo]
// B tiles.  The contraction over j is split over CTAs in contiguous ranges of
// stages, so that a CTA meets few slice boundaries: at each one the MMA issuer
// commits the slice's accumulator, the holding warps read it, multiply it by
// the slice's scale and add it into FP32 registers, and hand it back.
constexpr int LP_XFORM = 256;              // warps 0-7
constexpr int LP_THREADS = LP_XFORM + 64;  // + producer (warp 8) and MMA issuer (warp 9)
constexpr int LP_A_STAGES = 2;
constexpr int LP_A_SLOT_COLS = 8;          // 128 lanes x 32 bytes: eight 32-bit columns
constexpr int LP_D_COL0 = LP_A_STAGES * 8 * LP_A_SLOT_COLS;   // 8 slots per stage

__host__ __device__ constexpr int lp_nks(int eb, int tiles) {
  return (tiles == 1 && eb == 2) ? 8 : 4;
}

template <int EB, int NPAD, int TILES>
struct LpGeo {
  static constexpr int KJ = 32 / EB;                      // j per K step (one MMA)
  static constexpr int ROWS = 128 * TILES;
  // K steps per stage: 4 with two tiles (32 KB); 8 with one tile in BF16 (32 KB,
  // the two warpgroups filling four A slots each), 4 in e4m3 (whole-stage slices)
  static constexpr int NKS = lp_nks(EB, TILES);
  static constexpr int STAGE_BYTES = ROWS * NKS * 32;
  static constexpr int SBJ = KJ * NKS;                    // j per stage
  static constexpr int D_COLS = 2 * NPAD;                 // hi and lo halves of a tile's accumulator
  static constexpr int W_RAW = SBJ * NPAD;                // FP32 raw W floats per stage
  static constexpr int B_BYTES = NKS * 2 * NPAD * 32;     // stacked B tiles of one stage
  static constexpr size_t FIXED = (size_t)LP_A_STAGES * B_BYTES + 2048;
  static constexpr size_t PER_STAGE = (size_t)STAGE_BYTES + (size_t)W_RAW * 4;
  static constexpr int FIT = (int)((232448 - 1024 - FIXED) / PER_STAGE);
  static constexpr int X_STAGES = FIT < 6 ? FIT : 6;
  static_assert(LP_D_COL0 + TILES * D_COLS <= 512, "tensor memory overflow");
  static_assert(X_STAGES >= 2, "stage ring does not fit shared memory");
};

template <int EB, int NPAD, int TILES>
struct __align__(1024) LpSketchSmem {
  using G = LpGeo<EB, NPAD, TILES>;
  unsigned char x[G::X_STAGES][G::STAGE_BYTES];
  float wraw[G::X_STAGES][G::W_RAW];         // TMA box [k][SBJ j], rows k >= K zero-filled
  unsigned char b[LP_A_STAGES][G::B_BYTES];  // per K step: [hi rows | lo rows] in the canonical layout
  uint64_t full_x[G::X_STAGES], empty_x[G::X_STAGES];
  uint64_t full_a[LP_A_STAGES], empty_a[LP_A_STAGES];
  uint64_t seg_full, seg_empty;
  uint64_t drain;                            // arrives when every MMA this CTA issued has completed
  uint32_t tmem_base;
  int abort_flag;
};

// B tile of one K step (N = 2 NPAD rows x 32 bytes, K-major, no swizzle): byte
// (n >> 3) * 256 + (b >> 4) * 128 + (n & 7) * 16 + (b & 15) for byte b of row n,
// i.e. 8-row x 16-byte core matrices with LBO = 128 (K direction) and
// SBO = 256 (N direction); rows NPAD.. hold the lo parts.
__device__ __forceinline__ int lp_b_off(int n, int byte) {
  return (n >> 3) * 256 + (byte >> 4) * 128 + (n & 7) * 16 + (byte & 15);
}

// scale_mode: 0 none; 1 per column slice (n < N), slice = j / slice_len;
// 2 per row (n = N), row i scaled by scale[i].
template <int EB, int NPAD, bool M1, int TILES>
__global__ void __launch_bounds__(LP_THREADS, 1)
tc_sketch_lp_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmW, int I,
                    int64_t L, int64_t J, int K, float* __restrict__ part, const float* __restrict__ scale,
                    int scale_mode, int64_t slice_len, DevStatus* st) {
  using G = LpGeo<EB, NPAD, TILES>;
  constexpr int X_STAGES = G::X_STAGES, ROWS = G::ROWS, SBJ = G::SBJ, KJ = G::KJ, NKS = G::NKS;
  constexpr int D_COLS = G::D_COLS;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  LpSketchSmem<EB, NPAD, TILES>& sm = *reinterpret_cast<LpSketchSmem<EB, NPAD, TILES>*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int split = blockIdx.x;
  const int i0 = blockIdx.y * ROWS;
  const int rows = min(ROWS, I - i0);
  const int mt = (rows + 127) / 128;
  // contiguous ranges of stages per CTA
  const int64_t nblk = (J + SBJ - 1) / SBJ, nsplit = gridDim.x;
  const int64_t per = (nblk + nsplit - 1) / nsplit;
  const int64_t kb0 = (int64_t)split * per;
  const int nkb = kb0 < nblk ? (int)std::min<int64_t>(per, nblk - kb0) : 0;
  auto stage_j = [&](int kb) -> int64_t { return (kb0 + kb) * SBJ; };
  auto seg_of = [&](int kb) -> int64_t { return scale_mode == 1 ? stage_j(kb) / slice_len : 0; };
  auto seg_last = [&](int kb) -> bool { return kb == nkb - 1 || seg_of(kb + 1) != seg_of(kb); };
  constexpr uint32_t idesc = EB == 2 ? idesc_bf16(128, 2 * NPAD) : idesc_e4m3(128, 2 * NPAD);
  // warps holding accumulators: the tile's warpgroup (TILES = 2), warpgroup 0 (TILES = 1)
  constexpr int HOLDERS = 128 * TILES;

  if (tid == 0) {
    for (int s = 0; s < X_STAGES; ++s) {
      mbar_init(&sm.full_x[s], 1);
      mbar_init(&sm.empty_x[s], LP_XFORM);
    }
    for (int a = 0; a < LP_A_STAGES; ++a) {
      mbar_init(&sm.full_a[a], LP_XFORM);
      mbar_init(&sm.empty_a[a], 1);
    }
    mbar_init(&sm.seg_full, 1);
    mbar_init(&sm.seg_empty, HOLDERS);
    mbar_init(&sm.drain, 1);
    sm.abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == 9) {
    tmem_alloc(&sm.tmem_base, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm.tmem_base;
  volatile int* abort_flag = &sm.abort_flag;
  bool ok = true;
  int issued = 0;

  if (warp == 8) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      const uint32_t bytes = (uint32_t)G::STAGE_BYTES + (uint32_t)(G::W_RAW * 4);
      for (int kb = 0; kb < nkb && ok; ++kb) {
        const int s = kb % X_STAGES;
        if (!mbar_wait(&sm.empty_x[s], ((uint32_t)(kb / X_STAGES) & 1u) ^ 1u, abort_flag)) { ok = false; break; }
        issued = kb + 1;
        mbar_arrive_expect_tx(&sm.full_x[s], bytes);
        const int64_t jt = stage_j(kb);
        if (M1) {
          tma_load_2d(sm.x[s], &tmX, i0, (int)jt, &sm.full_x[s]);
        } else {
#pragma unroll
          for (int c = 0; c < NKS; ++c) {
            const int64_t jc = jt + (int64_t)KJ * c, rc = jc / L;
            tma_load_3d(sm.x[s] + c * ROWS * 32, &tmX, (int)(jc - rc * L), i0, (int)rc, &sm.full_x[s]);
          }
        }
        tma_load_2d(sm.wraw[s], &tmW, (int)jt, 0, &sm.full_x[s]);
      }
    }
  } else if (warp == 9) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int seg = 0;
      for (int kb = 0; kb < nkb && ok; ++kb) {
        const bool first = kb == 0 || seg_of(kb) != seg_of(kb - 1);
        if (first && kb > 0) {                          // the holders have drained the last slice
          if (!mbar_wait(&sm.seg_empty, (uint32_t)(seg - 1) & 1u, abort_flag)) { ok = false; break; }
        }
        const int a = kb % LP_A_STAGES;
        if (!mbar_wait(&sm.full_a[a], (uint32_t)(kb / LP_A_STAGES) & 1u, abort_flag)) { ok = false; break; }
        tc_fence_after();
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int t = u / NKS, c = u % NKS;
          if (t >= mt) continue;
          const uint32_t d = tmem + (uint32_t)(LP_D_COL0 + t * D_COLS);
          const uint32_t at = tmem + (uint32_t)(a * 8 * LP_A_SLOT_COLS + u * LP_A_SLOT_COLS);
          const uint64_t db = smem_desc_kmajor_nosw(smem_u32(sm.b[a] + c * 2 * NPAD * 32), 128, 256);
          const uint32_t acc = (first && c == 0) ? 0u : 1u;
          if (EB == 2) mma_bf16_ts(d, at, db, idesc, acc);
          else mma_e4m3_ts(d, at, db, idesc, acc);
        }
        mma_commit(&sm.empty_a[a]);
        if (seg_last(kb)) {
          mma_commit(&sm.seg_full);
          ++seg;
        }
      }
      mma_commit(&sm.drain);
    }
  } else {
    // ------------------------------------------------------------ transform (warps 0-7)
    const int quad = warp & 3, wg = warp >> 2;
    const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
    const int row_in_tile = quad * 32 + lane;
    const bool holder = TILES == 2 || wg == 0;
    const int ht = TILES == 2 ? wg : 0;                 // the tile this thread holds
    float acc[NPAD];
#pragma unroll
    for (int k = 0; k < NPAD; ++k) acc[k] = 0.f;
    int seg = 0;
    auto drain = [&](float s) -> bool {
      if (!mbar_wait(&sm.seg_full, (uint32_t)seg & 1u, abort_flag)) return false;
      tc_fence_after();
      if (ht < mt) {
#pragma unroll
        for (int c0 = 0; c0 < NPAD; c0 += 16) {
          uint32_t vh[16], vl[16];
          const uint32_t col = tmem + lane_base + (uint32_t)(LP_D_COL0 + ht * D_COLS + c0);
          tmem_ld_x16(col, vh);
          tmem_ld_x16(col + NPAD, vl);
          tmem_wait_ld();
#pragma unroll
          for (int c = 0; c < 16; ++c) acc[c0 + c] = fmaf(s, __uint_as_float(vh[c]) + __uint_as_float(vl[c]), acc[c0 + c]);
        }
      }
      tc_fence_before();
      mbar_arrive(&sm.seg_empty);
      ++seg;
      return true;
    };
    for (int kb = 0; kb < nkb && ok; ++kb) {
      const int s = kb % X_STAGES, a = kb % LP_A_STAGES;
      if (holder && kb > 0 && seg_of(kb) != seg_of(kb - 1)) {
        if (!drain(scale_mode == 1 ? scale[seg_of(kb - 1)] : 1.f)) { ok = false; break; }
      }
      if (!mbar_wait(&sm.empty_a[a], ((uint32_t)(kb / LP_A_STAGES) & 1u) ^ 1u, abort_flag)) { ok = false; break; }
      tc_fence_after();
      if (!mbar_wait(&sm.full_x[s], (uint32_t)(kb / X_STAGES) & 1u, abort_flag)) { ok = false; break; }
      // A slots of this warpgroup: u = 4 wg .. 4 wg + 3, (tile u / NKS, chunk u % NKS)
#pragma unroll
      for (int uu = 0; uu < 4; ++uu) {
        const int u = 4 * wg + uu;
        const int t = u / NKS, c = u % NKS;
        if (t < mt) {
          const int r = t * 128 + row_in_tile;
          uint32_t w[8];
          if (M1) {
            // column r of the [jj][ROWS] tile, elements jj = c KJ .. c KJ + KJ - 1
            const unsigned char* xb = sm.x[s] + ((size_t)c * KJ * ROWS + r) * EB;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              if (EB == 2) {
                const uint32_t lo16 = *reinterpret_cast<const uint16_t*>(xb + (size_t)(2 * q) * ROWS * 2);
                const uint32_t hi16 = *reinterpret_cast<const uint16_t*>(xb + (size_t)(2 * q + 1) * ROWS * 2);
                w[q] = lo16 | (hi16 << 16);
              } else {
                uint32_t v = 0;
#pragma unroll
                for (int e = 0; e < 4; ++e) v |= (uint32_t)xb[(size_t)(4 * q + e) * ROWS] << (8 * e);
                w[q] = v;
              }
            }
          } else {
            const uint4* xr = reinterpret_cast<const uint4*>(sm.x[s] + (size_t)c * ROWS * 32 + (size_t)r * 32);
            const uint4 p0 = xr[0], p1 = xr[1];
            w[0] = p0.x; w[1] = p0.y; w[2] = p0.z; w[3] = p0.w;
            w[4] = p1.x; w[5] = p1.y; w[6] = p1.z; w[7] = p1.w;
          }
          if (r >= rows) {
#pragma unroll
            for (int q = 0; q < 8; ++q) w[q] = 0u;
          }
          tmem_st_x8(tmem + lane_base + (uint32_t)(a * 8 * LP_A_SLOT_COLS + u * LP_A_SLOT_COLS), w);
        }
      }
      // stacked B tiles: work item = (chunk c, row n < NPAD, 16-byte half h); the
      // raw W tile is [k][SBJ j] FP32
      for (int it = tid; it < NKS * NPAD * 2; it += LP_XFORM) {
        const int h = it & 1, n = (it >> 1) % NPAD, c = (it >> 1) / NPAD;
        constexpr int PER16 = 16 / EB;                  // elements per 16-byte half
        const float* wr = sm.wraw[s] + (size_t)n * SBJ + c * KJ + h * PER16;
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) { hw[q] = 0u; lw[q] = 0u; }
#pragma unroll
        for (int e = 0; e < PER16; ++e) {
          const float v = n < K ? wr[e] : 0.f;
          const uint32_t hb = Fmt<EB>::bits(v);
          const uint32_t lb = Fmt<EB>::bits(v - Fmt<EB>::value(hb));
          hw[(e * EB) >> 2] |= hb << (8 * ((e * EB) & 3));
          lw[(e * EB) >> 2] |= lb << (8 * ((e * EB) & 3));
        }
        unsigned char* bt = sm.b[a] + c * 2 * NPAD * 32;
        *reinterpret_cast<uint4*>(bt + lp_b_off(n, 16 * h)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4*>(bt + lp_b_off(n + NPAD, 16 * h)) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
      }
      fence_proxy_async_smem();
      tmem_wait_st();
      tc_fence_before();
      mbar_arrive(&sm.full_a[a]);
      mbar_arrive(&sm.empty_x[s]);
    }
    // ------------------------------------------------------------ last slice and epilogue
    if (ok && holder && nkb > 0) ok = drain(scale_mode == 1 ? scale[seg_of(nkb - 1)] : 1.f);
    if (ok && holder && ht < mt) {
      const int64_t i = i0 + ht * 128 + row_in_tile;
      const float rs = (scale_mode == 2 && i < I) ? scale[i] : 1.f;
#pragma unroll
      for (int k = 0; k < NPAD; ++k)
        if (k < K && i < I) part[((int64_t)split * K + k) * I + i] = acc[k] * rs;
    }
  }
  if (!ok) {
    *abort_flag = 1;
    set_error(st, RHOSVD_ETIMEOUT);
  }
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
      while (!mbar_try_wait(&sm.drain, 0) && globaltimer_ns() - t0 < kWaitLimitNs) {
      }
    }
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// ---------------------------------------------------------------- mode-1 TTM Out = X_q,(1)^T M
// Out(j, k) = s(j) sum_i X_q(i, j) M(i, k) with j the columns of X_(1) (L = 1).
// Stage: 128 rows j x 128 bytes of i (BI = 64 BF16 or 128 e4m3 elements, four
// K steps), one 2-D box {BI i, 128 j} with 128-byte swizzle; each transform
// thread (row j = TMEM lane) reads its row's eight 16-byte pieces (piece c at
// c ^ (j & 7)) and stores them into tensor memory as the A operand.  The M
// tile comes as FP32 boxes {32 i, NPAD k} (128-byte swizzle) and is split into
// the stacked [M_hi; M_lo] B tiles.  Accumulation in tensor-memory segments of
// LP_SEG stages summed in FP32 registers (the tensor core rounds its FP32
// accumulator toward zero), as in the FP32 TTM.  Warps: 0-7 transform (two
// warpgroups, alternate stages), 8-11 epilogue, 12 producer, 13 MMA issuer.
constexpr int LPT_XFORM = 256, LPT_EPI = 128;
constexpr int LPT_PRODUCER = 12, LPT_MMA = 13;
constexpr int LPT_THREADS = LPT_XFORM + LPT_EPI + 64;
constexpr int LPT_A_STAGES = 2;
constexpr int LPT_A_COLS = 32;             // four K steps x eight 32-bit columns
constexpr int LPT_D_COL0 = LPT_A_STAGES * LPT_A_COLS;
constexpr int LP_SEG = 2;

template <int EB, int NPAD>
struct LptGeo {
  static constexpr int BI = 128 / EB;                     // i per stage
  static constexpr int KJ = 32 / EB;                      // i per K step
  static constexpr int NBOX = BI / 32;                    // FP32 M boxes of 32 i per stage
  static constexpr int M_RAW = NPAD * BI;                 // floats
  static constexpr int B_BYTES = 4 * 2 * NPAD * 32;
  static constexpr int D_COLS = 2 * NPAD;
  static constexpr int NBUF_FIT = (512 - LPT_D_COL0) / D_COLS;
  static constexpr int NBUF = NBUF_FIT < 4 ? NBUF_FIT : 4;
  static constexpr size_t FIXED = (size_t)LPT_A_STAGES * B_BYTES + 4 * 32 * 17 * 4 + 2048;
  static constexpr size_t PER_STAGE = 16384 + (size_t)M_RAW * 4;
  static constexpr int FIT = (int)((232448 - 1024 - FIXED) / PER_STAGE);
  static constexpr int X_STAGES = FIT < 8 ? FIT : 8;
  static_assert(X_STAGES >= 2, "stage ring does not fit shared memory");
};

template <int EB, int NPAD>
struct __align__(1024) LpTtmSmem {
  using G = LptGeo<EB, NPAD>;
  unsigned char x[G::X_STAGES][16384];       // [j][128 bytes of i], 128B swizzle
  float mraw[G::X_STAGES][G::M_RAW];         // [box][k][32 i], 128B swizzle
  unsigned char b[LPT_A_STAGES][G::B_BYTES];
  float ostage[4][32 * 17];
  uint64_t full_x[G::X_STAGES], empty_x[G::X_STAGES];
  uint64_t full_a[LPT_A_STAGES], empty_a[LPT_A_STAGES];
  uint64_t d_full[G::NBUF], d_empty[G::NBUF];
  uint64_t drain;
  uint32_t tmem_base;
  int abort_flag;
};

template <int EB, int NPAD>
__global__ void __launch_bounds__(LPT_THREADS, 1)
tc_ttm_lp_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmM, int I,
                 int64_t J, int K, float* __restrict__ out, int64_t o_k, int64_t o_r,
                 const float* __restrict__ scale, int64_t slice_len, DevStatus* st) {
  using G = LptGeo<EB, NPAD>;
  constexpr int X_STAGES = G::X_STAGES, BI = G::BI, KJ = G::KJ, NBUF = G::NBUF, D_COLS = G::D_COLS;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  LpTtmSmem<EB, NPAD>& sm = *reinterpret_cast<LpTtmSmem<EB, NPAD>*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = (int)((J + 127) / 128);
  const int nst = (I + BI - 1) / BI;
  const int nseg = (nst + LP_SEG - 1) / LP_SEG;
  constexpr uint32_t idesc = EB == 2 ? idesc_bf16(128, 2 * NPAD) : idesc_e4m3(128, 2 * NPAD);

  if (tid == 0) {
    for (int s = 0; s < X_STAGES; ++s) {
      mbar_init(&sm.full_x[s], 1);
      mbar_init(&sm.empty_x[s], 128);
    }
    for (int a = 0; a < LPT_A_STAGES; ++a) {
      mbar_init(&sm.full_a[a], 128);
      mbar_init(&sm.empty_a[a], 1);
    }
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(&sm.d_full[b], 1);
      mbar_init(&sm.d_empty[b], LPT_EPI);
    }
    mbar_init(&sm.drain, 1);
    sm.abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == LPT_MMA) {
    tmem_alloc(&sm.tmem_base, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm.tmem_base;
  volatile int* abort_flag = &sm.abort_flag;
  bool ok = true;
  const int my_tiles = (ntiles > (int)blockIdx.x) ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int total = my_tiles * nst;
  int issued = 0;

  if (warp == LPT_PRODUCER) {
    if (lane == 0) {
      const uint32_t bytes = 16384u + (uint32_t)(G::M_RAW * 4);
      for (int g = 0; g < total && ok; ++g) {
        const int s = g % X_STAGES;
        if (!mbar_wait(&sm.empty_x[s], ((uint32_t)(g / X_STAGES) & 1u) ^ 1u, abort_flag)) { ok = false; break; }
        const int tile = (int)blockIdx.x + (g / nst) * (int)gridDim.x;
        const int ib = (g % nst) * BI;
        issued = g + 1;
        mbar_arrive_expect_tx(&sm.full_x[s], bytes);
        tma_load_2d(sm.x[s], &tmX, ib, tile * 128, &sm.full_x[s]);
#pragma unroll
        for (int bx = 0; bx < G::NBOX; ++bx) tma_load_2d(sm.mraw[s] + bx * NPAD * 32, &tmM, ib + 32 * bx, 0, &sm.full_x[s]);
      }
    }
  } else if (warp == LPT_MMA) {
    if (lane == 0) {
      int ks0 = 0, gs = 0;                             // stage within the tile, segment over the CTA
      for (int g = 0; g < total && ok; ++g) {
        const int buf = gs % NBUF;
        const bool seg_first = (ks0 % LP_SEG) == 0, seg_end = (ks0 % LP_SEG) == LP_SEG - 1 || ks0 == nst - 1;
        if (seg_first) {
          if (!mbar_wait_fast(&sm.d_empty[buf], ((uint32_t)(gs / NBUF) & 1u) ^ 1u, abort_flag)) { ok = false; break; }
        }
        const int a = g % LPT_A_STAGES;
        if (!mbar_wait_fast(&sm.full_a[a], (uint32_t)(g / LPT_A_STAGES) & 1u, abort_flag)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(LPT_D_COL0 + buf * D_COLS);
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const uint32_t at = tmem + (uint32_t)(a * LPT_A_COLS + ks * 8);
          const uint64_t db = smem_desc_kmajor_nosw(smem_u32(sm.b[a] + ks * 2 * NPAD * 32), 128, 256);
          const uint32_t acc = (!seg_first || ks > 0) ? 1u : 0u;
          if (EB == 2) mma_bf16_ts(d, at, db, idesc, acc);
          else mma_e4m3_ts(d, at, db, idesc, acc);
        }
        mma_commit(&sm.empty_a[a]);
        if (seg_end) {
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
    const int row = quad * 32 + lane;
    const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
    const int xt = tid & 127;
    for (int g = wg; g < total && ok; g += 2) {
      const int s = g % X_STAGES, a = g % LPT_A_STAGES;
      if (!mbar_wait(&sm.full_x[s], (uint32_t)(g / X_STAGES) & 1u, abort_flag)) { ok = false; break; }
      if (!mbar_wait(&sm.empty_a[a], ((uint32_t)(g / LPT_A_STAGES) & 1u) ^ 1u, abort_flag)) { ok = false; break; }
      tc_fence_after();
      const uint4* xr = reinterpret_cast<const uint4*>(sm.x[s] + row * 128);
      uint32_t w0[16], w1[16];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const uint4 v = xr[c ^ (row & 7)];
        w0[4 * c] = v.x; w0[4 * c + 1] = v.y; w0[4 * c + 2] = v.z; w0[4 * c + 3] = v.w;
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const uint4 v = xr[(c + 4) ^ (row & 7)];
        w1[4 * c] = v.x; w1[4 * c + 1] = v.y; w1[4 * c + 2] = v.z; w1[4 * c + 3] = v.w;
      }
      const uint32_t col = tmem + (uint32_t)(a * LPT_A_COLS) + lane_base;
      tmem_st_x16(col, w0);
      tmem_st_x16(col + 16, w1);
      // stacked B tiles: work item (K step ks, row n < NPAD, 16-byte half h)
      for (int it = xt; it < 4 * NPAD * 2; it += 128) {
        const int h = it & 1, n = (it >> 1) % NPAD, ks = (it >> 1) / NPAD;
        constexpr int PER16 = 16 / EB;
        uint32_t hw[4] = {0u, 0u, 0u, 0u}, lw[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int e = 0; e < PER16; ++e) {
          const int i = ks * KJ + h * PER16 + e;             // within the stage
          const int bx = i >> 5, ii = i & 31;
          const float v = n < K ? sm.mraw[s][bx * NPAD * 32 + n * 32 + (((ii >> 2) ^ (n & 7)) << 2) + (ii & 3)] : 0.f;
          const uint32_t hb = Fmt<EB>::bits(v);
          const uint32_t lb = Fmt<EB>::bits(v - Fmt<EB>::value(hb));
          hw[(e * EB) >> 2] |= hb << (8 * ((e * EB) & 3));
          lw[(e * EB) >> 2] |= lb << (8 * ((e * EB) & 3));
        }
        unsigned char* bt = sm.b[a] + ks * 2 * NPAD * 32;
        *reinterpret_cast<uint4*>(bt + lp_b_off(n, 16 * h)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4*>(bt + lp_b_off(n + NPAD, 16 * h)) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
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
          const uint32_t dcol = tmem + lane_base + (uint32_t)(LPT_D_COL0 + buf * D_COLS + 16 * c0);
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
      const int64_t tj0 = (int64_t)tile * 128;
      const int64_t j = tj0 + quad * 32 + lane;
      const float rs = (scale != nullptr && j < J) ? scale[j / slice_len] : 1.f;
      if (o_k == 1) {
        // rows of the output contiguous in k: stage 32 rows x 16 columns per warp
        float* stg = sm.ostage[quad];
        const int64_t jw = tj0 + quad * 32;
#pragma unroll
        for (int c0 = 0; c0 < NPAD; c0 += 16) {
#pragma unroll
          for (int c = 0; c < 16; ++c) stg[lane * 17 + c] = acc[c0 + c] * rs;
          __syncwarp();
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int rr = 2 * q + (lane >> 4), cc = lane & 15;
            const int64_t jr = jw + rr;
            if (c0 + cc < K && jr < J) out[jr * o_r + c0 + cc] = stg[rr * 17 + cc];
          }
          __syncwarp();
        }
      } else {
#pragma unroll
        for (int k = 0; k < NPAD; ++k)
          if (k < K && j < J) out[j * o_r + (int64_t)k * o_k] = acc[k] * rs;
      }
    }
  }
  if (!ok) {
    *abort_flag = 1;
    set_error(st, RHOSVD_ETIMEOUT);
  }
  __syncthreads();
  if (sm.abort_flag && warp == LPT_PRODUCER && lane == 0) {
    for (int s = 0; s < X_STAGES && s < issued; ++s) {
      const int g_last = s + X_STAGES * ((issued - 1 - s) / X_STAGES);
      const uint64_t t0 = globaltimer_ns();
      while (!mbar_try_wait(&sm.full_x[s], (uint32_t)(g_last / X_STAGES) & 1u) &&
             globaltimer_ns() - t0 < kWaitLimitNs) {
      }
    }
  }
  if (warp == LPT_MMA) {
    if (sm.abort_flag && lane == 0) {
      const uint64_t t0 = globaltimer_ns();
      while (!mbar_try_wait(&sm.drain, 0) && globaltimer_ns() - t0 < kWaitLimitNs) {
      }
    }
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

}  // namespace

// ---------------------------------------------------------------- host side
namespace {

template <class F>
cudaError_t by_npad(int K, F&& f) {
  switch (((K + 15) / 16) * 16) {
    case 16: return f(std::integral_constant<int, 16>{});
    case 32: return f(std::integral_constant<int, 32>{});
    case 48: return f(std::integral_constant<int, 48>{});
    default: return f(std::integral_constant<int, 64>{});
  }
}

struct LpPlan {
  int tiles, mgroups, splits, sbj;
};
LpPlan plan_lp(int64_t I, int64_t J, int eb) {
  LpPlan p;
  p.tiles = I > 128 ? 2 : 1;
  p.mgroups = (int)((I + 128 * p.tiles - 1) / (128 * p.tiles));
  p.sbj = lp_nks(eb, p.tiles) * (32 / eb);
  const int64_t nblk = (J + p.sbj - 1) / p.sbj;
  p.splits = (int)std::min<int64_t>(std::max<int64_t>(1, device_sms() / p.mgroups), nblk);
  return p;
}

}  // namespace

cudaError_t launch_quantize(const float* X, int64_t n, int64_t slice_len, int eb, void* Xq, float* scale,
                            unsigned int* amax, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  if ((eb != 1 && eb != 2) || slice_len < 1 || n % slice_len != 0) return cudaErrorInvalidValue;
  const int64_t nslices = n / slice_len;
  const unsigned threads = 256;
  const unsigned blocks = (unsigned)((n + 16 * threads - 1) / (16 * threads));
  if (eb == 1) {
    cudaError_t e = cudaMemsetAsync(amax, 0, sizeof(unsigned int) * nslices, st);
    if (e != cudaSuccess) return e;
    const int64_t per_block = 256 * 64;
    const dim3 g((unsigned)std::min<int64_t>((slice_len + per_block - 1) / per_block, 1024),
                 (unsigned)std::min<int64_t>(nslices, 65535));
    slice_amax_kernel<<<g, 256, 0, st>>>(X, slice_len, nslices, amax);
    slice_scale_kernel<<<(unsigned)((nslices + 255) / 256), 256, 0, st>>>(amax, nslices, scale);
    quantize_kernel<1><<<blocks, threads, 0, st>>>(X, n, slice_len, scale, static_cast<unsigned char*>(Xq));
  } else {
    quantize_kernel<2><<<blocks, threads, 0, st>>>(X, n, slice_len, nullptr, static_cast<unsigned char*>(Xq));
  }
  return cudaGetLastError();
}

cudaError_t launch_round_to_format(float* a, int64_t n, int eb, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (eb == 2) round_to_format_kernel<2><<<blocks, 256, 0, st>>>(a, n);
  else if (eb == 1) round_to_format_kernel<1><<<blocks, 256, 0, st>>>(a, n);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_omega_rounded(uint64_t seed, uint32_t stream_id, int64_t rows, int cols, float* out,
                                 int64_t ld, int eb, cudaStream_t st) {
  if (rows == 0 || cols == 0) return cudaSuccess;
  const dim3 grid((unsigned)((rows + 255) / 256), (unsigned)((cols + 3) / 4));
  if (eb == 2) omega_rounded_kernel<2><<<grid, 256, 0, st>>>(seed, stream_id, rows, cols, out, ld);
  else if (eb == 1) omega_rounded_kernel<1><<<grid, 256, 0, st>>>(seed, stream_id, rows, cols, out, ld);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

bool tc_sketch_lp_supported(const View& x, int eb, int K, int scale_mode, int64_t slice_len) {
  if (eb != 1 && eb != 2) return false;
  const int64_t J = x.L * x.Rt;
  const int kj = 32 / eb, sbj = lp_nks(eb, x.I > 128 ? 2 : 1) * kj;
  if (K < 1 || K > 64 || x.I < 1 || x.I >= (int64_t(1) << 31) || J < 1 || J >= (int64_t(1) << 31) || J % 4 != 0)
    return false;
  if (scale_mode == 1 && (slice_len < 1 || slice_len % sbj != 0)) return false;
  if (x.L == 1) return x.s_i == 1 && x.s_r == x.I && (x.I * eb) % 16 == 0;
  if (x.L % kj != 0 || (x.s_i * eb) % 16 != 0 || (x.Rt > 1 && (x.s_r * eb) % 16 != 0)) return false;
  return x.L < (int64_t(1) << 31) && x.Rt < (int64_t(1) << 31);
}

size_t sketch_lp_scratch_floats(int64_t I, int K, int64_t J, int eb) {
  const LpPlan p = plan_lp(I, J, eb);
  return (size_t)p.splits * (size_t)K * (size_t)I;
}

cudaError_t launch_tc_sketch_lp(const View& x, const void* xq, int eb, const float* W, int K, float* Y,
                                int64_t ldy, const float* scale, int scale_mode, int64_t slice_len, float* part,
                                DevStatus* st, cudaStream_t stream) {
  if (!tc_sketch_lp_supported(x, eb, K, scale_mode, slice_len) || st == nullptr) return cudaErrorNotSupported;
  if ((reinterpret_cast<uintptr_t>(xq) & 15) || (reinterpret_cast<uintptr_t>(W) & 15)) return cudaErrorNotSupported;
  const int64_t I = x.I, J = x.L * x.Rt;
  const LpPlan pl = plan_lp(I, J, eb);
  const int rows = 128 * pl.tiles, kj = 32 / eb;
  const uint32_t npad = (uint32_t)(((K + 15) / 16) * 16);
  CUtensorMap tmX, tmW;
  {
    const uint64_t dims[2] = {(uint64_t)J, (uint64_t)K};
    const uint64_t strides[1] = {(uint64_t)J};
    const uint32_t box[2] = {(uint32_t)pl.sbj, npad};
    if (!make_tmap_f32(&tmW, W, 2, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_NONE)) return cudaErrorNotSupported;
  }
  const bool m1 = x.L == 1;
  if (m1) {
    const uint64_t dims[2] = {(uint64_t)I, (uint64_t)J};
    const uint64_t strides[1] = {(uint64_t)I};
    const uint32_t box[2] = {(uint32_t)rows, (uint32_t)pl.sbj};
    if (!make_tmap_u(&tmX, xq, eb, 2, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_NONE)) return cudaErrorNotSupported;
  } else {
    const uint64_t dims[3] = {(uint64_t)x.L, (uint64_t)I, (uint64_t)x.Rt};
    const uint64_t strides[2] = {(uint64_t)x.s_i, x.Rt > 1 ? (uint64_t)x.s_r : (uint64_t)x.s_i * (uint64_t)I};
    const uint32_t box[3] = {(uint32_t)kj, (uint32_t)rows, 1};
    if (!make_tmap_u(&tmX, xq, eb, 3, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_NONE)) return cudaErrorNotSupported;
  }
  const dim3 grid((unsigned)pl.splits, (unsigned)pl.mgroups);
  cudaError_t e = by_npad(K, [&](auto np) -> cudaError_t {
    constexpr int NP = decltype(np)::value;
    auto go = [&](auto ebc, auto m1c, auto tc) -> cudaError_t {
      constexpr int EB = decltype(ebc)::value, TL = decltype(tc)::value;
      constexpr bool M1 = decltype(m1c)::value;
      const size_t smem = sizeof(LpSketchSmem<EB, NP, TL>) + 1024;
      static_assert(sizeof(LpSketchSmem<EB, NP, TL>) + 1024 <= 232448, "sketch stages exceed shared memory");
      cudaError_t e2 = allow_dynamic_smem((const void*)tc_sketch_lp_kernel<EB, NP, M1, TL>, smem);
      if (e2 != cudaSuccess) return e2;
      tc_sketch_lp_kernel<EB, NP, M1, TL><<<grid, LP_THREADS, smem, stream>>>(tmX, tmW, (int)I, x.L, J, K, part, scale,
                                                                             scale_mode, slice_len, st);
      return cudaGetLastError();
    };
    using I1 = std::integral_constant<int, 1>;
    using I2 = std::integral_constant<int, 2>;
    using BT = std::true_type;
    using BF = std::false_type;
    if (eb == 2) {
      if (m1) return pl.tiles == 2 ? go(I2{}, BT{}, I2{}) : go(I2{}, BT{}, I1{});
      return pl.tiles == 2 ? go(I2{}, BF{}, I2{}) : go(I2{}, BF{}, I1{});
    }
    if (m1) return pl.tiles == 2 ? go(I1{}, BT{}, I2{}) : go(I1{}, BT{}, I1{});
    return pl.tiles == 2 ? go(I1{}, BF{}, I2{}) : go(I1{}, BF{}, I1{});
  });
  if (e != cudaSuccess) return e;
  return launch_reduce_partials_f(part, pl.splits, I, K, Y, ldy, stream);
}

bool tc_ttm_lp_supported(int64_t I, int64_t J, int eb, int K, int64_t ldm) {
  if (eb != 1 && eb != 2) return false;
  if (K < 1 || K > 64 || I < 1 || I >= (int64_t(1) << 31) || J < 1 || J >= (int64_t(1) << 38)) return false;
  if ((J + 127) / 128 >= (int64_t(1) << 31)) return false;
  return (I * eb) % 16 == 0 && ldm % 4 == 0 && ldm >= I;
}

cudaError_t launch_tc_ttm_lp(const void* xq, int eb, int64_t I, int64_t J, const float* M, int64_t ldm, int K,
                             float* out, int64_t o_k, int64_t o_r, const float* scale, int64_t slice_len,
                             DevStatus* st, cudaStream_t stream) {
  if (!tc_ttm_lp_supported(I, J, eb, K, ldm) || st == nullptr) return cudaErrorNotSupported;
  if ((reinterpret_cast<uintptr_t>(xq) & 15) || (reinterpret_cast<uintptr_t>(M) & 15)) return cudaErrorNotSupported;
  const uint32_t npad = (uint32_t)(((K + 15) / 16) * 16);
  CUtensorMap tmX, tmM;
  {
    const uint64_t dims[2] = {(uint64_t)I, (uint64_t)K};
    const uint64_t strides[1] = {(uint64_t)ldm};
    const uint32_t box[2] = {32, npad};
    if (!make_tmap_f32(&tmM, M, 2, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_128B)) return cudaErrorNotSupported;
  }
  {
    const uint64_t dims[2] = {(uint64_t)I, (uint64_t)J};
    const uint64_t strides[1] = {(uint64_t)I};
    const uint32_t box[2] = {(uint32_t)(128 / eb), 128};
    if (!make_tmap_u(&tmX, xq, eb, 2, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_128B)) return cudaErrorNotSupported;
  }
  const int ntiles = (int)((J + 127) / 128);
  const int grid = std::min(ntiles, device_sms());
  return by_npad(K, [&](auto np) -> cudaError_t {
    constexpr int NP = decltype(np)::value;
    auto go = [&](auto ebc) -> cudaError_t {
      constexpr int EB = decltype(ebc)::value;
      const size_t smem = sizeof(LpTtmSmem<EB, NP>) + 1024;
      static_assert(sizeof(LpTtmSmem<EB, NP>) + 1024 <= 232448, "TTM stages exceed shared memory");
      cudaError_t e2 = allow_dynamic_smem((const void*)tc_ttm_lp_kernel<EB, NP>, smem);
      if (e2 != cudaSuccess) return e2;
      tc_ttm_lp_kernel<EB, NP><<<grid, LPT_THREADS, smem, stream>>>(tmX, tmM, (int)I, J, K, out, o_k, o_r, scale,
                                                                    slice_len > 0 ? slice_len : J, st);
      return cudaGetLastError();
    };
    return eb == 2 ? go(std::integral_constant<int, 2>{}) : go(std::integral_constant<int, 1>{});
  });
}

}  // namespace rhosvd
