// Persistent batched R-STHOSVD (Alg. 8 with Alg. 1 per mode) for many small
// tensors of uneven sizes in one launch.
//
// Each CTA is a worker that takes the next tensor from a work queue (an atomic
// counter over a host-ordered table, largest work first) and runs the whole
// decomposition of that tensor by itself:
//   for n = 1..N on the current core S (geometry [L, I_n, Rt], J = L Rt):
//     Y = S_(n) Omega_n               (Omega_n generated in the kernel, stream n)
//     Q = orth(Y)                     (CGS2 by the CTA, Y in shared memory)
//     q times: Z = S_(n)^T Q, Z = a basis of range(Z) (one shifted CholeskyQR
//              pass, Fukaya et al. 2020), Y = S_(n) Z, Q = orth(Y)
//     B^T = S_(n)^T Q, G = B B^T, eigenvectors of G (two-sided Jacobi in one
//              warp), Ubar_R = the R leading ones
//     U_n = Q Ubar_R, S <- S x_n U_n^T through the shortcut S_(n) = Ubar_R^T B
// All arithmetic is FP32 on the CUDA cores: the tensors are small (modes up
// to 256), each contraction is a few MFLOP, and the win over one launch
// sequence per tensor is that every SM works on its own tensor with no launch
// or graph-node cost in between.  The per-CTA scratch (Z / B^T and two core
// buffers) sits in the workspace; the tiles of S, the test matrix, Q and the
// small K x K matrices sit in shared memory.
//
// Tunable per launch: threads per CTA (128 / 256 / 512), the j-chunk of the
// streamed contractions (32 / 64 columns of S_(n) per tile) and CTAs per SM;
// rhosvd_batch_tune times the feasible configurations on the batch itself.
#include <algorithm>
#include <math.h>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace rhosvd {

namespace {

constexpr int BT_GMAX = 4;      // sketch output groups (1 row x 8 columns) per thread, at most
constexpr int BT_TMAX = 4;      // TTM output groups per thread, at most
constexpr int BT_MAX_I = 256;   // largest mode size of a batched tensor
constexpr int BT_MAX_K = 32;    // largest sketch width
constexpr int BT_MAX_SWEEPS = 30;

// One tensor of the batch as the kernel sees it (device copy of the table).
struct BItem {
  const float* X;
  float* G;
  float* U[RHOSVD_MAX_MODES];
  int64_t d[RHOSVD_MAX_MODES];
  int32_t r[RHOSVD_MAX_MODES];
  int32_t K[RHOSVD_MAX_MODES];
  int32_t N;
  int32_t pad;
};

// Shared-memory carve-up (floats), identical on host and device.  The tiles
// of the streamed passes are double-buffered: the next tile is copied in
// (cp.async) while the current one is used.
struct BSmem {
  int ip, kp, jc, T, arow, abuf, wbuf;
  int as, ws, ys, ms, gs, vs, ub, red, total;
  __host__ __device__ BSmem(int imax, int kmax, int jc_, int T_) : jc(jc_), T(T_) {
    ip = imax | 1;                                  // odd pitch: conflict-free both ways
    kp = (kmax + 3) & ~3;
    arow = ip > kp + 1 ? ip : kp + 1;              // room for the odd-pitch Z tiles
    abuf = (jc * arow + 3) & ~3;
    wbuf = jc * kp;
    int o = 0;
    as = o; o += 2 * abuf;                          // 2 S tiles [jj][i] (or Z tiles [jj][k], pitch kp)
    ws = o; o += 2 * wbuf;                          // 2 Omega / Z tiles [jj][k]
    ys = o; o += ip * kp;                           // Y, Q column-major (ld ip)
    o = (o + 3) & ~3;
    ms = o; o += ip * kp;                           // Q row-major [i][k] for the TTM
    gs = o; o += kp * kp;                           // K x K Gram (col-major, ld kp)
    vs = o; o += kp * kp;                           // eigenvectors / L^-1
    ub = o; o += kp * kp;                           // Ubar (K x R, ld kp)
    red = o; o += T * 16;                           // Gram partials / rotations / scalars
    total = o;
  }
};

__device__ __forceinline__ int64_t prod_lt(const int64_t* d, int n) {
  int64_t p = 1;
  for (int k = 0; k < n; ++k) p *= d[k];
  return p;
}

__device__ __forceinline__ int tile_cols(int64_t J, int64_t j0, int jc) {
  return (int)(J - j0 < (int64_t)jc ? J - j0 : (int64_t)jc);
}

// 4-byte asynchronous global -> shared copy; an invalid element is written as
// zero (source size 0, nothing is read from src).
__device__ __forceinline__ void cp_async_f32(float* dst, const float* src, bool valid) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most one group of this thread's copies is still in flight
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Start copying the tile S_(n)(0:I, j0:j0+jc) to As[jj * arow + i] (zeros past J).
template <int T>
__device__ __forceinline__ void stage_s_tile(const float* S, int64_t L, int I, int64_t J, int64_t j0, int jc,
                                             float* As, int arow) {
  const int tid = threadIdx.x;
  const int nj = tile_cols(J, j0, jc);
  if (L == 1) {          // mode 1: the columns j0.. of S_(1) are one run of nj I floats
    const float* src = S + (int64_t)I * j0;
    const int nv = nj * I, n = jc * I;
    const int qd = T / I, rm = T - qd * I;        // a step of T elements = qd columns + rm rows
    int jj = tid / I, i = tid - jj * I;
    for (int e = tid; e < n; e += T) {
      cp_async_f32(As + jj * arow + i, e < nv ? src + e : S, e < nv);
      i += rm;
      jj += qd;
      if (i >= I) {
        i -= I;
        ++jj;
      }
    }
  } else {               // T is a multiple of jc: a thread keeps one column of the tile
    const int jj = tid % jc;
    const int64_t j = j0 + jj;
    const bool ok = jj < nj;
    const float* col = ok ? S + (j % L) + L * (int64_t)I * (j / L) : S;
    for (int i = tid / jc; i < I; i += T / jc) cp_async_f32(As + jj * arow + i, ok ? col + L * i : S, ok);
  }
}

// Start copying rows j0..j0+jc of the J x K matrix Z (ld J) to Zs[jj * pitch + k]
// for k < kfill (zeros past J and for K <= k < kfill).
template <int T>
__device__ __forceinline__ void stage_z_tile(const float* Z, int64_t J, int K, int64_t j0, int jc, int kfill,
                                             int pitch, float* Zs) {
  const int tid = threadIdx.x;
  const int jj = tid % jc;
  const bool row_ok = jj < tile_cols(J, j0, jc);
  for (int k = tid / jc; k < kfill; k += T / jc) {
    const bool ok = row_ok && k < K;
    cp_async_f32(Zs + jj * pitch + k, ok ? Z + (j0 + jj) + J * k : Z, ok);
  }
}

// body(j0, nj, Zs) for every row tile of Z (ld J) staged in shared memory, the
// next tile copied in while body runs on the current one.  A tile row holds
// K_pad = kp columns at pitch kp when the body reads float4 (zero-filled past
// K), or the K columns at the odd pitch kp + 1 (odd_pitch) when it reads single
// words with lanes on consecutive rows: then neither the copies nor the reads
// conflict in shared-memory banks.
template <int T, class F>
__device__ __forceinline__ void stream_z_tiles(const float* Z, int64_t J, int K, const BSmem& sm, float* smf,
                                               bool odd_pitch, F&& body) {
  const int jc = sm.jc, kp = sm.kp;
  const int pitch = odd_pitch ? kp + 1 : kp, kfill = odd_pitch ? K : kp;
  const int ntiles = (int)((J + jc - 1) / jc);
  __syncthreads();                                  // the staging buffers are free
  stage_z_tile<T>(Z, J, K, 0, jc, kfill, pitch, smf + sm.as);
  cp_async_commit();
  for (int t = 0; t < ntiles; ++t) {
    const int b = t & 1;
    const int64_t j0 = (int64_t)t * jc;
    if (t + 1 < ntiles) stage_z_tile<T>(Z, J, K, j0 + jc, jc, kfill, pitch, smf + sm.as + (b ^ 1) * sm.abuf);
    cp_async_commit();
    cp_async_wait_one();
    __syncthreads();
    body(j0, tile_cols(J, j0, jc), static_cast<const float*>(smf + sm.as + b * sm.abuf));
    __syncthreads();                                // the tile may be refilled
  }
}

// Y (I x K, column-major in shared memory, ld ip) = S_(n) W, with W the seeded
// Gaussian test matrix (Zg == nullptr; the omega kernel's values, stream
// `stream`) or the J x K matrix Zg in global memory (ld J).
template <int T>
__device__ void blk_sketch(const float* S, int64_t L, int64_t I, int64_t J, int K, const float* Zg, uint64_t seed,
                           uint32_t stream, const BSmem& sm, float* smf) {
  float* Ys = smf + sm.ys;
  const int tid = threadIdx.x, jc = sm.jc, kp = sm.kp, arow = sm.arow;
  const int kg = (K + 3) / 4;
  const int ng = (int)I * ((kg + 1) / 2);           // groups of one row and 8 columns
  const int ntiles = (int)((J + jc - 1) / jc);
  float acc[BT_GMAX][8];
#pragma unroll
  for (int u = 0; u < BT_GMAX; ++u)
#pragma unroll
    for (int t = 0; t < 8; ++t) acc[u][t] = 0.f;
  __syncthreads();                                  // the staging buffers are free
  stage_s_tile<T>(S, L, (int)I, J, 0, jc, smf + sm.as, arow);
  if (Zg != nullptr) stage_z_tile<T>(Zg, J, K, 0, jc, kp, kp, smf + sm.ws);
  cp_async_commit();
  for (int t = 0; t < ntiles; ++t) {
    const int b = t & 1;
    const int64_t j0 = (int64_t)t * jc;
    const float* As = smf + sm.as + b * sm.abuf;
    float* Ws = smf + sm.ws + b * sm.wbuf;
    if (t + 1 < ntiles) {                           // the next tile streams in meanwhile
      stage_s_tile<T>(S, L, (int)I, J, j0 + jc, jc, smf + sm.as + (b ^ 1) * sm.abuf, arow);
      if (Zg != nullptr) stage_z_tile<T>(Zg, J, K, j0 + jc, jc, kp, kp, smf + sm.ws + (b ^ 1) * sm.wbuf);
    }
    cp_async_commit();
    if (Zg == nullptr) {
      const int nj = tile_cols(J, j0, jc);
      for (int e = tid; e < jc * kg; e += T) {
        const int jj = e % jc, g = e / jc;
        float z[4] = {0.f, 0.f, 0.f, 0.f};
        if (jj < nj) omega_quad(seed, stream, (uint64_t)(j0 + jj), (uint32_t)g, z);
#pragma unroll
        for (int t2 = 0; t2 < 4; ++t2) Ws[jj * kp + 4 * g + t2] = (4 * g + t2 < K) ? z[t2] : 0.f;
      }
    }
    cp_async_wait_one();
    __syncthreads();
#pragma unroll
    for (int u = 0; u < BT_GMAX; ++u) {
      const int g = tid + T * u;
      if (g < ng) {
        // one row i against two 4-column groups of W: a shared load of S_(n)
        // serves 8 multiply-adds (the second group is absent at an odd kg)
        const int i = g % (int)I, c = 2 * (g / (int)I);
        if (c + 1 < kg) {
#pragma unroll 8
          for (int jj = 0; jj < jc; ++jj) {
            const float a = As[jj * arow + i];
            const float4 w0 = *reinterpret_cast<const float4*>(Ws + jj * kp + 4 * c);
            const float4 w1 = *reinterpret_cast<const float4*>(Ws + jj * kp + 4 * c + 4);
            acc[u][0] = fmaf(a, w0.x, acc[u][0]);
            acc[u][1] = fmaf(a, w0.y, acc[u][1]);
            acc[u][2] = fmaf(a, w0.z, acc[u][2]);
            acc[u][3] = fmaf(a, w0.w, acc[u][3]);
            acc[u][4] = fmaf(a, w1.x, acc[u][4]);
            acc[u][5] = fmaf(a, w1.y, acc[u][5]);
            acc[u][6] = fmaf(a, w1.z, acc[u][6]);
            acc[u][7] = fmaf(a, w1.w, acc[u][7]);
          }
        } else {
#pragma unroll 8
          for (int jj = 0; jj < jc; ++jj) {
            const float a = As[jj * arow + i];
            const float4 w0 = *reinterpret_cast<const float4*>(Ws + jj * kp + 4 * c);
            acc[u][0] = fmaf(a, w0.x, acc[u][0]);
            acc[u][1] = fmaf(a, w0.y, acc[u][1]);
            acc[u][2] = fmaf(a, w0.z, acc[u][2]);
            acc[u][3] = fmaf(a, w0.w, acc[u][3]);
          }
        }
      }
    }
    __syncthreads();                                // this tile's buffers may be refilled
  }
#pragma unroll
  for (int u = 0; u < BT_GMAX; ++u) {
    const int g = tid + T * u;
    if (g < ng) {
      const int i = g % (int)I, c = 2 * (g / (int)I);
#pragma unroll
      for (int t = 0; t < 8; ++t)
        if (4 * c + t < K) Ys[i + sm.ip * (4 * c + t)] = acc[u][t];
    }
  }
  __syncthreads();
}

// Out (J x K, global, ld J) = S_(n)^T M with M (I x K) row-major in shared memory (Ms).
template <int T>
__device__ void blk_ttm(const float* S, int64_t L, int64_t I, int64_t J, int K, float* __restrict__ out,
                        const BSmem& sm, float* smf) {
  const float* Ms = smf + sm.ms;
  const int tid = threadIdx.x, jc = sm.jc, kp = sm.kp, arow = sm.arow;
  const int kg = (K + 3) / 4;
  const int ng = jc * kg;
  const int ntiles = (int)((J + jc - 1) / jc);
  __syncthreads();                                  // the staging buffers are free
  stage_s_tile<T>(S, L, (int)I, J, 0, jc, smf + sm.as, arow);
  cp_async_commit();
  for (int t = 0; t < ntiles; ++t) {
    const int b = t & 1;
    const int64_t j0 = (int64_t)t * jc;
    const float* As = smf + sm.as + b * sm.abuf;
    if (t + 1 < ntiles) stage_s_tile<T>(S, L, (int)I, J, j0 + jc, jc, smf + sm.as + (b ^ 1) * sm.abuf, arow);
    cp_async_commit();
    cp_async_wait_one();
    __syncthreads();
#pragma unroll
    for (int u = 0; u < BT_TMAX; ++u) {
      const int g = tid + T * u;
      if (g < ng) {
        const int jj = g % jc, c = g / jc;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll 4
        for (int i = 0; i < (int)I; ++i) {
          const float a = As[jj * arow + i];
          const float4 m = *reinterpret_cast<const float4*>(Ms + i * kp + 4 * c);
          a0 = fmaf(a, m.x, a0);
          a1 = fmaf(a, m.y, a1);
          a2 = fmaf(a, m.z, a2);
          a3 = fmaf(a, m.w, a3);
        }
        const int64_t j = j0 + jj;
        if (j < J) {
          const float v[4] = {a0, a1, a2, a3};
#pragma unroll
          for (int t2 = 0; t2 < 4; ++t2)
            if (4 * c + t2 < K) out[j + J * (4 * c + t2)] = v[t2];
        }
      }
    }
    __syncthreads();                                // this tile's buffer may be refilled
  }
}

// (bi <= bj) of block pair p, pairs enumerated column by column of the upper triangle
__device__ __forceinline__ void block_pair(int p, int& bi, int& bj) {
  bj = 0;
  while (p > bj) {
    p -= bj + 1;
    ++bj;
  }
  bi = p;
}

// G (K x K, column-major in shared memory, ld kp) = Z^T Z for Z (J x K, global,
// ld J): rows streamed through a shared tile; each thread accumulates one 4 x 4
// block pair over every `phases`-th row, then the phases are summed in order.
template <int T>
__device__ void blk_gram(const float* __restrict__ Z, int64_t J, int K, const BSmem& sm, float* smf) {
  float* Gs = smf + sm.gs;
  float* red = smf + sm.red;
  const int tid = threadIdx.x, kp = sm.kp;
  const int nb = kp / 4, npairs = nb * (nb + 1) / 2;
  const int phases = T / npairs;
  const int ph = tid / npairs, p = tid % npairs;
  const bool active = ph < phases;
  int bi, bj;
  block_pair(p, bi, bj);
  float acc[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) acc[e] = 0.f;
  stream_z_tiles<T>(Z, J, K, sm, smf, false, [&](int64_t, int nj, const float* Zs) {
    if (active)
      for (int jj = ph; jj < nj; jj += phases) {
        const float4 a = *reinterpret_cast<const float4*>(Zs + jj * kp + 4 * bi);
        const float4 b = *reinterpret_cast<const float4*>(Zs + jj * kp + 4 * bj);
        const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[4 * u + v] = fmaf(av[u], bv[v], acc[4 * u + v]);
      }
  });
  __syncthreads();
  if (active)
#pragma unroll
    for (int e = 0; e < 16; ++e) red[(ph * npairs + p) * 16 + e] = acc[e];
  __syncthreads();
  for (int w = tid; w < npairs * 16; w += T) {
    const int pp = w / 16, e = w % 16;
    float v = 0.f;
    for (int q = 0; q < phases; ++q) v += red[(q * npairs + pp) * 16 + e];
    int ri, cj;
    block_pair(pp, ri, cj);
    const int a = 4 * ri + e / 4, b = 4 * cj + e % 4;
    Gs[a + kp * b] = v;
    Gs[b + kp * a] = v;
  }
  __syncthreads();
}


// ||y||^2 (y of length I in shared memory) by the whole CTA, summed in a
// fixed order; every thread returns the same value.  wp: T/32 floats.
template <int T>
__device__ float blk_norm2(const float* y, int I, float* wp) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float s = 0.f;
  for (int i = tid; i < I; i += T) s = fmaf(y[i], y[i], s);
  s = warp_sum(s);
  __syncthreads();                                  // earlier readers of wp are done
  if (lane == 0) wp[warp] = s;
  __syncthreads();
  float t = 0.f;
#pragma unroll
  for (int w = 0; w < T / 32; ++w) t += wp[w];
  return t;
}

// Q = orth(Y) in place for Y (I x K, column-major, ld `ld`) in shared memory,
// by the whole CTA: classical Gram-Schmidt with one reorthogonalisation per
// column (CGS2; Giraud, Langou, Rozloznik, van den Eshof 2005: orthogonal to
// working precision, like MGS2), the projections on all earlier columns of a
// pass computed together, one warp per column.  A column left at rounding
// level by the projections (rank below K) is replaced by the next unit vector
// that is still independent of the columns before it, orthogonalised the same
// way.  `red` holds 32 + T/32 floats of scratch.  Returns false (on every
// thread) if a column norm was not finite.
template <int T>
__device__ bool blk_cgs2(float* Y, int ld, int I, int K, float* red) {
  constexpr int NW = T / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float* d = red;                                   // projections d_c, c < k <= 32
  float* wp = red + 32;                             // per-warp partial sums
  bool finite = true;
  int e_next = 0;
  for (int k = 0; k < K; ++k) {
    float* y = Y + (size_t)ld * k;
    float n0 = blk_norm2<T>(y, I, wp);
    if (!isfinite(n0)) finite = false;
    float n1 = 0.f;
    for (int attempt = 0;; ++attempt) {
      for (int pass = 0; pass < 2 && k > 0; ++pass) {
        for (int c = warp; c < k; c += NW) {        // d_c = q_c^T y
          const float* qc = Y + (size_t)ld * c;
          float v = 0.f;
          for (int i = lane; i < I; i += 32) v = fmaf(qc[i], y[i], v);
          v = warp_sum(v);
          if (lane == 0) d[c] = v;
        }
        __syncthreads();
        for (int i = tid; i < I; i += T) {          // y -= Q(:, 0:k) d
          float v = y[i];
          for (int c = 0; c < k; ++c) v = fmaf(-d[c], Y[i + (size_t)ld * c], v);
          y[i] = v;
        }
        __syncthreads();
      }
      n1 = blk_norm2<T>(y, I, wp);
      if ((n1 > 1e-11f * n0 && n1 > 0.f && isfinite(n1)) || e_next >= I || attempt > I) break;
      // dependent (or non-finite) column: restart from the next unit vector
      for (int i = tid; i < I; i += T) y[i] = (i == e_next) ? 1.f : 0.f;
      ++e_next;
      n0 = 1.f;
      __syncthreads();
    }
    const float inv = (n1 > 0.f && isfinite(n1)) ? rsqrtf(n1) : 0.f;
    for (int i = tid; i < I; i += T) y[i] *= inv;
    __syncthreads();
  }
  return finite;
}

// The column sweep of one Jacobi round on a K x K matrix A (ld kp) in shared
// memory: for every pair (p, q, c, s) of the round, columns p and q become
// c a_p - s a_q and s a_p + c a_q; lane r takes row r.
__device__ __forceinline__ void rotate_cols(float* A, int kp, int K, const float4* rot, int npairs) {
  // the pairs of a round are disjoint: every element is loaded before the first
  // store, so the round costs one shared-memory latency rather than one per pair
  constexpr int NP = BT_MAX_K / 2;
  const int r = threadIdx.x & 31;
  if (r < K) {
    float gp[NP], gq[NP];
#pragma unroll
    for (int w = 0; w < NP; ++w) {
      const float4 t = rot[w < npairs ? w : 0];
      const int p = __float_as_int(t.x), q = __float_as_int(t.y);
      const bool live = w < npairs && q >= 0;
      gp[w] = live ? A[r + kp * p] : 0.f;
      gq[w] = live ? A[r + kp * q] : 0.f;
    }
#pragma unroll
    for (int w = 0; w < NP; ++w) {
      if (w >= npairs) break;
      const float4 t = rot[w];
      const int p = __float_as_int(t.x), q = __float_as_int(t.y);
      if (q < 0) continue;
      A[r + kp * p] = t.z * gp[w] - t.w * gq[w];
      A[r + kp * q] = t.w * gp[w] + t.z * gq[w];
    }
  }
  __syncwarp();
}

// The row sweep of the same round (rows p and q); lane c takes column c.
__device__ __forceinline__ void rotate_rows(float* A, int kp, int K, const float4* rot, int npairs) {
  constexpr int NP = BT_MAX_K / 2;
  const int col = threadIdx.x & 31;
  if (col < K) {
    float gp[NP], gq[NP];
#pragma unroll
    for (int w = 0; w < NP; ++w) {
      const float4 t = rot[w < npairs ? w : 0];
      const int p = __float_as_int(t.x), q = __float_as_int(t.y);
      const bool live = w < npairs && q >= 0;
      gp[w] = live ? A[p + kp * col] : 0.f;
      gq[w] = live ? A[q + kp * col] : 0.f;
    }
#pragma unroll
    for (int w = 0; w < NP; ++w) {
      if (w >= npairs) break;
      const float4 t = rot[w];
      const int p = __float_as_int(t.x), q = __float_as_int(t.y);
      if (q < 0) continue;
      A[p + kp * col] = t.z * gp[w] - t.w * gq[w];
      A[q + kp * col] = t.w * gp[w] + t.z * gq[w];
    }
  }
  __syncwarp();
}

// Eigenvectors of the symmetric K x K matrix G (ld kp, overwritten) by
// two-sided cyclic Jacobi (Jacobi 1846; parallel round-robin ordering, Brent &
// Luk 1985) in one warp: each round rotates K/2 disjoint pairs, first the
// columns of G, then its rows, then the columns of V.  A pair is rotated while
// |g_pq| > 5e-7 sqrt(|g_pp g_qq|) and |g_pq| > 1e-10 tr(G).  On return V (ld kp)
// holds the eigenvectors as columns and the diagonal of G the eigenvalues.
// Returns the number of sweeps.
__device__ int warp_jacobi(float* G, float* V, int kp, int K, float4* rot) {
  const int lane = threadIdx.x & 31;
  for (int e = lane; e < K * kp; e += 32) {
    const int r = e % kp, c = e / kp;
    V[e] = (r == c) ? 1.f : 0.f;
  }
  float tr = 0.f;
  for (int i = lane; i < K; i += 32) tr += G[i + kp * i];
  tr = warp_sum(tr);
  const float floor_abs = 1e-10f * tr;
  __syncwarp();
  const int n = K + (K & 1), npairs = n / 2;
  int sweep = 0;
  for (; sweep < BT_MAX_SWEEPS; ++sweep) {
    bool rotated = false;
    for (int s = 0; s < n - 1; ++s) {
      bool mine = false;
      if (lane < npairs) {
        const int w = lane;
        int xa = w - 1 + s, xb = n - 2 - w + s;      // circle method
        if (xa >= n - 1) xa -= n - 1;
        if (xb >= n - 1) xb -= n - 1;
        const int a = (w == 0) ? 0 : xa + 1, b = xb + 1;
        const int p = min(a, b), q = max(a, b);
        float4 t = make_float4(__int_as_float(p), __int_as_float(-1), 1.f, 0.f);
        if (q < K) {
          const float gpq = G[p + kp * q], gpp = G[p + kp * p], gqq = G[q + kp * q];
          if (fabsf(gpq) > floor_abs && fabsf(gpq) > 5e-7f * sqrtf(fabsf(gpp * gqq))) {
            // t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)) zeroes g_pq of J^T G J
            const float zeta = (gqq - gpp) / (2.f * gpq);
            const float az = fabsf(zeta);
            float tt;
            if (az < 1e15f) {
              const float h = fmaf(zeta, zeta, 1.f);
              tt = 1.f / (az + h * rsqrtf(h));
            } else {
              tt = 0.5f / az;
            }
            tt = copysignf(tt, zeta);
            const float c = rsqrtf(fmaf(tt, tt, 1.f));
            t = make_float4(__int_as_float(p), __int_as_float(q), c, c * tt);
            mine = true;
          }
        }
        rot[w] = t;
      }
      const bool any = __any_sync(0xffffffffu, mine);
      __syncwarp();
      if (!any) continue;
      rotated = true;
      rotate_cols(G, kp, K, rot, npairs);
      rotate_rows(G, kp, K, rot, npairs);
      rotate_cols(V, kp, K, rot, npairs);
    }
    if (!rotated) break;
  }
  return sweep + 1;
}

// Cholesky factor of A + s I (K x K, ld kp, lower part overwritten by L) and
// Linv = L^-1 (lower, ld kp), in one warp, FP32; lane r owns row r.  Returns
// false on a non-positive or non-finite pivot.
__device__ bool warp_chol_inv(float* A, float* Linv, int kp, int K, float shift) {
  const int r = threadIdx.x & 31;
  if (r < K) A[r + kp * r] += shift;
  __syncwarp();
  bool ok = true;
  for (int j = 0; j < K; ++j) {
    const float d = A[j + kp * j];
    if (!(d > 0.f) || !isfinite(d)) {
      ok = false;
      break;
    }
    const float rs = rsqrtf(d);
    if (r >= j && r < K) A[r + kp * j] *= rs;         // column j of L (L_jj = sqrt(d))
    __syncwarp();
    if (r > j && r < K) {
      const float lrj = A[r + kp * j];
      for (int c = j + 1; c <= r; ++c) A[r + kp * c] = fmaf(-lrj, A[c + kp * j], A[r + kp * c]);
    }
    __syncwarp();
  }
  if (!ok) return false;
  // column c of L^-1 by forward substitution (lane c)
  const int c = r;
  if (c < K)
    for (int i = 0; i < K; ++i) {
      if (i < c) {
        Linv[i + kp * c] = 0.f;
        continue;
      }
      float v = (i == c) ? 1.f : 0.f;
      for (int k = c; k < i; ++k) v = fmaf(-A[i + kp * k], Linv[k + kp * c], v);
      Linv[i + kp * c] = v / A[i + kp * i];
    }
  __syncwarp();
  return true;
}

// Z (J x K, global, ld J) <- Z R^-1 with R^T R = Z^T Z + s I, s = 1e-5 tr(Z^T Z):
// one shifted CholeskyQR pass (Fukaya, Kannan, Nakatsukasa, Yamamoto,
// Yanagisawa 2020).  The power iteration needs only range(Z); the shift keeps
// the FP32 factorisation from breaking down whatever cond(Z), and the next
// basis is formed by CGS2 with dependent columns replaced, which any
// conditioning of Y = S_(n) Z survives.
// Returns false (Z unchanged) if the factorisation failed.
template <int T>
__device__ bool blk_range_basis(float* __restrict__ Z, int64_t J, int K, const BSmem& sm, float* smf) {
  blk_gram<T>(Z, J, K, sm, smf);
  float* Gs = smf + sm.gs;
  float* Li = smf + sm.vs;
  int* flag = reinterpret_cast<int*>(smf + sm.red);
  const int tid = threadIdx.x, kp = sm.kp;
  if (tid < 32) {
    float tr = 0.f;
    for (int i = tid; i < K; i += 32) tr += Gs[i + kp * i];
    tr = warp_sum(tr);
    const bool ok = warp_chol_inv(Gs, Li, kp, K, 1e-5f * tr);
    if (tid == 0) *flag = ok ? 1 : 0;
  }
  __syncthreads();
  const bool ok = *flag != 0;
  if (ok) {
    // Z <- Z L^-T tile by tile: rows staged in shared memory ([jj][k], pitch kp + 1);
    // a tile is rewritten in place while the next one is copied in
    stream_z_tiles<T>(Z, J, K, sm, smf, true, [&](int64_t j0, int nj, const float* Zs) {
      for (int e = tid; e < nj * K; e += T) {
        const int jj = e % nj, k = e / nj;
        float v = 0.f;
        for (int c = 0; c <= k; ++c) v = fmaf(Zs[jj * (kp + 1) + c], Li[k + kp * c], v);
        Z[(j0 + jj) + J * k] = v;
      }
    });
  }
  __syncthreads();
  return ok;
}

// Ms (row-major [i][k], pitch kp) = Ys (column-major, ld ip), for the TTMs.
template <int T>
__device__ void q_to_rowmajor(const BSmem& sm, float* smf, int I, int K) {
  const float* Ys = smf + sm.ys;
  float* Ms = smf + sm.ms;
  for (int e = threadIdx.x; e < I * sm.kp; e += T) {
    const int i = e / sm.kp, k = e % sm.kp;
    Ms[e] = (k < K) ? Ys[i + sm.ip * k] : 0.f;
  }
  __syncthreads();
}

// One whole R-STHOSVD of the tensor *it by this CTA.  The current mode sizes
// live in shared memory (dims), and the item is read through its pointer, so
// the kernel keeps no per-thread arrays in local memory.
template <int T>
__device__ void decompose_one(const BItem* __restrict__ it, int q, uint64_t seed, float* Zb, float* Sb0, float* Sb1,
                              const BSmem& sm, float* smf, int64_t* dims, DevStatus* st) {
  const int tid = threadIdx.x, N = it->N, kp = sm.kp;
  if (tid < N) dims[tid] = it->d[tid];
  __syncthreads();
  const float* cur = it->X;
  float* const G = it->G;
  int ping = 0;
  float4* rot = reinterpret_cast<float4*>(smf + sm.red);
  int* order = reinterpret_cast<int*>(smf + sm.red + 64);
  float* Ys = smf + sm.ys;
  float* Gs = smf + sm.gs;
  float* Vs = smf + sm.vs;
  float* Ub = smf + sm.ub;
  for (int n = 0; n < N; ++n) {
    const int64_t I = dims[n], L = prod_lt(dims, n);
    int64_t Rt = 1;
    for (int k = n + 1; k < N; ++k) Rt *= dims[k];
    const int64_t J = L * Rt;
    const int R = it->r[n], K = it->K[n];
    const bool last = (n == N - 1);
    float* U = it->U[n];
    if (R == I) {                                   // nothing to reduce in this mode
      for (int64_t e = tid; e < I * I; e += T) U[e] = (e % I == e / I) ? 1.f : 0.f;
      if (last)
        for (int64_t e = tid; e < I * J; e += T) G[e] = cur[e];
      __syncthreads();
      continue;
    }
    // Y = S_(n) Omega_n, Q = orth(Y)
    blk_sketch<T>(cur, L, I, J, K, nullptr, seed, (uint32_t)n, sm, smf);
    if (!blk_cgs2<T>(Ys, sm.ip, (int)I, K, smf + sm.red) && tid == 0) set_error(st, RHOSVD_ENONFINITE);
    for (int p = 0; p < q; ++p) {
      q_to_rowmajor<T>(sm, smf, (int)I, K);
      blk_ttm<T>(cur, L, I, J, K, Zb, sm, smf);            // Z = S_(n)^T Q
      blk_range_basis<T>(Zb, J, K, sm, smf);                     // a basis of range(Z)
      blk_sketch<T>(cur, L, I, J, K, Zb, seed, 0, sm, smf);   // Y = S_(n) Z
      if (!blk_cgs2<T>(Ys, sm.ip, (int)I, K, smf + sm.red) && tid == 0) set_error(st, RHOSVD_ENONFINITE);
    }
    // B^T = S_(n)^T Q, G = B B^T, leading eigenvectors Ubar_R
    q_to_rowmajor<T>(sm, smf, (int)I, K);
    blk_ttm<T>(cur, L, I, J, K, Zb, sm, smf);
    blk_gram<T>(Zb, J, K, sm, smf);
    if (tid < 32) {
      const int sweeps = warp_jacobi(Gs, Vs, kp, K, rot);
      if (tid == 0 && sweeps > 1) atomicMax(&st->eig_sweeps, sweeps);
      // order by eigenvalue (descending, ties by index); Ubar = the R leading columns of V
      if (tid < K) {
        const float lc = Gs[tid + kp * tid];
        int rank = 0;
        for (int o = 0; o < K; ++o) {
          const float lo = Gs[o + kp * o];
          rank += (lo > lc) || (lo == lc && o < tid);
        }
        order[rank] = tid;
      }
      __syncwarp();
      for (int e = tid; e < K * R; e += 32) {
        const int k = e % K, a = e / K;
        Ub[k + kp * a] = Vs[k + kp * order[a]];
      }
    }
    __syncthreads();
    // U_n = Q Ubar_R (I x R, ld I)
    for (int64_t e = tid; e < I * R; e += T) {
      const int i = (int)(e % I), a = (int)(e / I);
      float v = 0.f;
      for (int k = 0; k < K; ++k) v = fmaf(Ys[i + sm.ip * k], Ub[k + kp * a], v);
      U[e] = v;
    }
    // S_new[l + L a + L R r] = sum_k Ubar(k, a) B^T(l + L r, k): rows of B^T staged
    // in shared memory ([jj][k], pitch kp + 1), one output (j, a) per thread and step
    float* dst = last ? G : (ping ? Sb1 : Sb0);
    stream_z_tiles<T>(Zb, J, K, sm, smf, true, [&](int64_t j0, int nj, const float* Bs) {
      for (int e = tid; e < nj * R; e += T) {
        const int jj = e % nj, a = e / nj;
        float v = 0.f;
        for (int k = 0; k < K; ++k) v = fmaf(Bs[jj * (kp + 1) + k], Ub[k + kp * a], v);
        const int64_t j = j0 + jj, l = j % L, r = j / L;
        dst[l + L * a + L * R * r] = v;
      }
    });
    __syncthreads();
    if (tid == 0) dims[n] = R;
    __syncthreads();
    cur = dst;
    ping ^= 1;
  }
}

// The sizes every index of decompose_one is bounded by: mode sizes and sketch
// widths within the shared-memory carve-up, J_n K_n within the per-CTA Z
// buffer and every intermediate core within a core buffer.
__device__ bool item_fits(const BItem* __restrict__ it, int imax, int kmax, int64_t zb_floats, int64_t s_floats) {
  const int N = it->N;
  if (N < 1 || N > RHOSVD_MAX_MODES) return false;
  for (int k = 0; k < N; ++k)
    if (it->d[k] < 1 || it->d[k] > imax) return false;
  for (int n = 0; n < N; ++n) {
    // before mode n the core has sizes R_1..R_{n-1}, I_n..I_N
    int64_t J = 1, core = 1;
    for (int k = 0; k < N; ++k) {
      const int64_t cur_k = (k < n) ? (int64_t)it->r[k] : it->d[k];
      if (k != n) J *= cur_k;
      core *= (k <= n) ? (int64_t)it->r[k] : it->d[k];
    }
    const int R = it->r[n], K = it->K[n];
    if (R < 1 || R > it->d[n] || K < R || K > kmax || K > it->d[n] || K > J || J * K > zb_floats) return false;
    if (core > s_floats) return false;
  }
  return true;
}

template <int T>
__global__ void __launch_bounds__(T, T == 512 ? 1 : 65536 / (T * 128))
batch_rsthosvd_kernel(const BItem* __restrict__ items, const int32_t* __restrict__ order, int n_items,
                      uint32_t* counter, float* scratch, int64_t zb_floats, int64_t s_floats, int imax, int kmax,
                      int jc, int q, uint64_t seed, DevStatus* st) {
  extern __shared__ __align__(16) float bt_smem[];
  __shared__ int64_t dims[RHOSVD_MAX_MODES];
  __shared__ int s_next;
  const BSmem sm(imax, kmax, jc, T);
  // the carve-up must fit the dynamic shared memory this launch was given
  uint32_t dyn_bytes;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_bytes));
  if ((size_t)sm.total * sizeof(float) > dyn_bytes || jc > 64 || T % jc != 0 || kmax > BT_MAX_K) {
    if (threadIdx.x == 0 && blockIdx.x == 0) set_error(st, RHOSVD_EINVAL);
    return;
  }
  float* Zb = scratch + (int64_t)blockIdx.x * (zb_floats + 2 * s_floats);
  float* Sb0 = Zb + zb_floats;
  float* Sb1 = Sb0 + s_floats;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_next = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int t = s_next;
    if (t >= n_items) break;
    const BItem* it = items + order[t];
    if (!item_fits(it, imax, kmax, zb_floats, s_floats)) {   // a table that disagrees with the plan
      if (threadIdx.x == 0) set_error(st, RHOSVD_EINVAL);
      continue;
    }
    decompose_one<T>(it, q, seed, Zb, Sb0, Sb1, sm, bt_smem, dims, st);
  }
}

}  // namespace

// ---------------------------------------------------------------- host side

namespace {

constexpr size_t BT_ALIGN = 256;
constexpr int BT_MAX_CTAS_PER_SM = 4;
const int kThreads[3] = {128, 256, 512};
const int kChunks[2] = {32, 64};

size_t align_up(size_t v) { return (v + BT_ALIGN - 1) / BT_ALIGN * BT_ALIGN; }

struct BLayout {
  size_t counter, items, order, scratch, total;
};

BLayout layout_of(const rhosvd_batch_plan& p) {
  BLayout l;
  size_t o = sizeof(DevStatus);
  l.counter = o;
  o = align_up(o + sizeof(uint32_t));
  l.items = o;
  o = align_up(o + sizeof(BItem) * (size_t)p.n_items);
  l.order = o;
  o = align_up(o + sizeof(int32_t) * (size_t)p.n_items);
  l.scratch = o;
  o += sizeof(float) * (size_t)p.max_ctas * (size_t)(p.zb_floats + 2 * p.s_floats);
  l.total = align_up(o);
  return l;
}

size_t smem_bytes(const rhosvd_batch_plan& p, int threads, int jc) {
  return sizeof(float) * (size_t)BSmem(p.imax, p.kmax, jc, threads).total;
}

const void* kernel_of(int threads) {
  switch (threads) {
    case 128: return (const void*)batch_rsthosvd_kernel<128>;
    case 256: return (const void*)batch_rsthosvd_kernel<256>;
    case 512: return (const void*)batch_rsthosvd_kernel<512>;
    default: return nullptr;
  }
}

// CTAs per SM the configuration can keep resident (0 = not launchable).
int resident_ctas(const rhosvd_batch_plan& p, int threads, int jc) {
  const void* k = kernel_of(threads);
  if (k == nullptr || (jc != 32 && jc != 64)) return 0;
  const int kg = (p.kmax + 3) / 4;
  if (p.imax * ((kg + 1) / 2) > BT_GMAX * threads || jc * kg > BT_TMAX * threads) return 0;
  const size_t smem = smem_bytes(p, threads, jc);
  if (smem > 200 * 1024) return 0;
  if (allow_dynamic_smem(k, smem) != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem) != cudaSuccess) return 0;
  return std::min(n, BT_MAX_CTAS_PER_SM);
}

cudaError_t launch_batch(const rhosvd_batch_plan& p, void* ws, cudaStream_t s) {
  const BLayout l = layout_of(p);
  char* base = static_cast<char*>(ws);
  const int ctas = std::min(p.max_ctas, p.sms * p.ctas_per_sm);
  cudaError_t e = cudaMemsetAsync(base + l.counter, 0, sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  const size_t smem = smem_bytes(p, p.threads, p.jc);
  const void* k = kernel_of(p.threads);
  if (k == nullptr) return cudaErrorInvalidValue;
  if ((e = allow_dynamic_smem(k, smem)) != cudaSuccess) return e;
  const BItem* items = reinterpret_cast<const BItem*>(base + l.items);
  const int32_t* order = reinterpret_cast<const int32_t*>(base + l.order);
  uint32_t* counter = reinterpret_cast<uint32_t*>(base + l.counter);
  float* scratch = reinterpret_cast<float*>(base + l.scratch);
  DevStatus* st = reinterpret_cast<DevStatus*>(base);
  switch (p.threads) {
    case 128:
      batch_rsthosvd_kernel<128><<<ctas, 128, smem, s>>>(items, order, p.n_items, counter, scratch, p.zb_floats,
                                                         p.s_floats, p.imax, p.kmax, p.jc, p.q, p.seed, st);
      break;
    case 256:
      batch_rsthosvd_kernel<256><<<ctas, 256, smem, s>>>(items, order, p.n_items, counter, scratch, p.zb_floats,
                                                         p.s_floats, p.imax, p.kmax, p.jc, p.q, p.seed, st);
      break;
    default:
      batch_rsthosvd_kernel<512><<<ctas, 512, smem, s>>>(items, order, p.n_items, counter, scratch, p.zb_floats,
                                                         p.s_floats, p.imax, p.kmax, p.jc, p.q, p.seed, st);
      break;
  }
  return cudaGetLastError();
}

}  // namespace
}  // namespace rhosvd

using namespace rhosvd;

extern "C" {

rhosvd_status rhosvd_batch_plan_create(const rhosvd_batch_item* items, int32_t n_items, const rhosvd_opts* opts,
                                       rhosvd_batch_plan* plan) {
  if (items == nullptr || opts == nullptr || plan == nullptr || n_items < 1) return RHOSVD_EINVAL;
  if (opts->algo != RHOSVD_ALGO_RSTHOSVD || opts->flags != 0 || opts->dtype != RHOSVD_F32 ||
      opts->refine_iters != 0 || opts->q < 0 || opts->q > 8 || opts->p < 0)
    return RHOSVD_EINVAL;
  rhosvd_batch_plan p{};
  p.n_items = n_items;
  p.q = opts->q;
  p.p = opts->p;
  p.seed = opts->seed;
  int imax = 1, kmax = 1;
  int64_t zb = 1, smax = 1;
  for (int32_t t = 0; t < n_items; ++t) {
    const rhosvd_batch_item& it = items[t];
    if (it.X == nullptr || it.G == nullptr || it.N < 1 || it.N > RHOSVD_MAX_MODES) return RHOSVD_EINVAL;
    rhosvd_shape sh{};
    sh.N = it.N;
    for (int n = 0; n < it.N; ++n) {
      if (it.dims[n] < 1 || it.dims[n] > BT_MAX_I || it.U[n] == nullptr) return RHOSVD_EINVAL;
      sh.dims[n] = it.dims[n];
    }
    int32_t K[RHOSVD_MAX_MODES];
    int64_t J[RHOSVD_MAX_MODES];
    if (rhosvd_plan(&sh, it.ranks, opts, K, nullptr, J) != RHOSVD_OK) return RHOSVD_EINVAL;
    int64_t cur[RHOSVD_MAX_MODES];
    for (int n = 0; n < it.N; ++n) cur[n] = it.dims[n];
    for (int n = 0; n < it.N; ++n) {
      if (K[n] > BT_MAX_K || J[n] * (int64_t)K[n] >= (int64_t(1) << 31)) return RHOSVD_EINVAL;
      imax = std::max<int>(imax, (int)it.dims[n]);
      kmax = std::max<int>(kmax, K[n]);
      zb = std::max<int64_t>(zb, J[n] * K[n]);
      cur[n] = it.ranks[n];
      int64_t v = 1;
      for (int k = 0; k < it.N; ++k) v *= cur[k];
      smax = std::max<int64_t>(smax, v);
    }
  }
  p.imax = imax;
  p.kmax = kmax;
  p.zb_floats = (zb + 63) / 64 * 64;
  p.s_floats = (smax + 63) / 64 * 64;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&p.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return RHOSVD_ECUDA;
  p.max_ctas = p.sms * BT_MAX_CTAS_PER_SM;
  // default configuration: 256 threads, 64-column tiles, as many CTAs per SM as fit
  p.threads = 256;
  p.jc = 64;
  p.ctas_per_sm = resident_ctas(p, 256, 64);
  if (p.ctas_per_sm == 0) {
    for (int T : kThreads)
      for (int jc : kChunks)
        if (p.ctas_per_sm == 0 && (p.ctas_per_sm = resident_ctas(p, T, jc)) > 0) {
          p.threads = T;
          p.jc = jc;
        }
    if (p.ctas_per_sm == 0) return RHOSVD_EINVAL;
  }
  p.ws_bytes = layout_of(p).total;
  *plan = p;
  return RHOSVD_OK;
}

rhosvd_status rhosvd_batch_upload(const rhosvd_batch_plan* plan, const rhosvd_batch_item* items, void* ws,
                                  size_t ws_bytes, void* stream) {
  if (plan == nullptr || items == nullptr || ws == nullptr || (reinterpret_cast<uintptr_t>(ws) % BT_ALIGN) != 0)
    return RHOSVD_EINVAL;
  const BLayout l = layout_of(*plan);
  if (ws_bytes < l.total) return RHOSVD_ENOMEM;
  rhosvd_opts o{};
  o.algo = RHOSVD_ALGO_RSTHOSVD;
  o.p = plan->p;
  o.q = plan->q;
  std::vector<BItem> table((size_t)plan->n_items);
  std::vector<std::pair<double, int32_t>> cost((size_t)plan->n_items);
  for (int32_t t = 0; t < plan->n_items; ++t) {
    const rhosvd_batch_item& it = items[t];
    if (it.X == nullptr || it.G == nullptr || it.N < 1 || it.N > RHOSVD_MAX_MODES) return RHOSVD_EINVAL;
    BItem b{};
    b.X = it.X;
    b.G = it.G;
    b.N = it.N;
    rhosvd_shape sh{};
    sh.N = it.N;
    double numel = 1.0;
    for (int n = 0; n < it.N; ++n) {
      if (it.dims[n] < 1 || it.dims[n] > plan->imax || it.U[n] == nullptr) return RHOSVD_EINVAL;
      b.U[n] = it.U[n];
      b.d[n] = it.dims[n];
      b.r[n] = it.ranks[n];
      sh.dims[n] = it.dims[n];
      numel *= (double)it.dims[n];
    }
    int32_t K[RHOSVD_MAX_MODES];
    int64_t J[RHOSVD_MAX_MODES];
    if (rhosvd_plan(&sh, it.ranks, &o, K, nullptr, J) != RHOSVD_OK) return RHOSVD_EINVAL;
    int64_t cur[RHOSVD_MAX_MODES];
    for (int n = 0; n < it.N; ++n) cur[n] = it.dims[n];
    for (int n = 0; n < it.N; ++n) {
      if (K[n] > plan->kmax || J[n] * (int64_t)K[n] > plan->zb_floats) return RHOSVD_EINVAL;
      b.K[n] = K[n];
      cur[n] = it.ranks[n];
      int64_t v = 1;
      for (int k = 0; k < it.N; ++k) v *= cur[k];
      if (v > plan->s_floats) return RHOSVD_EINVAL;
    }
    table[(size_t)t] = b;
    cost[(size_t)t] = {numel * (double)K[0], t};
  }
  // largest work first, so that the tail of the queue holds the short items
  std::stable_sort(cost.begin(), cost.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
  std::vector<int32_t> order((size_t)plan->n_items);
  for (size_t t = 0; t < order.size(); ++t) order[t] = cost[t].second;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(ws);
  if (cudaMemsetAsync(ws, 0, sizeof(DevStatus), s) != cudaSuccess ||
      cudaMemcpyAsync(base + l.items, table.data(), sizeof(BItem) * table.size(), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(base + l.order, order.data(), sizeof(int32_t) * order.size(), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)   // the host tables are freed on return
    return RHOSVD_ECUDA;
  return RHOSVD_OK;
}

rhosvd_status rhosvd_batch_run(const rhosvd_batch_plan* plan, void* ws, size_t ws_bytes, void* stream) {
  if (plan == nullptr || ws == nullptr || ws_bytes < layout_of(*plan).total) return RHOSVD_EINVAL;
  if (plan->ctas_per_sm < 1 || plan->ctas_per_sm > resident_ctas(*plan, plan->threads, plan->jc))
    return RHOSVD_EINVAL;
  return launch_batch(*plan, ws, static_cast<cudaStream_t>(stream)) == cudaSuccess ? RHOSVD_OK : RHOSVD_ECUDA;
}

rhosvd_status rhosvd_batch_tune(rhosvd_batch_plan* plan, void* ws, size_t ws_bytes, void* stream, float* best_ms) {
  if (plan == nullptr || ws == nullptr || ws_bytes < layout_of(*plan).total) return RHOSVD_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return RHOSVD_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return RHOSVD_ECUDA;
  }
  rhosvd_batch_plan best = *plan;
  float best_t = -1.f;
  rhosvd_status status = RHOSVD_OK;
  for (int T : kThreads)
    for (int jc : kChunks) {
      const int maxc = resident_ctas(*plan, T, jc);
      for (int c = 1; c <= maxc && status == RHOSVD_OK; ++c) {
        rhosvd_batch_plan cand = *plan;
        cand.threads = T;
        cand.jc = jc;
        cand.ctas_per_sm = c;
        float ms = 0.f;
        if (launch_batch(cand, ws, s) != cudaSuccess ||                 // warm
            cudaEventRecord(e0, s) != cudaSuccess || launch_batch(cand, ws, s) != cudaSuccess ||
            cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
          status = RHOSVD_ECUDA;
          break;
        }
        if (best_t < 0.f || ms < best_t) {
          best_t = ms;
          best = cand;
        }
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != RHOSVD_OK) return status;
  if (best_t < 0.f) return RHOSVD_EINVAL;
  *plan = best;
  if (best_ms != nullptr) *best_ms = best_t;
  return RHOSVD_OK;
}

}  // extern "C"
