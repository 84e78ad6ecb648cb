// Thin orthonormalisation of a tall m x K matrix (the orth steps of
// Alg. 1, Alg. 6 and Alg. 9): CholeskyQR2 with a Householder fallback.
//
// CholeskyQR2 (Fukaya, Nakatsukasa, Yanagisawa, Yamamoto 2014; Yamamoto et al.
// 2015): G = Y^T Y, R = chol(G), Q1 = Y R^-1, repeated once on Q1.  The Gram is
// accumulated in double-float (FP64-accurate, see gram.cu); the first pass's
// Cholesky runs in FP64 on one CTA, the second pass's in FP32 when its Gram is
// close to I; Y R^-1 is applied by row-parallel forward substitution.
// The first pass only rejects pivots that are numerically non-positive
// (<= K * 1e-15 * max diag): for larger condition numbers Q1 = Y R^-1 is still
// formed and the second pass assesses it; a second-pass pivot below 1e-4 * max
// diag (cond(Q1) above 100, so Q2 would not be orthonormal to FP32 accuracy)
// or a non-finite value marks a breakdown; the later kernels of the sequence
// then skip and a Householder QR
// (Golub & Van Loan Alg. 5.2.1 with the LAPACK geqr2/org2r conventions) forms
// Q instead.  The decision is taken on the device, so nothing synchronises.
#include <math.h>

#include "common.cuh"
#include "kernels.h"
#include "small_la.cuh"

namespace rhosvd {

namespace {

constexpr int CH_THREADS = 256;

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Cholesky factor L (G = L L^T) of one CholeskyQR pass.  G is first copied to
// shared memory with independent loads (one memory latency, not one per loop
// trip).  The first pass's Gram can have condition ~1e12 and is factored in
// double-word arithmetic; the second pass's in FP32 when every off-diagonal
// cosine G_ij / sqrt(G_ii G_jj) is at most 1e-2 (then cond(G) < 1.5 and FP32
// adds O(K u) to the orthogonality of Q2), in double-word otherwise.  Pivot
// thresholds relative to max diag: K * 1e-14 for the first pass (numerically
// non-positive at double-word precision), 1e-4 for the second (cond(Q1) > 100).
//
// With Minv != nullptr the kernel also writes R^-1 = L^-T (FP32, K x K,
// column-major, leading dimension ldm), so that the apply Q = Y R^-1 is a plain
// GEMM; the inverse comes from forward substitution run inside the
// factorisation's own steps (chol_grid), from the FP32 factor the row-wise
// solve would use.
template <int KB>
__global__ void __launch_bounds__(CH_THREADS)
chol_kernel(const double* __restrict__ G, int K, float* __restrict__ Lout, float* __restrict__ Minv, int ldm,
            int pass, int fail_code, DevStatus* st) {
  if (pass == 1 && st->orth_fail) return;
  extern __shared__ __align__(16) unsigned char ch_smem[];
  double* Gs = reinterpret_cast<double*>(ch_smem);                 // K x K FP64
  unsigned char* work = ch_smem + (size_t)K * K * sizeof(double);  // FP32 factorisation storage
  float* Tinv = (Minv != nullptr) ? reinterpret_cast<float*>(work + (size_t)K * K * sizeof(float)) : nullptr;
  __shared__ int nonfinite, flag;
  __shared__ float wmax[CH_THREADS / 32];
  __shared__ double maxdiag;
  __shared__ df64 rs_dw[RHOSVD_MAX_K];
  __shared__ float rs_f[RHOSVD_MAX_K];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) nonfinite = 0;
  __syncthreads();
  #pragma unroll 8
  for (int e = tid; e < K * K; e += CH_THREADS) {
    const double v = G[e];
    Gs[e] = v;
    if (!finite_bits(v)) nonfinite = 1;
  }
  __syncthreads();
  if (warp == 0) {
    double m = 0.0;
    for (int i = lane; i < K; i += 32) m = fmax(m, Gs[i + i * K]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) maxdiag = m;
  }
  float cmax = 0.f;                          // largest off-diagonal cosine, in FP32
  for (int e = tid; e < K * K; e += CH_THREADS) {
    const int c = e / K, r = e - c * K;
    if (r > c) {
      const float grr = f32_trunc(Gs[r + r * K]), gcc = f32_trunc(Gs[c + c * K]);
      const float cs = (grr > 0.f && gcc > 0.f) ? fabsf(f32_trunc(Gs[e])) * rsqrtf(grr) * rsqrtf(gcc) : 1.f;
      cmax = fminf(fmaxf(cmax, cs), 1.f);
    }
  }
  cmax = warp_max(cmax);
  if (lane == 0) wmax[warp] = cmax;
  __syncthreads();
  float allmax = 0.f;
#pragma unroll
  for (int w = 0; w < CH_THREADS / 32; ++w) allmax = fmaxf(allmax, wmax[w]);
  bool ok = !nonfinite && maxdiag > 0.0 && isfinite(maxdiag);
  if (ok) {
    const int e = 2 * (ilogb(maxdiag) / 2);  // even power of two: exact scaling and unscaling
    const double tol = ((pass == 0) ? (double)K * 1e-14 : 1e-4) * ldexp(maxdiag, -e);
    if (pass == 1 && allmax <= 1e-2f)
      ok = chol_grid<F32Ops, KB>(Gs, K, e, tol, false, Lout, reinterpret_cast<float*>(work), rs_f, &flag, Tinv);
    else
      // the double-word factor overwrites Gs in place: same element size, and each
      // element is read and rewritten by the same thread
      ok = chol_grid<DWOps, KB>(Gs, K, e, tol, false, Lout, reinterpret_cast<df64*>(Gs), rs_dw, &flag, Tinv);
  }
  if (!ok) {
    if (tid == 0) {
      st->orth_fail = 1;
      if (nonfinite) set_error(st, RHOSVD_ENONFINITE);
      else if (fail_code != 0) set_error(st, fail_code);
    }
    return;
  }
  if (pass == 0 && tid == 0) st->orth_fail = 0;
  if (Minv == nullptr) return;
  __syncthreads();
  for (int e = tid; e < K * K; e += CH_THREADS) {     // Minv(i, c) = (L^-1)(c, i) = Tinv(c, i) / L(c, c)
    const int i = e / K, c = e - i * K;
    Minv[i + (int64_t)c * ldm] = (c >= i) ? Tinv[c + i * K] / Lout[c + c * K] : 0.f;
  }
}

// Row-parallel triangular solves with the Cholesky factor L (K x K, lower):
// for every row y^T of Y (m x K, ld), mode 0 overwrites it with q^T where
// L q = y, i.e. Q = Y L^-T = Y R^-1 (the CholeskyQR apply); mode 1 then also
// solves L^T x = q, i.e. Y (L L^T)^-1 = Y G^-1 (normal-equation pseudo-inverse).
// One thread per row, the row in registers (KB >= K, fully unrolled), L in
// shared memory row-major for the forward sweep and column-major for the
// backward sweep.  Every load of the row and of L is issued before the first
// one is used (unrolled, no dependence between them), so the prologue costs
// one memory round trip rather than one per element; for a fixed column the
// 32 lanes of a warp touch 32 consecutive rows, so the accesses coalesce.
constexpr int TR_ROWS = 128;

template <int KB>
__global__ void __launch_bounds__(TR_ROWS)
trsm_rows_kernel(float* __restrict__ Y, int64_t m, int K, int64_t ld, const float* __restrict__ L, int mode,
                 const DevStatus* skip) {
  if (skip != nullptr && skip->orth_fail) return;
  extern __shared__ __align__(16) float tr_smem[];
  float* Lr = tr_smem;                 // K x KB row-major: Lr[c*KB + k] = L(c,k)
  float* Lc = Lr + KB * KB;            // KB x K column-major: Lc[k + c*KB] = L(k,c)
  float* dinv = Lc + KB * KB;          // 1 / L(c,c)
  const int tid = threadIdx.x;
  const int64_t row = (int64_t)blockIdx.x * TR_ROWS + tid;
  const bool live = row < m;
  float q[KB];
#pragma unroll
  for (int c = 0; c < KB; ++c) q[c] = (live && c < K) ? Y[row + (int64_t)c * ld] : 0.f;
  constexpr int LU = (KB * KB + TR_ROWS - 1) / TR_ROWS;
#pragma unroll 16
  for (int u = 0; u < LU; ++u) {
    const int e = tid + u * TR_ROWS;
    if (e < KB * KB) {
      const int c = e / KB, k = e - c * KB;
      const float v = (c < K && k < K) ? L[c + k * K] : 0.f;     // L(c,k)
      Lr[c * KB + k] = v;
      Lc[c + k * KB] = v;                                         // L(c,k) at column k
    }
  }
  if (tid < KB) dinv[tid] = (tid < K) ? 1.f / L[tid + tid * K] : 0.f;
  __syncthreads();
  if (!live) return;
  // forward: q_c = (y_c - sum_{k<c} L(c,k) q_k) / L(c,c); up to KB = 64 each dot
  // product runs as two interleaved partial sums, halving the dependent
  // multiply-add chain (wider rows would spill the second accumulator)
  constexpr bool two = KB <= 64;
#pragma unroll
  for (int c = 0; c < KB; ++c) {
    float s0 = q[c], s1 = 0.f;
    const float* lrow = Lr + c * KB;
    if (two) {
#pragma unroll
      for (int k = 0; k + 1 < c; k += 2) {
        s0 = fmaf(-lrow[k], q[k], s0);
        s1 = fmaf(-lrow[k + 1], q[k + 1], s1);
      }
      if (c & 1) s0 = fmaf(-lrow[c - 1], q[c - 1], s0);
    } else {
#pragma unroll
      for (int k = 0; k < c; ++k) s0 = fmaf(-lrow[k], q[k], s0);
    }
    q[c] = (s0 + s1) * dinv[c];
  }
  if (mode == 1) {
    // backward: x_c = (q_c - sum_{k>c} L(k,c) x_k) / L(c,c)
#pragma unroll
    for (int c = KB - 1; c >= 0; --c) {
      float s0 = q[c], s1 = 0.f;
      const float* lcol = Lc + c * KB;
      if (two) {
#pragma unroll
        for (int k = c + 1; k + 1 < KB; k += 2) {
          s0 = fmaf(-lcol[k], q[k], s0);
          s1 = fmaf(-lcol[k + 1], q[k + 1], s1);
        }
        if ((KB - 1 - c) & 1) s0 = fmaf(-lcol[KB - 1], q[KB - 1], s0);
      } else {
#pragma unroll
        for (int k = c + 1; k < KB; ++k) s0 = fmaf(-lcol[k], q[k], s0);
      }
      q[c] = (s0 + s1) * dinv[c];
    }
  }
#pragma unroll
  for (int c = 0; c < KB; ++c)
    if (c < K) Y[row + (int64_t)c * ld] = q[c];
}

// The CholeskyQR apply Q = Y R^-1 in place with the explicit inverse
// R^-1 = Minv (K x K upper triangular, column-major, ld ldm, written by
// chol_kernel): q_c = sum_{i <= c} y_i R^-1(i, c).  One thread per row with
// the row in registers; column c of R^-1 sits in shared memory as one
// contiguous run read as broadcast float4.  Unlike the forward substitution
// no output waits for another, so the K dot products overlap; each is an FP32
// multiply-add chain rounded to nearest.  A finite Gram (checked by the
// factorisation) implies a finite Y, so the zero padding of R^-1 past the
// diagonal adds exact zeros.  (Persistent CTAs that stage R^-1 once and loop
// over row blocks measured slower: the loads of a block then wait behind the
// arithmetic of the previous one.)
template <int KB>
__global__ void __launch_bounds__(TR_ROWS, KB <= 32 ? 4 : KB <= 48 ? 3 : 2)
apply_rinv_rows_kernel(float* __restrict__ Y, int64_t m, int K, int64_t ld, const float* __restrict__ Minv,
                       int ldm, const DevStatus* skip) {
  if (skip != nullptr && skip->orth_fail) return;
  __shared__ __align__(16) float Mc[KB * KB];     // Mc[c * KB + i] = R^-1(i, c), zero for i > c
  const int tid = threadIdx.x;
  const int64_t row = (int64_t)blockIdx.x * TR_ROWS + tid;
  const bool live = row < m;
  float y[KB];
#pragma unroll
  for (int i = 0; i < KB; ++i) y[i] = (live && i < K) ? Y[row + (int64_t)i * ld] : 0.f;
  // the loads of R^-1 are issued together (unrolled), behind those of the row:
  // the prologue costs one memory latency
  constexpr int MU = (KB * KB + TR_ROWS - 1) / TR_ROWS;
  float mv[MU];
#pragma unroll
  for (int u = 0; u < MU; ++u) {
    const int e = tid + u * TR_ROWS, c = e / KB, i = e - c * KB;
    mv[u] = (e < KB * KB && c < K && i <= c) ? Minv[i + (int64_t)c * ldm] : 0.f;
  }
#pragma unroll
  for (int u = 0; u < MU; ++u) {
    const int e = tid + u * TR_ROWS;
    if (e < KB * KB) Mc[e] = mv[u];
  }
  __syncthreads();
  if (!live) return;
#pragma unroll
  for (int c = 0; c < KB; ++c) {
    if (c < K) {
      const float4* mc = reinterpret_cast<const float4*>(Mc + c * KB);
      float s0 = 0.f, s1 = 0.f;
#pragma unroll
      for (int i4 = 0; i4 <= c / 4; ++i4) {
        const float4 w = mc[i4];
        s0 = fmaf(y[4 * i4], w.x, s0);
        s1 = fmaf(y[4 * i4 + 1], w.y, s1);
        s0 = fmaf(y[4 * i4 + 2], w.z, s0);
        s1 = fmaf(y[4 * i4 + 3], w.w, s1);
      }
      Y[row + (int64_t)c * ld] = s0 + s1;
    }
  }
}

constexpr int HH_THREADS = 1024;
constexpr int HH_GROUP = 8;

// Block-wide sum of up to HH_GROUP per-thread values; result broadcast in out[].
__device__ void block_sum_group(float (&v)[HH_GROUP], int nv, double* red, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = 0; t < nv; ++t) {
    double d = warp_sum((double)v[t]);
    if (lane == 0) red[warp * HH_GROUP + t] = d;
  }
  __syncthreads();
  if (warp == 0) {
    for (int t = 0; t < nv; ++t) {
      double d = red[lane * HH_GROUP + t];
      d = warp_sum(d);
      if (lane == 0) out[t] = d;
    }
  }
  __syncthreads();
}

// Apply H = I - tau v v^T, v = [1; A(j+1:m, j)], to columns c0..c1-1 of A, rows j..m-1.
__device__ void apply_reflector(float* A, int64_t m, int64_t ld, int j, double tau, int c0, int c1,
                                double* red, double* w) {
  const float* v = A + (int64_t)j * ld;
  for (int cg = c0; cg < c1; cg += HH_GROUP) {
    const int nc = min(HH_GROUP, c1 - cg);
    float part[HH_GROUP];
#pragma unroll
    for (int t = 0; t < HH_GROUP; ++t) part[t] = 0.f;
    for (int64_t i = j + 1 + threadIdx.x; i < m; i += HH_THREADS) {
      const float vi = v[i];
#pragma unroll
      for (int t = 0; t < HH_GROUP; ++t)
        if (t < nc) part[t] = fmaf(vi, A[i + (int64_t)(cg + t) * ld], part[t]);
    }
    if (threadIdx.x == 0) {
#pragma unroll
      for (int t = 0; t < HH_GROUP; ++t)
        if (t < nc) part[t] += A[j + (int64_t)(cg + t) * ld];
    }
    block_sum_group(part, nc, red, w);
    for (int64_t i = j + threadIdx.x; i < m; i += HH_THREADS) {
      const float vi = (i == j) ? 1.f : v[i];
      for (int t = 0; t < nc; ++t) A[i + (int64_t)(cg + t) * ld] -= (float)(tau * w[t]) * vi;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(HH_THREADS)
householder_kernel(float* A, int64_t m, int K, int64_t ld, DevStatus* st, int force) {
  if (!force && !st->orth_fail) return;
  __shared__ double red[32 * HH_GROUP];
  __shared__ double w[HH_GROUP];
  __shared__ double tau_s[RHOSVD_MAX_K];
  const int tid = threadIdx.x;
  // geqr2: reflectors stored below the diagonal, R on and above it
  for (int j = 0; j < K; ++j) {
    float* col = A + (int64_t)j * ld;
    float part[HH_GROUP];
    part[0] = 0.f;
    for (int64_t i = j + 1 + tid; i < m; i += HH_THREADS) part[0] = fmaf(col[i], col[i], part[0]);
    block_sum_group(part, 1, red, w);
    const double xnorm2 = w[0];
    const double alpha = col[j];
    double tau = 0.0;
    if (xnorm2 > 0.0) {
      const double beta = -copysign(sqrt(alpha * alpha + xnorm2), alpha);
      tau = (beta - alpha) / beta;
      const float scal = (float)(1.0 / (alpha - beta));
      for (int64_t i = j + 1 + tid; i < m; i += HH_THREADS) col[i] *= scal;
      __syncthreads();
      if (tid == 0) col[j] = (float)beta;
    }
    if (tid == 0) tau_s[j] = tau;
    __syncthreads();
    if (tau != 0.0) apply_reflector(A, m, ld, j, tau, j + 1, K, red, w);
  }
  // org2r: accumulate Q = H_1 ... H_K [I; 0] in place, last reflector first
  for (int j = K - 1; j >= 0; --j) {
    const double tau = tau_s[j];
    if (j < K - 1 && tau != 0.0) apply_reflector(A, m, ld, j, tau, j + 1, K, red, w);
    float* col = A + (int64_t)j * ld;
    for (int64_t i = tid; i < m; i += HH_THREADS) {
      if (i < j) col[i] = 0.f;
      else if (i == j) col[i] = (float)(1.0 - tau);
      else col[i] = (float)(-tau) * col[i];
    }
    __syncthreads();
  }
  if (tid == 0) {
    atomicOr(&st->flags, RHOSVD_FLAG_FALLBACK);
    st->fallbacks += 1;
    st->fallback_rows = (int32_t)(m < 2147483647 ? m : 2147483647);
    // a non-finite result means the input was already non-finite
    bool bad = false;
    for (int c = 0; c < K && !bad; ++c)
      if (!isfinite(A[c + (int64_t)c * ld])) bad = true;
    if (bad) set_error(st, RHOSVD_ENONFINITE);
  }
}

}  // namespace

template <int KB>
static cudaError_t launch_chol_kb(const double* G, int K, float* L, float* Minv, int ldm, int pass, int fail_code,
                                  DevStatus* st, cudaStream_t stream) {
  // Gram (FP64) + FP32 factor, + the inverse's working matrix when R^-1 is requested (K <= 64)
  const size_t smem = (size_t)K * K * (sizeof(double) + (Minv != nullptr ? 2 : 1) * sizeof(float));
  cudaError_t e = allow_dynamic_smem((const void*)chol_kernel<KB>,
                                     (size_t)KB * KB * (sizeof(double) + (KB <= 64 ? 2 : 1) * sizeof(float)));
  if (e != cudaSuccess) return e;
  chol_kernel<KB><<<1, CH_THREADS, smem, stream>>>(G, K, L, Minv, ldm, pass, fail_code, st);
  return cudaGetLastError();
}

cudaError_t launch_chol(const double* G, int K, float* L, float* Minv, int ldm, int pass, int fail_code,
                        DevStatus* st, cudaStream_t stream) {
  if (K <= 16) return launch_chol_kb<16>(G, K, L, Minv, ldm, pass, fail_code, st, stream);
  if (K <= 32) return launch_chol_kb<32>(G, K, L, Minv, ldm, pass, fail_code, st, stream);
  if (K <= 48) return launch_chol_kb<48>(G, K, L, Minv, ldm, pass, fail_code, st, stream);
  if (K <= 64) return launch_chol_kb<64>(G, K, L, Minv, ldm, pass, fail_code, st, stream);
  if (K <= 96) return launch_chol_kb<96>(G, K, L, nullptr, ldm, pass, fail_code, st, stream);
  return launch_chol_kb<128>(G, K, L, nullptr, ldm, pass, fail_code, st, stream);
}

template <int KB>
static cudaError_t launch_trsm_kb(float* Y, int64_t m, int K, int64_t ld, const float* L, int mode,
                                  const DevStatus* skip, cudaStream_t stream) {
  const size_t smem = (2 * (size_t)KB * KB + KB) * sizeof(float);
  cudaError_t e = allow_dynamic_smem((const void*)trsm_rows_kernel<KB>, smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((m + TR_ROWS - 1) / TR_ROWS);
  trsm_rows_kernel<KB><<<grid, TR_ROWS, smem, stream>>>(Y, m, K, ld, L, mode, skip);
  return cudaGetLastError();
}

cudaError_t launch_trsm_rows(float* Y, int64_t m, int K, int64_t ld, const float* L, int mode,
                             const DevStatus* skip, cudaStream_t stream) {
  if (m == 0) return cudaSuccess;
  if (K <= 16) return launch_trsm_kb<16>(Y, m, K, ld, L, mode, skip, stream);
  if (K <= 32) return launch_trsm_kb<32>(Y, m, K, ld, L, mode, skip, stream);
  if (K <= 48) return launch_trsm_kb<48>(Y, m, K, ld, L, mode, skip, stream);
  if (K <= 64) return launch_trsm_kb<64>(Y, m, K, ld, L, mode, skip, stream);
  if (K <= 96) return launch_trsm_kb<96>(Y, m, K, ld, L, mode, skip, stream);
  return launch_trsm_kb<128>(Y, m, K, ld, L, mode, skip, stream);
}

template <int KB>
static cudaError_t launch_rinv_kb(float* Y, int64_t m, int K, int64_t ld, const float* Minv, int ldm,
                                  const DevStatus* skip, cudaStream_t stream) {
  const unsigned grid = (unsigned)((m + TR_ROWS - 1) / TR_ROWS);
  apply_rinv_rows_kernel<KB><<<grid, TR_ROWS, 0, stream>>>(Y, m, K, ld, Minv, ldm, skip);
  return cudaGetLastError();
}

cudaError_t launch_apply_rinv_rows(float* Y, int64_t m, int K, int64_t ld, const float* Minv, int ldm,
                                   const DevStatus* skip, cudaStream_t stream) {
  if (m == 0) return cudaSuccess;
  if (K < 1 || K > RHOSVD_APPLY_RINV_MAX_K || ldm < K) return cudaErrorInvalidValue;
  if (K <= 16) return launch_rinv_kb<16>(Y, m, K, ld, Minv, ldm, skip, stream);
  if (K <= 32) return launch_rinv_kb<32>(Y, m, K, ld, Minv, ldm, skip, stream);
  if (K <= 48) return launch_rinv_kb<48>(Y, m, K, ld, Minv, ldm, skip, stream);
  return launch_rinv_kb<64>(Y, m, K, ld, Minv, ldm, skip, stream);
}

cudaError_t launch_householder(float* A, int64_t m, int K, int64_t ld, DevStatus* st, bool force,
                               cudaStream_t stream) {
  householder_kernel<<<1, HH_THREADS, 0, stream>>>(A, m, K, ld, st, force ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace rhosvd
