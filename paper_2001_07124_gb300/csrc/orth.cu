// Thin orthonormalisation of a tall m x K matrix (Alg. 1 step 3, Alg. 6 line 4,
// Alg. 9 line 2): CholeskyQR2 with a Householder fallback.
//
// CholeskyQR2 (Fukaya, Nakatsukasa, Yanagisawa, Yamamoto 2014; Yamamoto et al.
// 2015): G = Y^T Y, R = chol(G), Q1 = Y R^-1, repeated once on Q1.  The Gram is
// accumulated in double-float (FP64-accurate, see sketch.cu) and the Cholesky
// and triangular inverse run in FP64 on one CTA; the apply is the TTM kernel.
// The first pass only rejects pivots that are numerically non-positive
// (<= K * 1e-15 * max diag): for larger condition numbers Q1 = Y R^-1 is still
// formed and the second pass judges it; a second-pass pivot below 1e-4 * max
// diag (cond(Q1) above 100, so Q2 would not be orthonormal to FP32 accuracy)
// or a non-finite value marks a breakdown; the later kernels of the sequence
// then skip and a Householder QR
// (Golub & Van Loan Alg. 5.2.1 with the LAPACK geqr2/org2r conventions) forms
// Q instead.  The decision is taken on the device, so nothing synchronises.
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace rhosvd {

namespace {

constexpr int CH_THREADS = 256;

__global__ void __launch_bounds__(CH_THREADS)
chol_inv_kernel(const double* __restrict__ G, int K, float* __restrict__ Rinv, int pass, int fail_code,
                DevStatus* st) {
  if (pass == 1 && st->orth_fail) return;
  extern __shared__ double A[];          // K x K, A[i + j*K]
  double* diag = A + (size_t)K * K;      // K entries: diagonal of L^-1
  __shared__ int fail;
  __shared__ int nonfinite;
  __shared__ double maxdiag;
  const int tid = threadIdx.x;
  if (tid == 0) {
    fail = 0;
    nonfinite = 0;
    maxdiag = 0.0;
  }
  __syncthreads();
  for (int e = tid; e < K * K; e += CH_THREADS) {
    const double v = G[e];
    A[e] = v;
    if (!isfinite(v)) nonfinite = 1;
  }
  __syncthreads();
  if (tid == 0) {
    double m = 0.0;
    for (int i = 0; i < K; ++i) m = fmax(m, A[i + i * K]);
    maxdiag = m;
    if (nonfinite || !(m > 0.0)) fail = 1;
  }
  __syncthreads();
  const double tol = (pass == 0 ? (double)K * 1e-15 : 1e-4) * maxdiag;
  for (int j = 0; j < K && !fail; ++j) {
    if (tid == 0) {
      const double d = A[j + j * K];
      if (!(d > tol)) fail = 1;
      else A[j + j * K] = sqrt(d);
    }
    __syncthreads();
    if (fail) break;
    const double ljj = A[j + j * K];
    for (int i = j + 1 + tid; i < K; i += CH_THREADS) A[i + j * K] /= ljj;
    __syncthreads();
    // trailing update of the lower triangle: A[i,k] -= L[i,j] L[k,j], j < k <= i
    const int n = K - j - 1;
    for (int e = tid; e < n * n; e += CH_THREADS) {
      const int k = j + 1 + e / n, i = j + 1 + e % n;
      if (i >= k) A[i + k * K] -= A[i + j * K] * A[k + j * K];
    }
    __syncthreads();
  }
  if (fail) {
    if (tid == 0) {
      st->orth_fail = 1;
      if (nonfinite) set_error(st, RHOSVD_ENONFINITE);
      else if (fail_code != 0) set_error(st, fail_code);
    }
    return;
  }
  // L^-1 column c by thread c (forward substitution); L^-1(i,c), i > c, is kept
  // in the unused strict upper triangle at A[c + i*K], its diagonal in diag[].
  for (int c = tid; c < K; c += CH_THREADS) {
    diag[c] = 1.0 / A[c + c * K];
    for (int i = c + 1; i < K; ++i) {
      double s = A[i + c * K] * diag[c];
      for (int k = c + 1; k < i; ++k) s += A[i + k * K] * A[c + k * K];
      A[c + i * K] = -s / A[i + i * K];
    }
  }
  __syncthreads();
  // R^-1 = (L^T)^-1 = (L^-1)^T: R^-1(r, c) = L^-1(c, r), upper triangular
  for (int e = tid; e < K * K; e += CH_THREADS) {
    const int c = e / K, r = e % K;
    float v = 0.f;
    if (r < c) v = (float)A[r + c * K];
    else if (r == c) v = (float)diag[r];
    Rinv[e] = v;
  }
  if (pass == 0 && tid == 0) st->orth_fail = 0;
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

cudaError_t launch_chol_inv(const double* G, int K, float* Rinv, int pass, int fail_code, DevStatus* st,
                            cudaStream_t stream) {
  const size_t smem = ((size_t)K * K + K) * sizeof(double);
  static const size_t kMax = ((size_t)RHOSVD_MAX_K * RHOSVD_MAX_K + RHOSVD_MAX_K) * sizeof(double);
  cudaError_t e = allow_dynamic_smem((const void*)chol_inv_kernel, kMax);
  if (e != cudaSuccess) return e;
  chol_inv_kernel<<<1, CH_THREADS, smem, stream>>>(G, K, Rinv, pass, fail_code, st);
  return cudaGetLastError();
}

cudaError_t launch_householder(float* A, int64_t m, int K, int64_t ld, DevStatus* st, bool force,
                               cudaStream_t stream) {
  householder_kernel<<<1, HH_THREADS, 0, stream>>>(A, m, K, ld, st, force ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace rhosvd
