// Leading eigenvectors of a small symmetric positive semidefinite Gram matrix
// G = B B^T (K x K, FP64): the "SVD of B" step of Alg. 1 (steps 5-7) and the
// truncation of R-PET's recovered core (Alg. 9 line 5), where only the left
// singular vectors of B are needed (the EVD route of Sec. 4).
//
// Rather than rotating G itself (whose eigenvector accuracy in FP32 is limited
// by lambda_1 / (lambda_R - lambda_R+1)), G is first factored G = L L^T by a
// semidefinite Cholesky in FP64 (pivots at or below K * 1e-15 * max diag are
// dropped to zero columns), and the left singular vectors of L are found by
// one-sided (Hestenes) Jacobi on the columns of L^T in FP32 (Hestenes 1958;
// Demmel & Veselic 1992 for its relative accuracy): the rotations that make
// the columns of L^T V orthogonal accumulate V, the eigenvectors of G, and the
// column norms are the singular values sqrt(lambda).  Pairs are visited in the
// round-robin (circle) ordering so that K/2 rotations run at once, one warp each.
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace rhosvd {

namespace {

constexpr int EIG_THREADS = 1024;
constexpr int MAX_SWEEPS = 40;

__global__ void __launch_bounds__(EIG_THREADS)
small_eig_kernel(const double* __restrict__ G, int K, int R, float* __restrict__ Ub, float* __restrict__ sv,
                 DevStatus* st) {
  extern __shared__ double smem[];
  double* A = smem;                              // K x K FP64, then reused for M and V
  float* M = reinterpret_cast<float*>(smem);     // K x K FP32 (L^T)
  float* V = M + (size_t)K * K;                  // K x K FP32
  __shared__ double maxdiag;
  __shared__ int rotated;
  __shared__ int nonfinite;
  __shared__ float norms[RHOSVD_MAX_K];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  if (tid == 0) nonfinite = 0;
  __syncthreads();
  for (int e = tid; e < K * K; e += EIG_THREADS) {
    const double v = G[e];
    A[e] = v;
    if (!isfinite(v)) nonfinite = 1;
  }
  __syncthreads();
  if (nonfinite) {
    if (tid == 0) set_error(st, RHOSVD_ENONFINITE);
    for (int e = tid; e < K * R; e += EIG_THREADS) Ub[e] = 0.f;
    return;
  }
  if (tid == 0) {
    double m = 0.0;
    for (int i = 0; i < K; ++i) m = fmax(m, A[i + i * K]);
    maxdiag = m;
  }
  __syncthreads();
  const double tol = (double)K * 1e-15 * maxdiag;
  // semidefinite Cholesky, lower triangle in place
  for (int j = 0; j < K; ++j) {
    const double d = A[j + j * K];
    const bool keep = d > tol;
    const double ljj = keep ? sqrt(d) : 0.0;
    __syncthreads();
    if (tid == 0) A[j + j * K] = ljj;
    for (int i = j + 1 + tid; i < K; i += EIG_THREADS) A[i + j * K] = keep ? A[i + j * K] / ljj : 0.0;
    __syncthreads();
    const int n = K - j - 1;
    for (int e = tid; e < n * n; e += EIG_THREADS) {
      const int k = j + 1 + e / n, i = j + 1 + e % n;
      if (i >= k) A[i + k * K] -= A[i + j * K] * A[k + j * K];
    }
    __syncthreads();
  }
  // M = L^T (M(r, c) = L(c, r), zero below the diagonal of L^T), V = I, via registers
  constexpr int PER = (RHOSVD_MAX_K * RHOSVD_MAX_K + EIG_THREADS - 1) / EIG_THREADS;
  float tmp[PER];
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int e = tid + t * EIG_THREADS;
    float v = 0.f;
    if (e < K * K) {
      const int c = e / K, r = e % K;
      v = (c >= r) ? (float)A[c + r * K] : 0.f;
    }
    tmp[t] = v;
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int e = tid + t * EIG_THREADS;
    if (e < K * K) {
      M[e] = tmp[t];
      V[e] = ((e / K) == (e % K)) ? 1.f : 0.f;
    }
  }
  __syncthreads();

  const int n = K + (K & 1);            // even number of players (one dummy if K odd)
  const int npairs = n / 2;
  const int nwarps = EIG_THREADS / 32;
  const float jtol = 1e-6f;
  for (int sweep = 0; sweep < MAX_SWEEPS; ++sweep) {
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int s = 0; s < n - 1; ++s) {
      for (int w = warp; w < npairs; w += nwarps) {
        // circle method: slot 0 fixed, slots 1..n-1 rotate by s
        const int a = (w == 0) ? 0 : ((w - 1 + s) % (n - 1)) + 1;
        const int b = ((n - 1 - w - 1 + s) % (n - 1)) + 1;
        const int p = min(a, b), q = max(a, b);
        if (q >= K) continue;             // dummy partner
        float alpha = 0.f, beta = 0.f, gamma = 0.f;
        for (int r = lane; r < K; r += 32) {
          const float x = M[r + p * K], y = M[r + q * K];
          alpha = fmaf(x, x, alpha);
          beta = fmaf(y, y, beta);
          gamma = fmaf(x, y, gamma);
        }
        alpha = warp_sum(alpha);
        beta = warp_sum(beta);
        gamma = warp_sum(gamma);
        if (gamma != 0.f && fabsf(gamma) > jtol * sqrtf(alpha) * sqrtf(beta)) {
          const float zeta = (beta - alpha) / (2.f * gamma);
          const float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
          const float c = rsqrtf(1.f + t * t);
          const float sn = c * t;
          for (int r = lane; r < K; r += 32) {
            const float x = M[r + p * K], y = M[r + q * K];
            M[r + p * K] = c * x - sn * y;
            M[r + q * K] = sn * x + c * y;
            const float vx = V[r + p * K], vy = V[r + q * K];
            V[r + p * K] = c * vx - sn * vy;
            V[r + q * K] = sn * vx + c * vy;
          }
          if (lane == 0) rotated = 1;
        }
      }
      __syncthreads();
    }
    const int any = rotated;
    __syncthreads();
    if (!any) break;
  }
  // singular values = column norms of M; order descending (ties by index)
  for (int c = warp; c < K; c += nwarps) {
    float s = 0.f;
    for (int r = lane; r < K; r += 32) s = fmaf(M[r + c * K], M[r + c * K], s);
    s = warp_sum(s);
    if (lane == 0) norms[c] = sqrtf(s);
  }
  __syncthreads();
  for (int c = tid; c < K; c += EIG_THREADS) {
    int rank = 0;
    const float nc = norms[c];
    for (int o = 0; o < K; ++o) {
      const float no = norms[o];
      rank += (no > nc) || (no == nc && o < c);
    }
    if (sv != nullptr) sv[rank] = nc;
    if (rank < R)
      for (int r = 0; r < K; ++r) Ub[r + rank * K] = V[r + c * K];
  }
}

}  // namespace

cudaError_t launch_small_eig(const double* G, int K, int R, float* Ub, float* sv, DevStatus* st,
                             cudaStream_t stream) {
  const size_t smem = (size_t)K * K * sizeof(double);
  cudaError_t e = allow_dynamic_smem((const void*)small_eig_kernel,
                                     (size_t)RHOSVD_MAX_K * RHOSVD_MAX_K * sizeof(double));
  if (e != cudaSuccess) return e;
  small_eig_kernel<<<1, EIG_THREADS, smem, stream>>>(G, K, R, Ub, sv, st);
  return cudaGetLastError();
}

}  // namespace rhosvd
