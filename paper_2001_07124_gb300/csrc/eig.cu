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
constexpr int MAX_SWEEPS = 30;

__global__ void __launch_bounds__(EIG_THREADS)
small_eig_kernel(const double* __restrict__ G, int K, int R, float* __restrict__ Ub, float* __restrict__ sv,
                 DevStatus* st) {
  extern __shared__ double smem[];
  double* A = smem;                                       // K x K FP64 (scaled Gram), then M and V
  float* Lf = reinterpret_cast<float*>(smem + (size_t)K * K);   // K x K FP32 Cholesky factor
  float* M = reinterpret_cast<float*>(smem);              // K x K FP32 (L^T)
  float* V = M + (size_t)K * K;                           // K x K FP32
  __shared__ double maxdiag;
  __shared__ int rotated;
  __shared__ int nonfinite;
  __shared__ float norms[RHOSVD_MAX_K];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tx = tid & 31, ty = tid >> 5;                 // 32 x 32 thread grid

  if (tid == 0) nonfinite = 0;
  if (warp == 0) {
    double m = 0.0;
    for (int i = lane; i < K; i += 32) m = fmax(m, G[i + i * K]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) maxdiag = m;
  }
  __syncthreads();
  const double ginv = (maxdiag > 0.0) ? 1.0 / maxdiag : 0.0;
  for (int c = ty; c < K; c += 32)
    for (int r = tx; r < K; r += 32) {
      const double v = G[r + c * K];
      if (!isfinite(v)) nonfinite = 1;
      A[r + c * K] = (r >= c) ? v * ginv : 0.0;
      Lf[r + c * K] = 0.f;
    }
  __syncthreads();
  if (nonfinite || !isfinite(maxdiag)) {
    if (tid == 0) set_error(st, RHOSVD_ENONFINITE);
    for (int e = tid; e < K * R; e += EIG_THREADS) Ub[e] = 0.f;
    return;
  }
  // semidefinite Cholesky of the scaled Gram (pivots at or below K * 1e-15 are
  // dropped to zero columns), one barrier per step: column j of L goes to Lf,
  // the trailing update uses the unscaled column divided by its pivot.  The
  // per-step 1/sqrt(d) (0 for a dropped pivot) is computed once by the thread
  // that finalises the next pivot and broadcast (the FP64 pipe is narrow).
  __shared__ double rs_s[RHOSVD_MAX_K];
  const double tol = (double)K * 1e-15;
  if (tid == 0) rs_s[0] = (A[0] > tol) ? rsqrt_newton(A[0]) : 0.0;
  __syncthreads();
  for (int j = 0; j < K; ++j) {
    const double rs = rs_s[j];
    if (rs != 0.0) {                         // uniform
      const double r2 = rs * rs;
      for (int i = j + tid; i < K; i += EIG_THREADS) Lf[i + j * K] = (float)(A[i + j * K] * rs);
      for (int i = j + 1 + ty; i < K; i += 32) {
        const double aij = A[i + j * K] * r2;
        for (int k = j + 1 + tx; k <= i; k += 32) A[i + k * K] -= aij * A[k + j * K];
      }
    }
    if (tid == 0 && j + 1 < K) {             // thread (0,0) owns A(j+1, j+1)
      const double dn = A[(j + 1) + (j + 1) * K];
      rs_s[j + 1] = (dn > tol) ? rsqrt_newton(dn) : 0.0;
    }
    __syncthreads();
  }
  // M = L^T (M(r, c) = L(c, r)), V = I
  for (int c = ty; c < K; c += 32)
    for (int r = tx; r < K; r += 32) {
      M[r + c * K] = Lf[c + r * K];
      V[r + c * K] = (r == c) ? 1.f : 0.f;
    }
  __syncthreads();

  const int n = K + (K & 1);            // even number of players (one dummy if K odd)
  const int npairs = n / 2;
  const int nwarps = EIG_THREADS / 32;
  const float jtol = 1e-6f;
  // Squared column norms alpha_c are kept in shared memory: a rotation with
  // tangent t changes them by -t*gamma and +t*gamma exactly (the Hestenes
  // update), so each pair needs only its inner product gamma.  They are
  // recomputed from M at the start of every sweep to shed rounding drift.
  int sweeps = 0;
  for (int sweep = 0; sweep < MAX_SWEEPS; ++sweep) {
    sweeps = sweep + 1;
    for (int c = warp; c < K; c += nwarps) {
      float s2 = 0.f;
      for (int r = lane; r < K; r += 32) s2 = fmaf(M[r + c * K], M[r + c * K], s2);
      s2 = warp_sum(s2);
      if (lane == 0) norms[c] = s2;
    }
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int s = 0; s < n - 1; ++s) {
      for (int w = warp; w < npairs; w += nwarps) {
        // circle method: slot 0 fixed, slots 1..n-1 rotate by s
        int xa = w - 1 + s, xb = n - 2 - w + s;          // both < 2(n-1)
        if (xa >= n - 1) xa -= n - 1;
        if (xb >= n - 1) xb -= n - 1;
        const int a = (w == 0) ? 0 : xa + 1;
        const int b = xb + 1;
        const int p = min(a, b), q = max(a, b);
        if (q >= K) continue;             // dummy partner
        float gamma = 0.f;
        for (int r = lane; r < K; r += 32) gamma = fmaf(M[r + p * K], M[r + q * K], gamma);
        gamma = warp_sum(gamma);
        const float alpha = norms[p], beta = norms[q];
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
          if (lane == 0) {
            norms[p] = fmaxf(alpha - t * gamma, 0.f);
            norms[q] = beta + t * gamma;
            rotated = 1;
          }
        }
      }
      __syncthreads();
    }
    const int any = rotated;
    __syncthreads();
    if (!any) break;
  }
  if (tid == 0) atomicMax(&st->eig_sweeps, sweeps);
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
    if (sv != nullptr) sv[rank] = nc * (float)sqrt(maxdiag);
    if (rank < R)
      for (int r = 0; r < K; ++r) Ub[r + rank * K] = V[r + c * K];
  }
}

}  // namespace

cudaError_t launch_small_eig(const double* G, int K, int R, float* Ub, float* sv, DevStatus* st,
                             cudaStream_t stream) {
  const size_t smem = (size_t)K * K * (sizeof(double) + sizeof(float));
  cudaError_t e = allow_dynamic_smem((const void*)small_eig_kernel,
                                     (size_t)RHOSVD_MAX_K * RHOSVD_MAX_K * (sizeof(double) + sizeof(float)));
  if (e != cudaSuccess) return e;
  small_eig_kernel<<<1, EIG_THREADS, smem, stream>>>(G, K, R, Ub, sv, st);
  return cudaGetLastError();
}

}  // namespace rhosvd
