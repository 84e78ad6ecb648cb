// Leading eigenvectors of a small symmetric positive semidefinite Gram matrix
// G = B B^T (K x K, FP64): the SVD of the small projected matrix B in Alg. 1
// and the truncation of R-PET's recovered core (Alg. 9), where only the left
// singular vectors of B are needed (the EVD route of Sec. 4).
//
// Rotating G itself in FP32 would limit eigenvector accuracy by
// lambda_1 / (lambda_R - lambda_R+1).  Instead G is factored G = L L^T by a
// semidefinite Cholesky in double-word arithmetic (pivots at or below
// K * 1e-14 * max diag give zero columns), and the left singular vectors of L
// are found by one-sided Jacobi (Hestenes 1958) on the columns of L itself --
// the preconditioned orientation of Drmac & Veselic (2008): B^T = Q_B R with
// R = L^T, and Jacobi on R^T = L converges in few sweeps.  At convergence
// L V = U Sigma, so U is the normalised columns of the rotated L and V is never
// accumulated; accuracy is set by sigma_1 / (sigma_R - sigma_R+1) in FP32.
// Pairs follow the round-robin (circle) ordering; each rotation is handled by
// a group of 8 lanes (4 pairs per warp, 3-shuffle dot products), which keeps
// the number of warps, and so the issue slots a round takes, small.
// Columns at FP32 noise level (rank below R) are replaced by an orthonormal
// completion (Gram-Schmidt on unit vectors).
#include <math.h>

#include "common.cuh"
#include "kernels.h"
#include "small_la.cuh"

namespace rhosvd {

namespace {

constexpr int MAX_SWEEPS = 30;
constexpr int PAIR_LANES = 8;            // lanes per rotation pair

template <int KB>                        // KB >= K, a multiple of 16
__global__ void __launch_bounds__(512, 1)
small_eig_kernel(const double* __restrict__ G, int K, int R, float* __restrict__ Ub, int ldu,
                 float* __restrict__ sv, DevStatus* st) {
  extern __shared__ __align__(16) unsigned char eig_smem[];
  double* Gs = reinterpret_cast<double*>(eig_smem);                       // K x K FP64, then the DW factor
  float* X = reinterpret_cast<float*>(eig_smem + (size_t)K * K * sizeof(double));   // K x K FP32
  __shared__ float norms[RHOSVD_MAX_K];
  __shared__ int order[RHOSVD_MAX_K];
  __shared__ df64 rs_dw[RHOSVD_MAX_K];
  __shared__ double maxdiag;
  __shared__ int nonfinite, flag, rotated;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;

  if (tid == 0) nonfinite = 0;
  __syncthreads();
  #pragma unroll 8
  for (int e = tid; e < K * K; e += blockDim.x) {      // one bulk load, independent requests
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
  __syncthreads();
  if (nonfinite || !isfinite(maxdiag)) {
    if (tid == 0) set_error(st, RHOSVD_ENONFINITE);
    for (int e = tid; e < K * R; e += blockDim.x) Ub[(e % K) + (e / K) * ldu] = 0.f;
    return;
  }
  int e2 = 0;
  if (maxdiag > 0.0) {
    e2 = 2 * (ilogb(maxdiag) / 2);
    chol_grid<DWOps, KB>(Gs, K, e2, (double)K * 1e-14 * ldexp(maxdiag, -e2), true, X,
                         reinterpret_cast<df64*>(Gs), rs_dw, &flag);
  } else {
    for (int e = tid; e < K * K; e += blockDim.x) X[e] = 0.f;
  }
  __syncthreads();
  // ------------------------------------------------ one-sided Jacobi on the columns of X = L
  const int n = K + (K & 1);
  const int npairs = n / 2;
  const float jtol = 2e-6f;
  for (int sweep = 0; sweep < MAX_SWEEPS; ++sweep) {
    for (int c = warp; c < K; c += nwarps) {
      float s2 = 0.f;
      for (int r = lane; r < K; r += 32) s2 = fmaf(X[r + c * K], X[r + c * K], s2);
      s2 = warp_sum(s2);
      if (lane == 0) norms[c] = s2;
    }
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int s = 0; s < n - 1; ++s) {
      const int g = lane / PAIR_LANES, gl = lane % PAIR_LANES;
      for (int w = warp * (32 / PAIR_LANES) + g; w < npairs + g; w += nwarps * (32 / PAIR_LANES)) {
        // every lane of the warp takes part in the shuffles; groups past the last pair idle
        const bool live = w < npairs;
        int xa = w - 1 + s, xb = n - 2 - w + s;          // circle method, both < 2(n-1)
        if (xa >= n - 1) xa -= n - 1;
        if (xb >= n - 1) xb -= n - 1;
        const int a = (w == 0) ? 0 : xa + 1, b = xb + 1;
        const int p = min(a, b), q = live ? max(a, b) : K;
        // the pair's columns stay in registers from the dot product to the rotation
        constexpr int NR = KB / PAIR_LANES;
        float xv[NR], yv[NR];
        float gamma = 0.f;
#pragma unroll
        for (int u = 0; u < NR; ++u) {
          const int r = gl + PAIR_LANES * u;
          const bool in = (q < K) && (r < K);
          xv[u] = in ? X[r + p * K] : 0.f;
          yv[u] = in ? X[r + q * K] : 0.f;
          gamma = fmaf(xv[u], yv[u], gamma);
        }
#pragma unroll
        for (int o = PAIR_LANES / 2; o > 0; o >>= 1) gamma += __shfl_xor_sync(0xffffffffu, gamma, o);
        if (q >= K) continue;
        const float alpha = norms[p], beta = norms[q];
        // gamma != 0 implies alpha, beta > 0; sqrt(v) = v * rsqrt(v) avoids the product's underflow
        if (gamma != 0.f && fabsf(gamma) > jtol * (alpha * rsqrtf(alpha)) * (beta * rsqrtf(beta))) {
          // t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)); c, s from t keep the rotation
          // orthogonal to rounding whatever t's own accuracy
          const float zeta = __fdividef(beta - alpha, 2.f * gamma);
          const float az = fabsf(zeta);
          float t;
          if (az < 1e15f) {
            const float h = fmaf(zeta, zeta, 1.f);
            t = __fdividef(1.f, az + h * rsqrtf(h));
          } else {
            t = __fdividef(0.5f, az);
          }
          t = copysignf(t, zeta);
          const float c = rsqrtf(fmaf(t, t, 1.f));
          const float sn = c * t;
#pragma unroll
          for (int u = 0; u < NR; ++u) {
            const int r = gl + PAIR_LANES * u;
            if (r < K) {
              X[r + p * K] = c * xv[u] - sn * yv[u];
              X[r + q * K] = sn * xv[u] + c * yv[u];
            }
          }
          if (gl == 0) {
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
    if (!any) {
      if (tid == 0) atomicMax(&st->eig_sweeps, sweep + 1);
      break;
    }
  }
  // ------------------------------------------------ order by singular value, normalise
  for (int c = warp; c < K; c += nwarps) {
    float s2 = 0.f;
    for (int r = lane; r < K; r += 32) s2 = fmaf(X[r + c * K], X[r + c * K], s2);
    s2 = warp_sum(s2);
    if (lane == 0) norms[c] = sqrtf(s2);
  }
  __syncthreads();
  if (tid < K) {
    const int c = tid;
    const float nc = norms[c];
    int rank = 0;
    for (int o = 0; o < K; ++o) rank += (norms[o] > nc) || (norms[o] == nc && o < c);
    order[rank] = c;
    if (sv != nullptr) sv[rank] = nc;          // X holds the unscaled factor L (chol_grid undoes 2^-e2)
  }
  __syncthreads();
  const float smax = norms[order[0]];
  for (int e = tid; e < K * R; e += blockDim.x) {
    const int rank = e / K, r = e - rank * K;
    const int c = order[rank];
    const float nc = norms[c];
    Ub[r + rank * ldu] = (nc > 1e-6f * smax && nc > 0.f) ? X[r + c * K] / nc : 0.f;
  }
  __syncthreads();
  if (tid == 0) {
    // orthonormal completion of columns at noise level (only when rank < R)
    int e_next = 0;
    for (int rank = 0; rank < R; ++rank) {
      const float nc = norms[order[rank]];
      if (nc > 1e-6f * smax && nc > 0.f) continue;
      for (; e_next < K; ++e_next) {
        float* u = Ub + rank * ldu;
        for (int r = 0; r < K; ++r) u[r] = (r == e_next) ? 1.f : 0.f;
        for (int pass = 0; pass < 2; ++pass)
          for (int o = 0; o < R; ++o) {
            if (o == rank) continue;
            const float* v = Ub + o * ldu;
            float d = 0.f, vv = 0.f;
            for (int r = 0; r < K; ++r) {
              d = fmaf(v[r], u[r], d);
              vv = fmaf(v[r], v[r], vv);
            }
            if (vv > 0.5f)
              for (int r = 0; r < K; ++r) u[r] = fmaf(-d, v[r], u[r]);
          }
        float uu = 0.f;
        for (int r = 0; r < K; ++r) uu = fmaf(u[r], u[r], uu);
        if (uu > 0.25f) {
          const float inv = rsqrtf(uu);
          for (int r = 0; r < K; ++r) u[r] *= inv;
          ++e_next;
          break;
        }
      }
    }
  }
  // ------------------------------------------------ orthonormality polish
  // The Jacobi stop (column cosines <= jtol) leaves the columns orthonormal to
  // about 2e-6.  One first-order step of U <- U (U^T U)^(-1/2), namely
  // U <- U - U D / 2 with D = U^T U - I, brings that to FP32 rounding level; it
  // multiplies U from the right by an invertible R x R matrix, so range(U)
  // (the truncation's subspace) is unchanged.  D is formed with compensated
  // dot products (Ogita, Rump & Oishi 2005, Dot2) since its entries are
  // differences from 1 far below the FP32 unit roundoff of the diagonal.
  __syncthreads();
  float* Us = X;                                            // K x R copy of the columns (X is free now)
  float* D = reinterpret_cast<float*>(Gs);                 // R x R, fits in the K x K FP64 region
  for (int e = tid; e < K * R; e += blockDim.x) {
    const int r = e % K, a = e / K;
    Us[r + a * K] = Ub[r + a * ldu];
  }
  __syncthreads();
  for (int e = tid; e < R * R; e += blockDim.x) {
    const int a = e % R, b = e / R;
    const float* ua = Us + a * K;
    const float* ub = Us + b * K;
    float sum = 0.f, comp = 0.f;
    for (int r = 0; r < K; ++r) {
      // _rn intrinsics: never contracted into FMAs, so the error terms stay exact
      const float p = __fmul_rn(ua[r], ub[r]);
      const float pe = fmaf(ua[r], ub[r], -p);             // exact product error
      const float t = __fadd_rn(sum, p);                    // two-sum of sum and p
      const float bv = __fsub_rn(t, sum);
      comp += __fadd_rn(__fsub_rn(sum, __fsub_rn(t, bv)), __fsub_rn(p, bv)) + pe;
      sum = t;
    }
    D[a + b * R] = (sum - (a == b ? 1.f : 0.f)) + comp;
  }
  __syncthreads();
  for (int e = tid; e < K * R; e += blockDim.x) {
    const int r = e % K, a = e / K;
    float corr = 0.f;
    for (int b = 0; b < R; ++b) corr = fmaf(Us[r + b * K], D[b + a * R], corr);
    Ub[r + a * ldu] = fmaf(-0.5f, corr, Us[r + a * K]);
  }
}

template <int KB>
static cudaError_t launch_eig_kb(const double* G, int K, int R, float* Ub, int ldu, float* sv, DevStatus* st,
                                 cudaStream_t stream) {
  const size_t smem = (size_t)K * K * (sizeof(double) + sizeof(float));
  cudaError_t e = allow_dynamic_smem((const void*)small_eig_kernel<KB>,
                                     (size_t)KB * KB * (sizeof(double) + sizeof(float)));
  if (e != cudaSuccess) return e;
  // one 8-lane group per rotation pair, at least the 256 threads the factorisation uses
  const int npairs = (K + 1) / 2;
  int warps = (npairs + 32 / PAIR_LANES - 1) / (32 / PAIR_LANES);
  warps = warps < 8 ? 8 : warps;
  small_eig_kernel<KB><<<1, 32 * warps, smem, stream>>>(G, K, R, Ub, ldu, sv, st);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_small_eig(const double* G, int K, int R, float* Ub, int ldu, float* sv, DevStatus* st,
                             cudaStream_t stream) {
  if (K <= 16) return launch_eig_kb<16>(G, K, R, Ub, ldu, sv, st, stream);
  if (K <= 32) return launch_eig_kb<32>(G, K, R, Ub, ldu, sv, st, stream);
  if (K <= 48) return launch_eig_kb<48>(G, K, R, Ub, ldu, sv, st, stream);
  if (K <= 64) return launch_eig_kb<64>(G, K, R, Ub, ldu, sv, st, stream);
  if (K <= 96) return launch_eig_kb<96>(G, K, R, Ub, ldu, sv, st, stream);
  return launch_eig_kb<128>(G, K, R, Ub, ldu, sv, st, stream);
}

}  // namespace rhosvd
