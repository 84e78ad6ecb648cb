// Small dense factorisations shared by the CholeskyQR kernel (orth.cu) and the
// truncation kernel (eig.cu).
#pragma once

#include "common.cuh"

namespace rhosvd {

constexpr int CHOL_GRID_THREADS = 256;

// Arithmetic policies for the small factorisation: FP32, or double-word FP32
// pairs (common.cuh) where FP64-level precision is needed without the FP64 pipe.
struct F32Ops {
  using T = float;
  __device__ static T from(double v) { return __double2float_rn(v); }
  __device__ static T zero() { return 0.f; }
  __device__ static T mul(T a, T b) { return a * b; }
  __device__ static T sub(T a, T b) { return a - b; }
  __device__ static T rsqrt(T d) { return rsqrtf(d); }
  __device__ static float hi(T a) { return a; }
};
struct DWOps {
  using T = df64;
  __device__ static T from(double v) { return dw_from_double(v); }
  __device__ static T zero() { return df64{0.f, 0.f}; }
  __device__ static T mul(T a, T b) { return dw_mul(a, b); }
  __device__ static T sub(T a, T b) { return dw_add(a, dw_neg(b)); }
  __device__ static T rsqrt(T d) { return dw_rsqrt(d); }
  __device__ static float hi(T a) { return a.hi; }
};

// Right-looking Cholesky of Gs * 2^-e (Gs: K x K FP64 in shared memory, e even
// so that the scaling and its undoing are exact) on a 16 x 16 grid of the
// block's first 256 threads (the others only join the barriers).
// Step j writes column j of L' (scaled by 1/sqrt(pivot)) to out and updates
// the trailing lower triangle with the unscaled column, A(i,k) -= A(i,j)
// A(k,j) / d.  The next pivot's 1/sqrt is computed once, by the thread that
// finalises it (thread 0 updates A(j+1,j+1)), and broadcast through shared
// memory, so each step needs one barrier.  semidef: a pivot at or below tol
// gives a zero column instead of failure.  out (FP32, column-major, zero above
// the diagonal) receives L = 2^(e/2) L'.  Returns false (uniformly) on failure.
template <class Ops>
__device__ bool chol_grid(const double* Gs, int K, int e, double tol, bool semidef,
                          float* __restrict__ out, typename Ops::T* A, typename Ops::T* rs_s, int* flag) {
  using T = typename Ops::T;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const bool active = tid < CHOL_GRID_THREADS;     // larger blocks only join the barriers
  if (active)
    for (int c = ty; c < K; c += 16)
      for (int r = tx; r < K; r += 16) A[r + c * K] = (r >= c) ? Ops::from(ldexp(Gs[r + c * K], -e)) : Ops::zero();
  __syncthreads();
  const float scale = ldexpf(1.f, e / 2);
  if (tid == 0) {
    *flag = 0;
    const T d0 = A[0];
    if (Ops::hi(d0) > (float)tol) rs_s[0] = Ops::rsqrt(d0);
    else if (semidef) rs_s[0] = Ops::zero();
    else *flag = 1;
  }
  __syncthreads();
  for (int j = 0; j < K; ++j) {
    if (*flag) return false;                       // uniform: set before the last barrier
    const T rs = rs_s[j];
    const float rsh = Ops::hi(rs);
    if (active)
      for (int i = j + tid; i < K; i += CHOL_GRID_THREADS) out[i + j * K] = Ops::hi(A[i + j * K]) * rsh * scale;
    if (rsh != 0.f && active) {
      const T r2 = Ops::mul(rs, rs);
      for (int i = j + 1 + ty; i < K; i += 16) {
        const T aij = Ops::mul(A[i + j * K], r2);
        for (int k = j + 1 + tx; k <= i; k += 16) A[i + k * K] = Ops::sub(A[i + k * K], Ops::mul(aij, A[k + j * K]));
      }
    }
    if (tid == 0 && j + 1 < K) {                   // thread (0,0) owns A(j+1, j+1)
      const T dn = A[(j + 1) + (j + 1) * K];
      if (Ops::hi(dn) > (float)tol) rs_s[j + 1] = Ops::rsqrt(dn);
      else if (semidef) rs_s[j + 1] = Ops::zero();
      else *flag = 1;
    }
    __syncthreads();
  }
  if (active)
    for (int c = ty; c < K; c += 16)
      for (int r = tx; r < c; r += 16) out[r + c * K] = 0.f;
  return true;
}

}  // namespace rhosvd
