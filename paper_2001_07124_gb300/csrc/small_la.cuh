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
  __device__ static T from_scaled(double v, int e) { return dw_from_double_scaled(v, e).hi; }
  __device__ static T zero() { return 0.f; }
  __device__ static T mul(T a, T b) { return a * b; }
  __device__ static T sub(T a, T b) { return a - b; }
  __device__ static T rsqrt(T d) { return rsqrtf(d); }
  __device__ static float hi(T a) { return a; }
};
struct DWOps {
  using T = df64;
  __device__ static T from(double v) { return dw_from_double(v); }
  __device__ static T from_scaled(double v, int e) { return dw_from_double_scaled(v, e); }
  __device__ static T zero() { return df64{0.f, 0.f}; }
  __device__ static T mul(T a, T b) { return dw_mul(a, b); }
  // the trailing update only needs backward stability: the cheaper DW sum suffices
  __device__ static T sub(T a, T b) { return dw_add_sloppy(a, dw_neg(b)); }
  __device__ static T rsqrt(T d) { return dw_rsqrt(d); }
  __device__ static float hi(T a) { return a.hi; }
};

// Right-looking Cholesky of Gs * 2^-e (Gs: K x K FP64 in shared memory, e even
// so that the scaling and its undoing are exact) on a 16 x 16 grid of the
// block's first 256 threads (the others only join the barriers).
// Step j writes column j of L' (scaled by 1/sqrt(pivot)) to out and updates
// the trailing lower triangle with the unscaled column, A(i,k) -= A(i,j)
// A(k,j) / d.  The next pivot's 1/sqrt is computed once, by the thread that
// finalises it (thread 0 updates A(j+1,j+1), first among its rows), and
// broadcast through shared memory, so each step needs one barrier.  Each row's
// shared-memory loads are issued together before its arithmetic, so a step
// costs about one load latency per row instead of one per element.  semidef: a pivot at or below tol
// gives a zero column instead of failure.  out (FP32, column-major, zero above
// the diagonal) receives L = 2^(e/2) L'.  Returns false (uniformly) on failure.
//
// With Tinv != nullptr (K x K FP32 shared memory) the same steps also run
// forward substitution for L X = I on every column of I at once, right-looking:
// at step j row j of Tinv is final, x_j = Tinv(j, c) / L(j, j), and every row
// i > j takes Tinv(i, c) -= L(i, j) x_j; on return Tinv(i, c) / L(i, i) =
// (L^-1)(i, c).
// Thread (ty, tx) owns rows i = ty + 16m and columns c = tx + 16n, so no extra
// barrier is needed (L(i, j) comes from the shared column j of A).
template <class Ops, int KB>                       // KB >= K, a multiple of 16
__device__ bool chol_grid(const double* Gs, int K, int e, double tol, bool semidef,
                          float* __restrict__ out, typename Ops::T* A, typename Ops::T* rs_s, int* flag,
                          float* Tinv = nullptr) {
  using T = typename Ops::T;
  constexpr int NC = KB / 16;                      // columns per thread and step, at most
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const bool active = tid < CHOL_GRID_THREADS;     // larger blocks only join the barriers
  if (active)
    for (int c = ty; c < K; c += 16)
      for (int r = tx; r < K; r += 16) A[r + c * K] = (r >= c) ? Ops::from_scaled(Gs[r + c * K], e) : Ops::zero();
  if (active && Tinv != nullptr)
    for (int i = ty; i < K; i += 16)
      for (int c = tx; c < K; c += 16) Tinv[i + c * K] = (i == c) ? 1.f : 0.f;
  __syncthreads();
  const float scale = ldexpf(1.f, e / 2);
  const float tolf = (float)tol;                    // converted once (FP64 pipe)
  if (tid == 0) {
    *flag = 0;
    const T d0 = A[0];
    if (Ops::hi(d0) > tolf) rs_s[0] = Ops::rsqrt(d0);
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
    const bool upd = rsh != 0.f && active;
    if (upd && Tinv != nullptr) {
      // L(i, j) / L(j, j) = A(i, j) rs^2 (the scale 2^(e/2) cancels)
      const float r2h = rsh * rsh;
      float tj[NC];
#pragma unroll
      for (int n = 0; n < NC; ++n) {
        const int c = tx + 16 * n;
        tj[n] = (c <= j) ? Tinv[j + c * K] : 0.f;
      }
      for (int i = j + 1 + ty; i < K; i += 16) {
        const float m = Ops::hi(A[i + j * K]) * r2h;
        float v[NC];
#pragma unroll
        for (int n = 0; n < NC; ++n) {
          const int c = tx + 16 * n;
          if (c <= j) v[n] = Tinv[i + c * K];
        }
#pragma unroll
        for (int n = 0; n < NC; ++n) {
          const int c = tx + 16 * n;
          if (c <= j) Tinv[i + c * K] = fmaf(-m, tj[n], v[n]);
        }
      }
    }
    if (upd) {
      // trailing update A(i, k) -= A(i, j) A(k, j) / d for j < k <= i: column j of the
      // thread's k values is read once per step; each row's loads are issued together
      const T r2 = Ops::mul(rs, rs);
      T ck[NC];
#pragma unroll
      for (int n = 0; n < NC; ++n) {
        const int k = j + 1 + tx + 16 * n;
        ck[n] = (k < K) ? A[k + j * K] : Ops::zero();
      }
      for (int i = j + 1 + ty; i < K; i += 16) {
        const T aij = Ops::mul(A[i + j * K], r2);
        T v[NC];
#pragma unroll
        for (int n = 0; n < NC; ++n) {
          const int k = j + 1 + tx + 16 * n;
          if (k <= i) v[n] = A[i + k * K];
        }
#pragma unroll
        for (int n = 0; n < NC; ++n) {
          const int k = j + 1 + tx + 16 * n;
          if (k <= i) A[i + k * K] = Ops::sub(v[n], Ops::mul(aij, ck[n]));
        }
        if (tid == 0 && i == j + 1) {              // thread (0,0) has just finalised A(j+1, j+1)
          const T dn = A[(j + 1) + (j + 1) * K];
          if (Ops::hi(dn) > tolf) rs_s[j + 1] = Ops::rsqrt(dn);
          else if (semidef) rs_s[j + 1] = Ops::zero();
          else *flag = 1;
        }
      }
    } else if (tid == 0 && j + 1 < K) {            // zero column: the next pivot is unchanged
      const T dn = A[(j + 1) + (j + 1) * K];
      if (Ops::hi(dn) > tolf) rs_s[j + 1] = Ops::rsqrt(dn);
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
