// Gaussian test matrices Omega (the test matrices of Alg. 1) drawn from a counter-based
// generator: entry (j, k) depends only on (seed, stream_id, j, k), so any
// block of Omega can be produced by any thread in any order.
#include "common.cuh"
#include "kernels.h"

namespace rhosvd {

namespace {

// One thread per (row j, group of four columns); rows are contiguous in memory.
__global__ void omega_kernel(uint64_t seed, uint32_t stream_id, int64_t rows, int cols,
                             float* __restrict__ out, int64_t ld) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int g = blockIdx.y;
  if (j >= rows) return;
  float z[4];
  omega_quad(seed, stream_id, (uint64_t)j, (uint32_t)g, z);
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int k = 4 * g + t;
    if (k < cols) out[j + (int64_t)k * ld] = z[t];
  }
}

// out (cols x rows, column-major) = in^T, in rows x cols with leading dimension ld
__global__ void transpose_kernel(const float* __restrict__ in, int64_t rows, int64_t cols, int64_t ld,
                                 float* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  const int64_t c = e / rows, r = e - c * rows;      // read in column order (coalesced)
  out[c + r * cols] = in[r + c * ld];
}

// out (I x L*Rt, column-major) = the unfolding of in viewed as [L, I, Rt]:
// out[i + I (l + L r)] = in[l + L (i + I r)]
__global__ void unfold_kernel(const float* __restrict__ in, int64_t L, int64_t I, int64_t Rt,
                              float* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // index into in (coalesced reads)
  if (e >= L * I * Rt) return;
  const int64_t l = e % L, t = e / L, i = t % I, r = t / I;
  out[i + I * (l + L * r)] = in[e];
}

__global__ void axpy_kernel(float* __restrict__ y, const float* __restrict__ x, float a, int64_t n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) y[e] = fmaf(a, x[e], y[e]);
}

// Sign convention of a factor: column c of U (I x R, ld I) is flipped, together
// with column c of Ub (K x R, ld ldu), so that its entry of largest magnitude
// (the first such on ties) is positive.  One block per column.
__global__ void sign_canon_kernel(float* __restrict__ U, int64_t I, float* __restrict__ Ub, int ldu, int K) {
  const int c = blockIdx.x;
  float* u = U + (int64_t)c * I;
  __shared__ float sv[256];
  __shared__ int64_t si[256];
  float best = -1.f;
  int64_t bi = 0;
  for (int64_t i = threadIdx.x; i < I; i += blockDim.x) {
    const float a = fabsf(u[i]);
    if (a > best) {
      best = a;
      bi = i;
    }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const float a = sv[threadIdx.x + o];
      const int64_t ia = si[threadIdx.x + o];
      if (a > sv[threadIdx.x] || (a == sv[threadIdx.x] && ia < si[threadIdx.x])) {
        sv[threadIdx.x] = a;
        si[threadIdx.x] = ia;
      }
    }
    __syncthreads();
  }
  const bool flip = u[si[0]] < 0.f;
  __syncthreads();
  if (!flip) return;
  for (int64_t i = threadIdx.x; i < I; i += blockDim.x) u[i] = -u[i];
  for (int k = threadIdx.x; k < K; k += blockDim.x) Ub[k + (int64_t)c * ldu] = -Ub[k + (int64_t)c * ldu];
}

// First-order correction of the projected energy of A onto range(Q) for a
// basis Q that is orthonormal only to FP32 storage: with M = Q^T Q = I + D and
// C = B B^T, B = Q^T A (both K x K, FP64), ||Q M^-1 Q^T A||_F^2 = tr(M^-1 C)
// = tr(C) - sum_ij D_ij C_ij + O(||D||^2 tr C); out = sum_ij D_ij C_ij.  C
// need only be accurate to a few digits (the term is ~1e-6 tr C).  One block,
// fixed summation order.
__global__ void proj_energy_kernel(const double* __restrict__ M, const double* __restrict__ C, int K,
                                   double* __restrict__ out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
    const int i = e % K, j = e / K;
    const double d = M[e] - (i == j ? 1.0 : 0.0);
    acc += d * C[e];
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

__global__ void fill_identity_kernel(float* U, int64_t I, int R) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= I * R) return;
  const int64_t c = e / I, r = e - c * I;
  U[e] = (r == c) ? 1.f : 0.f;
}

}  // namespace

cudaError_t launch_omega(uint64_t seed, uint32_t stream_id, int64_t rows, int cols, float* out, int64_t ld,
                         cudaStream_t st) {
  if (rows == 0 || cols == 0) return cudaSuccess;
  dim3 grid((unsigned)((rows + 255) / 256), (unsigned)((cols + 3) / 4));
  omega_kernel<<<grid, 256, 0, st>>>(seed, stream_id, rows, cols, out, ld);
  return cudaGetLastError();
}

cudaError_t launch_transpose(const float* in, int64_t rows, int64_t cols, int64_t ld, float* out,
                             cudaStream_t st) {
  const int64_t n = rows * cols;
  if (n == 0) return cudaSuccess;
  transpose_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, rows, cols, ld, out);
  return cudaGetLastError();
}

cudaError_t launch_unfold(const float* in, int64_t L, int64_t I, int64_t Rt, float* out, cudaStream_t st) {
  const int64_t n = L * I * Rt;
  if (n == 0) return cudaSuccess;
  unfold_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, L, I, Rt, out);
  return cudaGetLastError();
}

cudaError_t launch_axpy(float* y, const float* x, float a, int64_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  axpy_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(y, x, a, n);
  return cudaGetLastError();
}

cudaError_t launch_sign_canon(float* U, int64_t I, int R, float* Ub, int ldu, int K, cudaStream_t st) {
  if (R == 0 || I == 0) return cudaSuccess;
  sign_canon_kernel<<<(unsigned)R, 256, 0, st>>>(U, I, Ub, ldu, K);
  return cudaGetLastError();
}

cudaError_t launch_proj_energy(const double* M, const double* C, int K, double* out, cudaStream_t st) {
  if (K < 1) return cudaErrorInvalidValue;
  proj_energy_kernel<<<1, 256, 0, st>>>(M, C, K, out);
  return cudaGetLastError();
}

cudaError_t launch_fill_identity(float* U, int64_t I, int R, cudaStream_t st) {
  const int64_t n = I * R;
  if (n == 0) return cudaSuccess;
  fill_identity_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(U, I, R);
  return cudaGetLastError();
}

}  // namespace rhosvd
