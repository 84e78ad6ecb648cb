// Shared device-side definitions for the randomized HOSVD kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rhosvd.h"

namespace rhosvd {

// ---------------------------------------------------------------- status word
// The first 256 bytes of every workspace hold a DevStatus.  Kernels record the
// first error they meet with atomicCAS (so the earliest error wins) and OR
// informational flags; the host reads the block back in rhosvd_device_status.
struct DevStatus {
  int32_t code;           // rhosvd_status of the first device-detected error
  int32_t flags;          // RHOSVD_FLAG_* bits
  int32_t orth_fail;      // set by a Cholesky pass that broke down, cleared per orth call
  int32_t fallbacks;      // number of Householder fallbacks that ran
  int32_t fallback_rows;  // rows m of the last matrix that needed the fallback
  int32_t eig_sweeps;     // largest number of Jacobi sweeps a truncation needed
  int32_t pad[58];
};
static_assert(sizeof(DevStatus) == 256, "status block is 256 bytes");

__device__ __forceinline__ void set_error(DevStatus* st, int32_t code) {
  if (st) atomicCAS(&st->code, 0, code);
}

// ---------------------------------------------------------------- mode views
// X of sizes (I_1..I_N), column-major, seen along mode n as a 3-way array
// [L, I, Rt] with L = prod_{k<n} I_k and Rt = prod_{k>n} I_k.  Column j of the
// unfolding X_(n) is j = l + L*r (Sec. 2 with 0-based indices), so
// X_(n)(i, j) = X[l + L*i + L*I*r].
struct ModeView {
  int64_t L, I, Rt;
  __host__ __device__ int64_t J() const { return L * Rt; }
};

// ---------------------------------------------------------------- df64 arithmetic
// Double-float accumulation from FP32 products: TwoProd by FMA (the product
// error is exact), TwoSum of Knuth; the pair (hi, lo) carries ~48 bits.
// Ogita, Rump, Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 2005.
struct df64 {
  float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// acc += a*b, error-free product, compensated sum (Dot2 step).
__device__ __forceinline__ void df64_fma(df64& acc, float a, float b) {
  float p = a * b;
  float pe = fmaf(a, b, -p);
  float s, se;
  two_sum(acc.hi, p, s, se);
  acc.hi = s;
  acc.lo += se + pe;
}

__device__ __forceinline__ double df64_to_double(df64 v) { return (double)v.hi + (double)v.lo; }

// Double-word ("double-float") arithmetic on FP32 pairs, hi + lo with
// |lo| <= ulp(hi)/2: the FMA-based algorithms of Joldes, Muller, Popescu,
// "Tight and rigorous error bounds for basic building blocks of double-word
// arithmetic", ACM TOMS 2017 (relative errors ~2^-44..2^-46).  Used where a
// short sequential chain needs more than FP32 precision and GB300's narrow
// FP64 pipe would dominate the latency.
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {   // |a| >= |b|
  s = a + b;
  e = b - (s - a);
}
// 2^k as a float for -126 <= k <= 127 (0 below, +inf above).
__device__ __forceinline__ float pow2f(int k) {
  return (k < -126) ? 0.f : (k > 127 ? __int_as_float(0x7f800000) : __int_as_float((k + 127) << 23));
}
// Double-word pair of a finite double times 2^-e, with integer and FP32
// instructions only (GB300's FP64 pipe is narrow): the significand's top 24
// bits give the high part exactly, the low 29 bits, rounded, the low part, and
// one FastTwoSum renormalises (48 significant bits in all).  Values whose
// scaled magnitude is below 2^-126 become 0.
__device__ __forceinline__ df64 dw_from_double_scaled(double v, int e) {
  const long long b = __double_as_longlong(v);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex == 0) return df64{0.f, 0.f};
  const long long m = (b & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;   // 53-bit significand
  const int E = ex - 1075 - e;                                        // v 2^-e = m 2^E
  const float h = (float)(int)(m >> 29) * pow2f(E + 29);
  const float l = (float)(int)(m & 0x1FFFFFFF) * pow2f(E);
  float hi, lo;
  fast_two_sum(h, l, hi, lo);
  return (b < 0) ? df64{-hi, -lo} : df64{hi, lo};
}
// A double's value truncated to float (no rounding; 0 below the normal float
// range), by bit manipulation: for estimates that must not use the FP64 pipe.
__device__ __forceinline__ float f32_trunc(double v) {
  const long long b = __double_as_longlong(v);
  const int ex = (int)((b >> 52) & 0x7ff) - 1023 + 127;
  const int sign = (int)((b >> 32) & 0x80000000LL);
  if (ex <= 0) return __int_as_float(sign);
  if (ex >= 255) return __int_as_float(sign | 0x7f800000);
  return __int_as_float(sign | (ex << 23) | (int)((b >> 29) & 0x7fffff));
}
__device__ __forceinline__ bool finite_bits(double v) {
  return ((__double_as_longlong(v) >> 52) & 0x7ff) != 0x7ff;
}
__device__ __forceinline__ df64 dw_from_double(double v) {
  const float hi = __double2float_rn(v);
  return df64{hi, __double2float_rn(v - (double)hi)};
}
// DW + DW, the accurate algorithm (two TwoSums and two renormalisations)
__device__ __forceinline__ df64 dw_add(df64 x, df64 y) {
  float s, t, e, f;
  two_sum(x.hi, y.hi, s, t);
  two_sum(x.lo, y.lo, e, f);
  t += e;
  fast_two_sum(s, t, s, t);
  t += f;
  fast_two_sum(s, t, s, t);
  return df64{s, t};
}
__device__ __forceinline__ df64 dw_neg(df64 x) { return df64{-x.hi, -x.lo}; }
// DW + DW, the cheaper ("sloppy") algorithm: one TwoSum on the high parts and
// one renormalisation; its error is bounded relative to |x| + |y| rather than
// |x + y| (Joldes, Muller, Popescu 2017), which is what a backward-stable
// elimination such as Cholesky needs (|dA| <= c u |L||L^T| with u ~ 2^-44).
__device__ __forceinline__ df64 dw_add_sloppy(df64 x, df64 y) {
  float s, t;
  two_sum(x.hi, y.hi, s, t);
  t += x.lo + y.lo;
  fast_two_sum(s, t, s, t);
  return df64{s, t};
}
// DW x DW with FMA
__device__ __forceinline__ df64 dw_mul(df64 x, df64 y) {
  const float ch = x.hi * y.hi;
  float cl = fmaf(x.hi, y.hi, -ch);
  const float tl = fmaf(x.lo, y.hi, x.hi * y.lo);
  cl += tl;
  float s, e;
  fast_two_sum(ch, cl, s, e);
  return df64{s, e};
}
// 1/sqrt(d) for a positive double-word d: the FP32 estimate plus one Newton
// correction r = r0 + r0 (1 - d r0^2) / 2 evaluated in double-word arithmetic.
__device__ __forceinline__ df64 dw_rsqrt(df64 d) {
  const float r0 = rsqrtf(d.hi);
  const df64 r = df64{r0, 0.f};
  const df64 q = dw_mul(dw_mul(d, r), r);
  const df64 e = dw_add(df64{1.f, 0.f}, dw_neg(q));
  float s, t;
  fast_two_sum(r0, 0.5f * r0 * e.hi, s, t);
  return df64{s, t};
}

// 1/sqrt(d) in FP64: the FP32 hardware estimate refined by two Newton steps
// y <- y (3 - d y^2) / 2 (each step doubles the correct bits: ~2^-22 -> 2^-44
// -> full precision).  Callers pass pivots of Gram matrices scaled to max
// diagonal 1, well inside the FP32 exponent range.
__device__ __forceinline__ double rsqrt_newton(double d) {
  double y = (double)rsqrtf((float)d);
  y = y * (1.5 - 0.5 * d * y * y);
  y = y * (1.5 - 0.5 * d * y * y);
  return y;
}
__device__ __forceinline__ float rsqrt_newton(float d) { return rsqrtf(d); }

// ---------------------------------------------------------------- warp helpers
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
// SC 2011.  Round: (c0,c1,c2,c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2),
// hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); the key advances by (W0, W1) between rounds.
struct U4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint32_t lo0 = M0 * c.x, hi0 = __umulhi(M0, c.x);
    uint32_t lo1 = M1 * c.z, hi1 = __umulhi(M1, c.z);
    U4 n;
    n.x = hi1 ^ c.y ^ k0;
    n.y = lo1;
    n.z = hi0 ^ c.w ^ k1;
    n.w = lo0;
    c = n;
  }
  return c;
}

// Box-Muller (1958) on 24-bit uniforms: u1 = (a+1) 2^-24 in (0,1], u2 = b 2^-24.
__device__ __forceinline__ void box_muller24(uint32_t wa, uint32_t wb, float& z0, float& z1) {
  float u1 = (float)((wa >> 8) + 1u) * 5.9604644775390625e-8f;   // exact
  float u2 = (float)(wb >> 8) * 5.9604644775390625e-8f;           // exact
  float r = sqrtf(-2.0f * logf(u1));
  float s, c;
  sincospif(2.0f * u2, &s, &c);
  z0 = r * c;
  z1 = r * s;
}

// Omega(j, k) of (seed, stream): four normals per counter (j, k/4).
__device__ __forceinline__ void omega_quad(uint64_t seed, uint32_t stream, uint64_t j, uint32_t kq,
                                           float out[4]) {
  U4 c{(uint32_t)j, (uint32_t)(j >> 32), kq, stream};
  U4 w = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  box_muller24(w.x, w.y, out[0], out[1]);
  box_muller24(w.z, w.w, out[2], out[3]);
}

}  // namespace rhosvd
