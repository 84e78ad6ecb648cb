// Host-side launchers of the device kernels (one translation unit each family).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rhosvd.h"

namespace rhosvd {

struct DevStatus;

// Raise a kernel's dynamic shared memory limit to `bytes`, once per device and
// kernel (the attribute is process-wide; setting it on every launch costs host time).
cudaError_t allow_dynamic_smem(const void* kernel, size_t bytes);

// Strided view of a contraction operand: entry (i, j) with j = l + L*r lives at
// base[l + i*s_i + r*s_r]; l in [0,L), r in [0,Rt), i in [0,I).
struct View {
  const float* p;
  int64_t L, I, Rt;
  int64_t s_i, s_r;
};

// Tall operand W(j, k) = base[l + r*w_r + k*w_k] with the same j = l + L*r split.
struct WView {
  const float* p;
  int64_t w_r, w_k;
};

// Output of a TTM: Out(j, k) at base[l + k*o_k + r*o_r], where j = l + L*r is
// split with L = o_L when o_L > 0 (an input read as a flat matrix whose rows
// map onto a strided output), else with the input view's L.
struct OView {
  float* p;
  int64_t o_k, o_r;
  int64_t o_L = 0;
};

// ---- sketch.cu
// Split plan of a sketch Y(i,k) = sum_j X(i,j) W(j,k).
struct SketchPlan {
  int tiles_i, tiles_k, splits;
  int64_t jchunk;
  int tu;           // outputs per thread and dimension: 16 tu x 16 tu per CTA
};
SketchPlan plan_sketch(int64_t I, int K, int64_t J);
size_t sketch_partial_floats(const SketchPlan& pl, int64_t I, int K);

// Y = X_(n) W in FP32 (partials in ws_part, deterministic fixed-order reduction).
cudaError_t launch_sketch(const View& x, const WView& w, int K, float* Y, int64_t ldy,
                          float* ws_part, cudaStream_t st);
// Same computation with the contraction split into at most max_splits parts, so
// that the partial sums fit a caller-provided scratch of max_splits * I * K floats.
cudaError_t launch_sketch_capped(const View& x, const WView& w, int K, float* Y, int64_t ldy,
                                 float* part, int max_splits, cudaStream_t st);
// Fixed-order FP32 reduction of sketch partials part[s][k][i] into Y (ld ldy).
cudaError_t launch_reduce_partials_f(const float* part, int splits, int64_t I, int K, float* Y, int64_t ldy,
                                     cudaStream_t st);

// ---- tc_sketch.cu: tcgen05 (3xTF32) sketch for mode-1 layouts
struct TcSketchPlan {
  int splits, mgroups;
  int64_t jchunk;   // j per block; blocks are dealt round-robin over the splits
};
bool tc_sketch_supported(const View& x, const WView& w, int K);
TcSketchPlan plan_tc_sketch(int64_t I, int K, int64_t J);
cudaError_t launch_tc_sketch(const View& x, const WView& w, int K, float* Y, int64_t ldy, float* part,
                             DevStatus* st, cudaStream_t stream);

// Sketch with the fastest kernel that supports the layout; part must hold
// sketch_scratch_floats(x.I, K, J) floats.
size_t sketch_scratch_floats(int64_t I, int K, int64_t J);
// The tensor-core sketch with W = the seeded Gaussian Omega of (seed, stream_id),
// generated inside the kernel; cudaErrorNotSupported when the view does not
// take the tensor-core path (the caller then materialises Omega).
bool tc_sketch_seeded_supported(const View& x, int K);
cudaError_t launch_tc_sketch_seeded(const View& x, int K, uint64_t seed, uint32_t stream_id, float* Y, int64_t ldy,
                                    float* part, DevStatus* st, cudaStream_t stream);
cudaError_t launch_sketch_auto(const View& x, const WView& w, int K, float* Y, int64_t ldy, float* part,
                               DevStatus* st, cudaStream_t stream);
// G = X_(n) W accumulated in double-float, reduced in FP64 to Gd (K x I... as I x K, ld = I).
cudaError_t launch_sketch_df(const View& x, const WView& w, int K, double* Gd, int64_t ldg,
                             double* ws_part, cudaStream_t st);

// Out(j,k) = sum_i X(i,j) M(i,k), M(i,k) = Mp[i*m_i + k*m_k].  In-place on the
// X buffer is allowed when Out addresses only rows j of X's own columns.
cudaError_t launch_ttm(const View& x, const float* Mp, int64_t m_i, int64_t m_k, int K,
                       const OView& out, const DevStatus* skip_if_orth_fail, cudaStream_t st);

// ---- tc_ttm.cu: tcgen05 (3xTF32) n-mode product for mode-1 layouts
bool tc_ttm_supported(const View& x, int64_t m_i, int64_t m_k, int K, const OView& out);
cudaError_t launch_tc_ttm(const View& x, const float* Mp, int64_t m_k, int K, const OView& out,
                          const DevStatus* skip, DevStatus* st, cudaStream_t stream);
// TTM with the fastest kernel that supports the layout (st receives device errors).
cudaError_t launch_ttm_auto(const View& x, const float* Mp, int64_t m_i, int64_t m_k, int K, const OView& out,
                            const DevStatus* skip, DevStatus* st, cudaStream_t stream);

// ---- tc_lp.cu: reduced-precision copy of X (eb = bytes per element: 2 BF16, 1 e4m3)
// X_q = format(X / s_slice) for frontal slices of slice_len elements; e4m3 also
// writes the power-of-two scales (n / slice_len floats, amax: as many uints of
// scratch); BF16 is unscaled (scale untouched).
cudaError_t launch_quantize(const float* X, int64_t n, int64_t slice_len, int eb, void* Xq, float* scale,
                            unsigned int* amax, cudaStream_t st);
// a <- nearest value of the format, in place (test matrices of a reduced-precision run)
cudaError_t launch_round_to_format(float* a, int64_t n, int eb, cudaStream_t st);
// the seeded test matrix of launch_omega with every entry rounded to the format (eb bytes)
cudaError_t launch_omega_rounded(uint64_t seed, uint32_t stream_id, int64_t rows, int cols, float* out,
                                 int64_t ld, int eb, cudaStream_t st);
// Y = X_q,(n) W with the view x in elements (x.p unused; the data is xq) and W
// a plain J x K FP32 matrix; scale_mode 0 none, 1 per column slice (slice =
// j / slice_len), 2 per row (scale[i]).  part: sketch_lp_scratch_floats floats.
bool tc_sketch_lp_supported(const View& x, int eb, int K, int scale_mode, int64_t slice_len);
size_t sketch_lp_scratch_floats(int64_t I, int K, int64_t J, int eb);
cudaError_t launch_tc_sketch_lp(const View& x, const void* xq, int eb, const float* W, int K, float* Y,
                                int64_t ldy, const float* scale, int scale_mode, int64_t slice_len, float* part,
                                DevStatus* st, cudaStream_t stream);
// Out(j, k) = s(j / slice_len) sum_i X_q(i, j) M(i, k) for the mode-1 unfolding
// (X_q I x J, i contiguous), M column-major with ldm; Out(j, k) at
// out[j * o_r + k * o_k]; scale may be NULL.
bool tc_ttm_lp_supported(int64_t I, int64_t J, int eb, int K, int64_t ldm);
cudaError_t launch_tc_ttm_lp(const void* xq, int eb, int64_t I, int64_t J, const float* M, int64_t ldm, int K,
                             float* out, int64_t o_k, int64_t o_r, const float* scale, int64_t slice_len,
                             DevStatus* st, cudaStream_t stream);

// ---- gram.cu
// G (K x K, FP64) = A^T A for A m x K (ld).  exact: double-float products
// (FP64-accurate for ill-conditioned A); otherwise FP32 within 64-row tiles and
// FP64 across them (for nearly orthonormal A).  part: ctas * K * K doubles.
struct GramPlan {
  int ctas;
  int64_t rows_per_cta;
};
GramPlan plan_gram(int64_t m, int K, bool exact);
cudaError_t launch_gram(const float* A, int64_t m, int K, int64_t ld, double* G, double* part, bool exact,
                        cudaStream_t st);

// ---- omega.cu
cudaError_t launch_omega(uint64_t seed, uint32_t stream_id, int64_t rows, int cols, float* out,
                         int64_t ld, cudaStream_t st);

// ---- orth.cu
// Cholesky factor L (K x K, FP32, column-major lower, zero above) of the FP64
// Gram G = L L^T.  pass 0 writes orth_fail; pass 1 runs only if orth_fail is
// clear; pass 2 (shifted CholeskyQR: G + 100 u tr(G) I in FP32) writes orth_fail.  Breakdown sets orth_fail and, if fail_code is non-zero, records
// fail_code as the device error.  Minv (nullable) receives R^-1 = L^-T (K x K,
// column-major, leading dimension ldm) for the GEMM form of the apply.
cudaError_t launch_chol(const double* G, int K, float* L, float* Minv, int ldm, int pass, int fail_code,
                        DevStatus* st, cudaStream_t stream);
// Row-parallel triangular solves with L: mode 0 replaces every row y^T of Y
// (m x K, ld) by y^T L^-T (= Y R^-1 with R = L^T); mode 1 by y^T (L L^T)^-1.
// Skipped when skip is non-NULL and orth_fail is set.
cudaError_t launch_trsm_rows(float* Y, int64_t m, int K, int64_t ld, const float* L, int mode,
                             const DevStatus* skip, cudaStream_t stream);
// Q = Y R^-1 in place with the explicit upper-triangular R^-1 (K x K, ld ldm),
// one thread per row (K <= RHOSVD_APPLY_RINV_MAX_K).
constexpr int RHOSVD_APPLY_RINV_MAX_K = 64;
cudaError_t launch_apply_rinv_rows(float* Y, int64_t m, int K, int64_t ld, const float* Minv, int ldm,
                                   const DevStatus* skip, cudaStream_t stream);
// Householder QR of A (m x K, ld) into its Q factor, in place; runs only when
// orth_fail is set (or always if force).
cudaError_t launch_householder(float* A, int64_t m, int K, int64_t ld, DevStatus* st, bool force,
                               cudaStream_t stream);
// Fixed-order sum of FP64 partials: out[e] = sum_s part[s*n + e], e < n.
cudaError_t launch_reduce_d(const double* part, int splits, int64_t n, double* out, cudaStream_t st);

// ---- eig.cu
// Leading R eigenvectors (descending) of the symmetric PSD K x K FP64 matrix
// G: semidefinite Cholesky G = L L^T (FP64), then one-sided Jacobi on L^T in
// FP32.  Ub is K x R (leading dimension ldu >= K); sv (nullable) receives sqrt(eigenvalues), K entries.
cudaError_t launch_small_eig(const double* G, int K, int R, float* Ub, int ldu, float* sv, DevStatus* st,
                             cudaStream_t stream);

// ---- misc
// out (cols x rows, column-major) = in^T for a small rows x cols matrix (ld).
cudaError_t launch_transpose(const float* in, int64_t rows, int64_t cols, int64_t ld, float* out,
                             cudaStream_t st);
cudaError_t launch_fill_identity(float* U, int64_t I, int R, cudaStream_t st);
// flip columns of U (I x R) and of Ub (K x R, ld ldu) so that each U column's
// largest-magnitude entry is positive
cudaError_t launch_sign_canon(float* U, int64_t I, int R, float* Ub, int ldu, int K, cudaStream_t st);
// out[0] = sum_ij (M - I)_ij C_ij: the first-order correction tr(C) - tr(M^-1 C)
// of the projected energy, for M = Q^T Q and C = (Q^T A)(Q^T A)^T (K x K, FP64)
cudaError_t launch_proj_energy(const double* M, const double* C, int K, double* out, cudaStream_t st);
// y += a x (n elements)
cudaError_t launch_axpy(float* y, const float* x, float a, int64_t n, cudaStream_t st);
// out (I x L*Rt, column-major) = mode unfolding of in viewed as [L, I, Rt]
cudaError_t launch_unfold(const float* in, int64_t L, int64_t I, int64_t Rt, float* out, cudaStream_t st);

}  // namespace rhosvd
