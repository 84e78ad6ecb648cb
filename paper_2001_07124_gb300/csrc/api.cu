// C ABI of the randomized HOSVD library: argument validation, workspace
// planning and the algorithm drivers (RP-HOSVD = Alg. 6 with Alg. 1 per mode,
// R-STHOSVD = Alg. 8, R-PET = Alg. 9).  Every driver is written once and run
// either "dry" (only carving the workspace, to size it) or for real, so the
// size query and the execution can never disagree.  All device work goes to
// the caller's stream; nothing here synchronises except rhosvd_device_status
// and rhosvd_orth with a non-NULL fallback_used.
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace rhosvd {
namespace {

constexpr size_t ALIGN = 256;

struct Ctx {
  bool dry = true;
  char* base = nullptr;
  size_t off = 0, high = 0;
  cudaStream_t s = nullptr;
  DevStatus* st = nullptr;
  cudaError_t err = cudaSuccess;
  int64_t launches = 0;   // kernels enqueued (counted in dry runs too)

  template <class T>
  T* take(size_t n) {
    off = (off + ALIGN - 1) / ALIGN * ALIGN;
    T* p = dry ? nullptr : reinterpret_cast<T*>(base + off);
    off += std::max<size_t>(n, 1) * sizeof(T);
    high = std::max(high, off);
    return p;
  }
  void check(cudaError_t e) {
    if (e != cudaSuccess && err == cudaSuccess) err = e;
  }
};

struct Scope {   // stack discipline for temporaries
  Ctx& c;
  size_t saved;
  explicit Scope(Ctx& c_) : c(c_), saved(c_.off) {}
  ~Scope() { c.off = saved; }
};

struct Geom {
  int N = 0;
  int64_t d[RHOSVD_MAX_MODES] = {0};
  int64_t L(int n) const { int64_t v = 1; for (int k = 0; k < n; ++k) v *= d[k]; return v; }
  int64_t Rt(int n) const { int64_t v = 1; for (int k = n + 1; k < N; ++k) v *= d[k]; return v; }
  int64_t J(int n) const { return L(n) * Rt(n); }
  int64_t numel() const { int64_t v = 1; for (int k = 0; k < N; ++k) v *= d[k]; return v; }
};

View mode_view(const float* p, const Geom& g, int n) {
  View v;
  v.p = p;
  v.L = g.L(n);
  v.I = g.d[n];
  v.Rt = g.Rt(n);
  v.s_i = v.L;
  v.s_r = v.L * v.I;
  return v;
}
// A tall column-major matrix (m x K, ld) seen as the mode-2 unfolding of an
// (m, K) tensor: X(i = column, j = row).
View matrix_view(const float* p, int64_t m, int K, int64_t ld) {
  View v;
  v.p = p;
  v.L = m;
  v.I = K;
  v.Rt = 1;
  v.s_i = ld;
  v.s_r = 0;
  return v;
}

// ------------------------------------------------------------------ primitive ops

// Y (I x K, ld) = X_(n) W with W(j,k) = w.p[l + r*w_r + k*w_k]
void op_sketch(Ctx& c, const View& x, const WView& w, int K, float* Y, int64_t ldy) {
  Scope sc(c);
  float* part = c.take<float>(sketch_scratch_floats(x.I, K, x.L * x.Rt));
  c.launches += 2;
  if (!c.dry) c.check(launch_sketch_auto(x, w, K, Y, ldy, part, c.st, c.s));
}

// Gd (I x I, FP64) = X_(n) W accumulated in double-float
void op_gram_df(Ctx& c, const View& x, const WView& w, int K, double* Gd) {
  Scope sc(c);
  SketchPlan pl = plan_sketch(x.I, K, x.L * x.Rt);
  double* part = c.take<double>(sketch_partial_floats(pl, x.I, K));
  c.launches += 2;
  if (!c.dry) c.check(launch_sketch_df(x, w, K, Gd, x.I, part, c.s));
}

// Gd (K x K, FP64) = A^T A for a tall matrix; exact = FP64-accurate products
void op_gram_matrix(Ctx& c, const float* A, int64_t m, int K, int64_t ld, double* Gd, bool exact = true) {
  Scope sc(c);
  GramPlan pl = plan_gram(m, K, exact);
  double* part = c.take<double>((size_t)pl.ctas * K * K);
  c.launches += 2;
  if (!c.dry) c.check(launch_gram(A, m, K, ld, Gd, part, exact, c.s));
}

void op_ttm(Ctx& c, const View& x, const float* M, int64_t m_i, int64_t m_k, int K, const OView& out,
            const DevStatus* skip = nullptr) {
  if (x.L * x.Rt > 0 && K > 0) c.launches += 1;
  if (!c.dry) c.check(launch_ttm_auto(x, M, m_i, m_k, K, out, skip, c.st, c.s));
}

// CholeskyQR with device-side Householder fallback, in place on Y (m x K, ld).
// passes = 2 is CholeskyQR2 (Q orthonormal to FP32 accuracy); passes = 1 is
// used for the intermediate bases of the power iteration (Alg. 1),
// where only range(Q) matters: a second pass would re-orthonormalise Q1 within
// range(Q1) without changing it, and Q1 from the FP64-accurate first pass is
// well conditioned whenever that pass succeeds.  On tall matrices
// (m >= 32768) the apply Y R^-1 multiplies by the explicit R^-1: row by row on
// the CUDA cores up to K = 64 (independent dot products, memory-bound), as a
// tensor-core GEMM beyond; shorter matrices take the row-wise triangular solve,
// which needs no inverse from the factorisation.
void op_orth(Ctx& c, float* Y, int64_t m, int K, int64_t ld, int passes = 2) {
  Scope sc(c);
  double* G = c.take<double>((size_t)K * K);
  float* L = c.take<float>((size_t)K * K);
  const int ldm = (K + 3) & ~3;
  float* Minv = c.take<float>((size_t)ldm * K);
  const View yv = matrix_view(Y, m, K, ld);
  // forming R^-1 pays only on tall matrices
  const bool rows = c.st != nullptr && m >= 32768 && K <= RHOSVD_APPLY_RINV_MAX_K;
  const bool gemm = !rows && c.st != nullptr && m >= 32768 && tc_ttm_supported(yv, 1, ldm, K, OView{Y, ld, 0});
  for (int pass = 0; pass < passes; ++pass) {
    op_gram_matrix(c, Y, m, K, ld, G, pass == 0);
    c.launches += 2;
    if (!c.dry) c.check(launch_chol(G, K, L, (rows || gemm) ? Minv : nullptr, ldm, pass, 0, c.st, c.s));
    if (rows) {
      if (!c.dry) c.check(launch_apply_rinv_rows(Y, m, K, ld, Minv, ldm, c.st, c.s));
    } else if (gemm) {
      if (!c.dry) c.check(launch_tc_ttm(yv, Minv, ldm, K, OView{Y, ld, 0}, c.st, c.st, c.s));
    } else {
      if (!c.dry) c.check(launch_trsm_rows(Y, m, K, ld, L, 0, c.st, c.s));
    }
  }
  c.launches += 1;
  if (!c.dry) c.check(launch_householder(Y, m, K, ld, c.st, false, c.s));
}

// Leading dimension of the small K x R factor Ub: a multiple of 4 so that the
// tensor-core TTMs can stream it with TMA.
inline int ldu_of(int K) { return (K + 3) & ~3; }

// Leading R eigenvectors (K x R) of the Gram of a tall matrix Bt (m x K, ld)
void op_truncate(Ctx& c, const float* Bt, int64_t m, int K, int64_t ld, int R, float* Ub) {
  Scope sc(c);
  double* G = c.take<double>((size_t)K * K);
  op_gram_matrix(c, Bt, m, K, ld, G);
  c.launches += 1;
  if (!c.dry) c.check(launch_small_eig(G, K, R, Ub, ldu_of(K), nullptr, c.st, c.s));
}

void op_omega(Ctx& c, uint64_t seed, uint32_t stream_id, int64_t rows, int cols, float* out) {
  c.launches += 1;
  if (!c.dry) c.check(launch_omega(seed, stream_id, rows, cols, out, rows, c.s));
}

// Y = X_(n) Omega with Omega the seeded Gaussian test matrix of (seed, stream_id)
// (J x K, Alg. 1).  Where the tensor-core sketch can generate it (modes
// with I > 128), Omega is computed inside the sketch kernel and never stored;
// otherwise it is drawn into Om (J x K, caller's buffer) and sketched from memory.
void op_sketch_seeded(Ctx& c, const View& x, int K, uint64_t seed, uint32_t stream_id, float* Y, int64_t ldy,
                      float* Om) {
  const int64_t J = x.L * x.Rt;
  if (tc_sketch_seeded_supported(x, K)) {          // same decision in dry runs (launch counting)
    Scope sc(c);
    float* part = c.take<float>(sketch_scratch_floats(x.I, K, J));
    c.launches += 2;
    if (!c.dry) c.check(launch_tc_sketch_seeded(x, K, seed, stream_id, Y, ldy, part, c.st, c.s));
    return;
  }
  op_omega(c, seed, stream_id, J, K, Om);
  op_sketch(c, x, WView{Om, x.L, J}, K, Y, ldy);
}

// ------------------------------------------------------------------ reduced-precision copy of X

// X_q (BF16 or e4m3) with one scale per frontal slice of the last mode (e4m3).
struct LpCopy {
  int eb = 0;                   // bytes per element: 2 BF16, 1 e4m3; 0 = no copy
  const void* xq = nullptr;
  const float* scale = nullptr; // e4m3 only
  int64_t slice_len = 0;        // elements of one frontal slice
  int64_t nslices = 0;          // I_N
};

int eb_of(int dtype) { return dtype == RHOSVD_BF16 ? 2 : dtype == RHOSVD_E4M3 ? 1 : 0; }

// Quantise X into a copy carved from the workspace (left taken until the end of the call).
LpCopy lp_make(Ctx& c, const float* X, const Geom& g, int dtype) {
  LpCopy lp;
  lp.eb = eb_of(dtype);
  if (lp.eb == 0 || g.N < 2) {
    lp.eb = 0;
    return lp;
  }
  const int64_t n = g.numel();
  lp.nslices = g.d[g.N - 1];
  lp.slice_len = n / lp.nslices;
  unsigned char* xq = c.take<unsigned char>((size_t)n * lp.eb);
  float* sc = lp.eb == 1 ? c.take<float>((size_t)lp.nslices) : nullptr;
  unsigned int* amax = lp.eb == 1 ? c.take<unsigned int>((size_t)lp.nslices) : nullptr;
  lp.xq = xq;
  lp.scale = sc;
  c.launches += lp.eb == 1 ? 3 : 1;
  if (!c.dry) c.check(launch_quantize(X, n, lp.slice_len, lp.eb, xq, sc, amax, c.s));
  return lp;
}

// Elements of the mode-n unfolding's columns per frontal slice of the last mode.
int64_t lp_col_slice(const LpCopy& lp, const Geom& g, int n) { return g.J(n) / lp.nslices; }

// Y = X_q,(n) W on the tensor cores if the layout allows; false leaves the pass to FP32.
bool lp_sketch(Ctx& c, const LpCopy& lp, const Geom& g, int n, const float* W, int K, float* Y) {
  if (lp.eb == 0) return false;
  const View xv = mode_view(nullptr, g, n);
  const bool last = n == g.N - 1;
  const int mode = lp.scale == nullptr ? 0 : (last ? 2 : 1);
  const int64_t sl = last ? 0 : lp_col_slice(lp, g, n);
  if (!tc_sketch_lp_supported(xv, lp.eb, K, mode, sl)) return false;
  Scope sc(c);
  float* part = c.take<float>(sketch_lp_scratch_floats(xv.I, K, g.J(n), lp.eb));
  c.launches += 2;
  if (!c.dry)
    c.check(launch_tc_sketch_lp(xv, lp.xq, lp.eb, W, K, Y, g.d[n], lp.scale, mode, sl, part, c.st, c.s));
  return true;
}

// Out(j, k) = (X_q,(1)^T M)(j, k) on the tensor cores; false leaves it to FP32.
bool lp_ttm1(Ctx& c, const LpCopy& lp, const Geom& g, const float* M, int64_t ldm, int K, float* out,
             int64_t o_k, int64_t o_r) {
  if (lp.eb == 0 || !tc_ttm_lp_supported(g.d[0], g.J(0), lp.eb, K, ldm)) return false;
  c.launches += 1;
  if (!c.dry)
    c.check(launch_tc_ttm_lp(lp.xq, lp.eb, g.d[0], g.J(0), M, ldm, K, out, o_k, o_r, lp.scale,
                             lp_col_slice(lp, g, 0), c.st, c.s));
  return true;
}

// The seeded test matrix of (seed, stream_id), rounded to the copy's format as it is drawn.
void lp_omega(Ctx& c, const LpCopy& lp, uint64_t seed, uint32_t stream_id, int64_t rows, int cols, float* out) {
  c.launches += 1;
  if (!c.dry) c.check(launch_omega_rounded(seed, stream_id, rows, cols, out, rows, lp.eb, c.s));
}

// ------------------------------------------------------------------ Alg. 1 on one mode

struct ModeResult {
  float* Q;     // I x K orthonormal (ld I)
  float* Bt;    // J x K: Bt(j, k) = (Q^T X_(n))(k, j)   (Z layout, ld J)
  float* Ub;    // K x R leading eigenvectors of B B^T (ld ldu_of(K))
};

// Steps 1-5 of Alg. 1 on the mode-n unfolding of the tensor at x (geometry g):
// sketch, orth, q power iterations, projection B, truncation of B B^T.
// Buffers Yb (I x K), Zb (J x K), Om (J x K, unless explicit) and Ub (K x R, ld ldu_of(K))
// belong to the caller.
// The test matrix is seeded on stream_id stream_base + n.  With lp (mode 1 of
// the original X only) the power-iteration products read the reduced-precision
// copy where its kernels take the layout.
void alg1_mode(Ctx& c, const float* x, const Geom& g, int n, int K, int R, int q, uint64_t seed,
               const float* omega_explicit, float* Yb, float* Zb, float* Om, float* Ub, uint32_t stream_base = 0,
               const LpCopy* lp = nullptr) {
  const View xv = mode_view(x, g, n);
  const int64_t I = g.d[n], L = g.L(n), J = g.J(n);
  if (omega_explicit != nullptr)
    op_sketch(c, xv, WView{omega_explicit, L, J}, K, Yb, I);   // Y = X_(n) Omega
  else
    op_sketch_seeded(c, xv, K, seed, stream_base + (uint32_t)n, Yb, I, Om);
  op_orth(c, Yb, I, K, I, q > 0 ? 1 : 2);               // Q = orth(Y)
  const OView zo{Zb, J, L};                              // Z(j,k) at j + k*J
  const bool use_lp = lp != nullptr && lp->eb != 0 && n == 0;
  for (int it = 0; it < q; ++it) {
    if (!(use_lp && lp_ttm1(c, *lp, g, Yb, I, K, Zb, J, 1)))
      op_ttm(c, xv, Yb, 1, I, K, zo);                    // Z = X_(n)^T Q
    op_orth(c, Zb, J, K, J, 1);                          // Z = orth(X_(n)^T Q)
    if (!(use_lp && lp_sketch(c, *lp, g, n, Zb, K, Yb)))
      op_sketch(c, xv, WView{Zb, L, J}, K, Yb, I);       // Y = X_(n) Z
    op_orth(c, Yb, I, K, I, it + 1 < q ? 1 : 2);         // Q = orth(Y)
  }
  op_ttm(c, xv, Yb, 1, I, K, zo);                        // B^T = X_(n)^T Q
  op_truncate(c, Zb, J, K, J, R, Ub);                    // Ubar_R of B
}

// U (I x R) = Q Ub
void lift_factor(Ctx& c, const float* Q, int64_t I, int K, const float* Ub, int R, float* U) {
  op_ttm(c, matrix_view(Q, I, K, I), Ub, 1, ldu_of(K), R, OView{U, I, 0});
}

// S_new[l, a, r] = sum_k Ub(k, a) Bt(l + L r, k): the shortcut S_(n) = Ubar_R^T B.
// Bt is read as a flat J x K matrix (a tall GEMM); the output rows j = l + L r
// are scattered into the mode-n layout of S_new.
void refold_core(Ctx& c, const float* Bt, const Geom& g, int n, int K, const float* Ub, int R, float* Snew) {
  const int64_t L = g.L(n), J = g.J(n);
  op_ttm(c, matrix_view(Bt, J, K, J), Ub, 1, ldu_of(K), R, OView{Snew, L, L * R, L});
}

// T = X x_n M^T with M (I_n x K, m_i/m_k strides): output dims d[n] -> K
void ttm_mode(Ctx& c, const float* x, const Geom& g, int n, const float* M, int64_t m_i, int64_t m_k, int K,
              float* out) {
  const int64_t L = g.L(n);
  op_ttm(c, mode_view(x, g, n), M, m_i, m_k, K, OView{out, L, L * K});
}

// ------------------------------------------------------------------ widths

struct Plan {
  int K[RHOSVD_MAX_MODES];
  int S[RHOSVD_MAX_MODES];
  int64_t J[RHOSVD_MAX_MODES];
  int kron = 0;             // R-PET with Kronecker-structured factor sketches: width k of each Phi_p
  int dtype = RHOSVD_F32;   // arithmetic of the sketch passes
  int refine = 0;           // RP-HOOI sweeps after the decomposition
  int p = 0;                // oversampling (also of the refinement's sketches)
};

rhosvd_status validate_shape(const rhosvd_shape* sh, Geom& g) {
  if (sh == nullptr || sh->N < 1 || sh->N > RHOSVD_MAX_MODES) return RHOSVD_EINVAL;
  g.N = sh->N;
  int64_t tot = 1;
  for (int n = 0; n < g.N; ++n) {
    if (sh->dims[n] < 1 || sh->dims[n] > (int64_t(1) << 40)) return RHOSVD_EINVAL;
    g.d[n] = sh->dims[n];
    if (tot > (int64_t(1) << 62) / g.d[n]) return RHOSVD_EINVAL;
    tot *= g.d[n];
  }
  return RHOSVD_OK;
}

rhosvd_status make_plan(const Geom& g, const int32_t* ranks, const rhosvd_opts* o, Plan& pl) {
  if (ranks == nullptr || o == nullptr) return RHOSVD_EINVAL;
  if (o->algo < RHOSVD_ALGO_RHOSVD || o->algo > RHOSVD_ALGO_RPET) return RHOSVD_EINVAL;
  if (o->p < 0 || o->q < 0 || o->q > 64) return RHOSVD_EINVAL;
  if (o->dtype < RHOSVD_F32 || o->dtype > RHOSVD_E4M3 || o->refine_iters < 0 || o->refine_iters > 8)
    return RHOSVD_EINVAL;
  pl.dtype = o->dtype;
  pl.refine = o->refine_iters;
  pl.p = o->p;
  int64_t cur[RHOSVD_MAX_MODES];
  for (int n = 0; n < g.N; ++n) cur[n] = g.d[n];
  for (int n = 0; n < g.N; ++n) {
    int64_t J = 1;
    for (int k = 0; k < g.N; ++k)
      if (k != n) J *= cur[k];
    const int64_t R = ranks[n];
    if (R < 1 || R > g.d[n] || R > J) return RHOSVD_EINVAL;
    int64_t K;
    if (o->algo == RHOSVD_ALGO_RPET && o->K[n] > 0) K = o->K[n];
    else K = std::min<int64_t>(R + o->p, std::min<int64_t>(g.d[n], J));
    if (K < R || K > g.d[n] || K > J || K > RHOSVD_MAX_K) return RHOSVD_EINVAL;
    pl.K[n] = (int)K;
    pl.J[n] = J;
    pl.S[n] = 0;
    if (o->algo == RHOSVD_ALGO_RPET) {
      int64_t S = o->S[n] > 0 ? o->S[n] : 2 * K + 1;
      if (S < K || S > (int64_t(1) << 20)) return RHOSVD_EINVAL;
      pl.S[n] = (int)S;
    }
    if (o->algo == RHOSVD_ALGO_RSTHOSVD) cur[n] = R;
  }
  if (o->flags & ~RHOSVD_OPT_KRONECKER) return RHOSVD_EINVAL;
  if (o->flags & RHOSVD_OPT_KRONECKER) {
    // every factor sketch has k^(N-1) columns, k the smallest width that reaches
    // the largest requested K_n; S_n defaults to 2 K_n + 1 of that width
    if (o->algo != RHOSVD_ALGO_RPET || g.N < 2) return RHOSVD_EINVAL;
    int kmax = 1;
    for (int n = 0; n < g.N; ++n) kmax = std::max(kmax, pl.K[n]);
    int64_t k = 1, kp = 1;
    for (;;) {
      kp = 1;
      for (int e = 0; e < g.N - 1; ++e) kp *= k;
      if (kp >= kmax) break;
      ++k;
    }
    for (int n = 0; n < g.N; ++n) {
      if (kp > g.d[n] || kp > pl.J[n] || kp > RHOSVD_MAX_K || k > g.d[n]) return RHOSVD_EINVAL;
      pl.K[n] = (int)kp;
      const int64_t S = o->S[n] > 0 ? o->S[n] : 2 * kp + 1;
      if (S < kp || S > (int64_t(1) << 20)) return RHOSVD_EINVAL;
      pl.S[n] = (int)S;
    }
    pl.kron = (int)k;
  }
  return RHOSVD_OK;
}

// ------------------------------------------------------------------ drivers

void run_rsthosvd(Ctx& c, const float* X, const Geom& g0, const int32_t* ranks, const Plan& pl, int q,
                  uint64_t seed, const float* const* Omega, float* const* U, float* G) {
  size_t max_jk = 1, max_ik = 1, max_s = 1, max_kk = 1;
  {
    Geom g = g0;
    for (int n = 0; n < g.N; ++n) {
      max_jk = std::max<size_t>(max_jk, (size_t)g.J(n) * pl.K[n]);
      max_ik = std::max<size_t>(max_ik, (size_t)g.d[n] * pl.K[n]);
      max_kk = std::max<size_t>(max_kk, (size_t)ldu_of(pl.K[n]) * ranks[n]);
      g.d[n] = ranks[n];
      max_s = std::max<size_t>(max_s, (size_t)g.numel());
    }
  }
  float* Yb = c.take<float>(max_ik);
  float* Zb = c.take<float>(max_jk);
  float* Ub = c.take<float>(max_kk);
  bool need_om = false;
  for (int n = 0; n < g0.N; ++n) need_om |= (Omega == nullptr || Omega[n] == nullptr);
  float* Om = need_om ? c.take<float>(max_jk) : nullptr;
  float* Sb[2] = {c.take<float>(max_s), c.take<float>(max_s)};
  // the reduced-precision copy serves the power products of mode 1 (the original X)
  const LpCopy lp = (q > 0 && pl.dtype != RHOSVD_F32) ? lp_make(c, X, g0, pl.dtype) : LpCopy{};
  Geom g = g0;
  const float* cur = X;
  int ping = 0;
  for (int n = 0; n < g.N; ++n) {
    const int K = pl.K[n], R = ranks[n];
    const int64_t I = g.d[n];
    const bool last = (n == g.N - 1);
    if (R == I) {   // nothing to reduce in this mode (the small-mode remark of Sec. 4)
      c.launches += 1;
      if (!c.dry) c.check(launch_fill_identity(U[n], I, R, c.s));
      if (last && !c.dry) c.check(cudaMemcpyAsync(G, cur, sizeof(float) * g.numel(), cudaMemcpyDeviceToDevice, c.s));
      continue;
    }
    const float* om = (Omega != nullptr) ? Omega[n] : nullptr;
    alg1_mode(c, cur, g, n, K, R, q, seed, om, Yb, Zb, Om, Ub, 0, n == 0 ? &lp : nullptr);
    lift_factor(c, Yb, I, K, Ub, R, U[n]);
    float* dst = last ? G : Sb[ping];
    refold_core(c, Zb, g, n, K, Ub, R, dst);
    g.d[n] = R;
    cur = dst;
    ping ^= 1;
  }
}

void run_rhosvd(Ctx& c, const float* X, const Geom& g, const int32_t* ranks, const Plan& pl, int q,
                uint64_t seed, const float* const* Omega, float* const* U, float* G) {
  size_t max_jk = 1, max_ik = 1, max_kk = 1;
  for (int n = 0; n < g.N; ++n) {
    max_jk = std::max<size_t>(max_jk, (size_t)g.J(n) * pl.K[n]);
    max_ik = std::max<size_t>(max_ik, (size_t)g.d[n] * pl.K[n]);
    max_kk = std::max<size_t>(max_kk, (size_t)ldu_of(pl.K[n]) * ranks[n]);
  }
  // core chain sizes: T_n = X x_1 U_1^T ... x_n U_n^T
  size_t max_t = 1;
  {
    Geom t = g;
    for (int n = 0; n < g.N; ++n) {
      t.d[n] = ranks[n];
      max_t = std::max<size_t>(max_t, (size_t)t.numel());
    }
  }
  float* Yb = c.take<float>(max_ik);
  float* Zb = c.take<float>(max_jk);
  float* Ub = c.take<float>(max_kk);
  bool need_om = false;
  for (int n = 0; n < g.N; ++n) need_om |= (Omega == nullptr || Omega[n] == nullptr);
  float* Om = need_om ? c.take<float>(max_jk) : nullptr;
  float* Tb[2] = {c.take<float>(max_t), c.take<float>(max_t)};
  const LpCopy lp = (q > 0 && pl.dtype != RHOSVD_F32) ? lp_make(c, X, g, pl.dtype) : LpCopy{};
  // factors of modes N-1..1 first, mode 0 last so its projection B_1 (still in
  // Zb) gives the first core step X x_1 U_1^T = Ubar^T B_1 without a pass over X
  const float* chain = X;
  Geom t = g;
  int ping = 0;
  for (int n = g.N - 1; n >= 0; --n) {
    const int K = pl.K[n], R = ranks[n];
    const int64_t I = g.d[n];
    if (R == I) {
      c.launches += 1;
      if (!c.dry) c.check(launch_fill_identity(U[n], I, R, c.s));
      continue;
    }
    const float* om = (Omega != nullptr) ? Omega[n] : nullptr;
    alg1_mode(c, X, g, n, K, R, q, seed, om, Yb, Zb, Om, Ub, 0, n == 0 ? &lp : nullptr);
    lift_factor(c, Yb, I, K, Ub, R, U[n]);
    if (n == 0) {
      float* dst = (g.N == 1) ? G : Tb[ping];
      refold_core(c, Zb, g, 0, K, Ub, R, dst);
      t.d[0] = R;
      chain = dst;
      ping ^= 1;
    }
  }
  // remaining core steps S = T x_n U_n^T (Eq. "Core")
  int last_reduced = -1;
  for (int n = 1; n < g.N; ++n)
    if (ranks[n] != g.d[n]) last_reduced = n;
  for (int n = 1; n < g.N; ++n) {
    const int R = ranks[n];
    if (R == g.d[n]) continue;
    float* dst = (n == last_reduced) ? G : Tb[ping];
    ttm_mode(c, chain, t, n, U[n], 1, g.d[n], R, dst);
    t.d[n] = R;
    chain = dst;
    ping ^= 1;
  }
  if (chain != G && !c.dry)
    c.check(cudaMemcpyAsync(G, chain, sizeof(float) * t.numel(), cudaMemcpyDeviceToDevice, c.s));
}

// Core sketch chain H = X x_1 Omega~_1 ... x_N Omega~_N (the core sketch of Alg. 9).
void core_sketch_chain(Ctx& c, const float* X, const Geom& g, const int* S, uint64_t seed,
                       const float* const* Om_t, float* const* om_t_buf, float* H, const LpCopy* lp = nullptr) {
  size_t max_t = 1, max_m = 1;
  {
    Geom t = g;
    for (int n = 0; n < g.N; ++n) {
      t.d[n] = S[n];
      max_t = std::max<size_t>(max_t, (size_t)t.numel());
      max_m = std::max<size_t>(max_m, (size_t)g.d[n] * S[n]);
    }
  }
  Scope sc(c);
  float* Tb[2] = {c.take<float>(max_t), c.take<float>(max_t)};
  float* Mt = c.take<float>(max_m);                   // Omega~_n^T, I_n x S_n column-major
  Geom t = g;
  const float* cur = X;
  int ping = 0;
  (void)seed;
  for (int n = 0; n < g.N; ++n) {
    const float* om = (Om_t != nullptr && Om_t[n] != nullptr) ? Om_t[n] : om_t_buf[n];
    float* dst = (n == g.N - 1) ? H : Tb[ping];
    // the TTM takes M(i, s) = Omega~(s, i) column-major (I_n x S_n), the layout the
    // tensor-core kernel streams with TMA
    c.launches += 1;
    if (!c.dry) c.check(launch_transpose(om, S[n], g.d[n], S[n], Mt, c.s));
    // the first product reads X: from the reduced-precision copy when there is one
    const bool done = n == 0 && lp != nullptr && lp_ttm1(c, *lp, g, Mt, g.d[0], S[0], dst, 1, S[0]);
    if (!done) ttm_mode(c, cur, t, n, Mt, 1, g.d[n], S[n], dst);
    t.d[n] = S[n];
    cur = dst;
    ping ^= 1;
  }
}

// R-PET's sketches with Kronecker-structured factor test matrices (the
// memory-efficient form of Sec. 5.1): Y_n = (X x_{p != n} Phi_p^T)_(n) =
// X_(n) (Phi_N x ... x Phi_1, without Phi_n), Phi_p Gaussian I_p x k, and the
// core sketch H = X x_1 Omega~_1 ... x_N Omega~_N, from two reads of X, both
// in layouts the TMA streams at full rate:
//   * C = X x_1 [Omega~_1^T Phi_1], written column-major in (j, s): its first
//     S_1 columns are the tensor X x_1 Omega~_1 with mode 1 moved last
//     (I_2 x ... x I_N x S_1), the last k columns X x_1 Phi_1^T likewise; the
//     core chain reduces the first part (H comes out with S_1 last and is
//     transposed once), every Y_n with n > 1 reduces the second;
//   * E = X x_2 Phi_2^T, which Y_1 reduces further.
// Y_n with n > 1 comes out with its columns in a permuted order (Phi_1's
// index slowest); a column permutation leaves range(Y_n), and so R-PET's
// result, unchanged.  The products after the first act on tensors k / I_p
// (or S_1 / I_1) of X's size.
void rpet_kron_sketches(Ctx& c, const float* X, const Geom& g, const Plan& pl, uint64_t seed,
                        const float* const* Omega, const float* const* Omega_t, float* const* Omt,
                        float* const* Ys, float* H) {
  const int N = g.N, k = pl.kron;
  const int S0 = pl.S[0];
  const int64_t J0 = g.J(0);
  Scope sc(c);
  // Phi_p (I_p x k), explicit or drawn on stream_id 10N + p
  const float* Phi[RHOSVD_MAX_MODES];
  for (int p = 0; p < N; ++p) {
    if (Omega != nullptr && Omega[p] != nullptr) {
      Phi[p] = Omega[p];
    } else {
      float* f = c.take<float>((size_t)g.d[p] * k);
      op_omega(c, seed, (uint32_t)(10 * N + p), g.d[p], k, f);
      Phi[p] = f;
    }
  }
  for (int n = 0; n < N; ++n)
    if (Omt[n] != nullptr) op_omega(c, seed, (uint32_t)(N + n), pl.S[n], (int)g.d[n], Omt[n]);
  auto omt = [&](int n) { return (Omega_t != nullptr && Omega_t[n] != nullptr) ? Omega_t[n] : Omt[n]; };
  // T: X's modes 2..N at positions 0..N-2, then the first product's index
  Geom tg;
  tg.N = N;
  for (int q = 0; q + 1 < N; ++q) tg.d[q] = g.d[q + 1];
  size_t max_t = 1, max_m = 1;
  {
    Geom t = tg;
    t.d[N - 1] = S0;
    for (int q = 0; q + 1 < N; ++q) {
      t.d[q] = pl.S[q + 1];
      max_t = std::max<size_t>(max_t, (size_t)t.numel());
    }
    for (int n = 0; n < N; ++n) max_m = std::max<size_t>(max_m, (size_t)g.d[n] * std::max(pl.S[n], k));
    // a factor chain only shrinks its start (k <= I_p), so its intermediates are
    // bounded by X x_1 Phi_1^T or X x_2 Phi_2^T
    max_t = std::max<size_t>(max_t, (size_t)J0 * k);
    max_t = std::max<size_t>(max_t, (size_t)g.J(N > 1 ? 1 : 0) * k);
  }
  float* Mc = c.take<float>((size_t)g.d[0] * (S0 + k));
  float* C = c.take<float>((size_t)J0 * (S0 + k));
  float* E = c.take<float>((size_t)g.J(1) * k);
  float* Hp = c.take<float>((size_t)max_t);
  float* Tb[2] = {c.take<float>(max_t), c.take<float>(max_t)};
  float* Mt = c.take<float>(max_m);
  size_t max_w = 1;
  for (int n = 0; n < N; ++n) max_w = std::max<size_t>(max_w, (size_t)g.d[n] * pl.K[n]);
  float* Wn = c.take<float>(max_w);
  // read 1: C(j, s) = (X x_1 [Omega~_1^T Phi_1])(s, j), column-major in (j, s)
  c.launches += 1;
  if (!c.dry) {
    c.check(launch_transpose(omt(0), S0, g.d[0], S0, Mc, c.s));
    c.check(cudaMemcpyAsync(Mc + (size_t)g.d[0] * S0, Phi[0], sizeof(float) * g.d[0] * k,
                            cudaMemcpyDeviceToDevice, c.s));
  }
  op_ttm(c, mode_view(X, g, 0), Mc, 1, g.d[0], S0 + k, OView{C, J0, 1});
  // chain src (geometry t) over the listed (position, X mode) pairs; the last product into dst
  auto chain = [&](const float* src, Geom t, const int* pos, const int* xm, int nm, bool core,
                   float* dst) -> Geom {
    const float* cur = src;
    int ping = 0;
    for (int q = 0; q < nm; ++q) {
      const int p = pos[q], m = xm[q];
      const int width = core ? pl.S[m] : k;
      const float* M = Phi[m];
      if (core) {                                  // the TTM takes Omega~_m^T (I_m x S_m)
        c.launches += 1;
        if (!c.dry) c.check(launch_transpose(omt(m), pl.S[m], g.d[m], pl.S[m], Mt, c.s));
        M = Mt;
      }
      float* out = (q == nm - 1) ? dst : Tb[ping];
      ttm_mode(c, cur, t, p, M, 1, g.d[m], width, out);
      t.d[p] = width;
      cur = out;
      ping ^= 1;
    }
    return t;
  };
  auto emit = [&](const float* red, const Geom& t, int p, int n) {   // Y_n = unfolding at position p
    c.launches += 1;
    if (!c.dry) c.check(launch_unfold(red, t.L(p), t.d[p], t.Rt(p), Ys[n], c.s));
  };
  int pos[RHOSVD_MAX_MODES], xm[RHOSVD_MAX_MODES], nm;
  // core sketch: H' = (X x_1 Omega~_1) x_2 Omega~_2 ... (S_2 x ... x S_N x S_1), then H = H'^T
  {
    Geom t = tg;
    t.d[N - 1] = S0;
    nm = 0;
    for (int q = 0; q + 1 < N; ++q) {
      pos[nm] = q;
      xm[nm++] = q + 1;
    }
    const int64_t rest = t.numel() / S0;
    int64_t hrest = 1;
    for (int q = 1; q < N; ++q) hrest *= pl.S[q];
    if (nm > 0) chain(C, t, pos, xm, nm, true, Hp);
    c.launches += 1;
    if (!c.dry) c.check(launch_transpose(nm > 0 ? Hp : C, nm > 0 ? hrest : rest, S0, nm > 0 ? hrest : rest, H, c.s));
  }
  // factor sketches of modes 2..N from X x_1 Phi_1^T (mode n at position n - 1)
  const float* CF = C + (size_t)J0 * S0;
  for (int n = 1; n < N; ++n) {
    Geom t = tg;
    t.d[N - 1] = k;
    nm = 0;
    for (int q = 0; q + 1 < N; ++q)
      if (q != n - 1) {
        pos[nm] = q;
        xm[nm++] = q + 1;
      }
    if (nm == 0) {
      emit(CF, t, n - 1, n);
    } else {
      const Geom r = chain(CF, t, pos, xm, nm, false, Wn);
      emit(Wn, r, n - 1, n);
    }
  }
  // read 2: E = X x_2 Phi_2^T, then Y_1
  ttm_mode(c, X, g, 1, Phi[1], 1, g.d[1], k, E);
  {
    Geom t = g;
    t.d[1] = k;
    nm = 0;
    for (int p = 2; p < N; ++p) {
      pos[nm] = p;
      xm[nm++] = p;
    }
    if (nm == 0) {
      emit(E, t, 0, 0);
    } else {
      const Geom r = chain(E, t, pos, xm, nm, false, Wn);
      emit(Wn, r, 0, 0);
    }
  }
  for (int n = 0; n < N; ++n) op_orth(c, Ys[n], g.d[n], pl.K[n], g.d[n]);
}

void run_rpet(Ctx& c, const float* X, const Geom& g, const int32_t* ranks, const Plan& pl, uint64_t seed,
              const float* const* Omega, const float* const* Omega_t, float* const* U, float* G) {
  const int N = g.N;
  size_t max_jk = 1, max_kk = 1;
  for (int n = 0; n < N; ++n) {
    max_jk = std::max<size_t>(max_jk, (size_t)g.J(n) * pl.K[n]);
    max_kk = std::max<size_t>(max_kk, (size_t)pl.K[n] * pl.K[n]);
  }
  float* Ys[RHOSVD_MAX_MODES];
  float* Omt[RHOSVD_MAX_MODES];
  float* Pt[RHOSVD_MAX_MODES];
  float* Vb[RHOSVD_MAX_MODES];
  for (int n = 0; n < N; ++n) {
    Ys[n] = c.take<float>((size_t)g.d[n] * pl.K[n]);
    const bool gen = (Omega_t == nullptr || Omega_t[n] == nullptr);
    Omt[n] = gen ? c.take<float>((size_t)pl.S[n] * g.d[n]) : nullptr;
    Pt[n] = c.take<float>((size_t)pl.S[n] * pl.K[n]);
    Vb[n] = c.take<float>((size_t)ldu_of(pl.K[n]) * ranks[n]);
  }
  bool need_om = false;
  for (int n = 0; n < N; ++n) need_om |= (Omega == nullptr || Omega[n] == nullptr);
  float* Om = (need_om && pl.kron == 0) ? c.take<float>(max_jk) : nullptr;
  Geom hs = g, cs = g;
  for (int n = 0; n < N; ++n) {
    hs.d[n] = pl.S[n];
    cs.d[n] = pl.K[n];
  }
  float* H = c.take<float>((size_t)hs.numel());
  size_t max_c = 1;
  {
    Geom t = hs;
    for (int n = 0; n < N; ++n) {
      t.d[n] = pl.K[n];
      max_c = std::max<size_t>(max_c, (size_t)t.numel());
    }
  }
  float* Cb[2] = {c.take<float>(max_c), c.take<float>(max_c)};
  double* Gd = c.take<double>(max_kk);
  float* Lf = c.take<float>(max_kk);

  // R-PET (Alg. 9, Sec. 5.1): factor sketches and their bases, the core
  // sketch, recovery of the core by pseudo-inverses, truncation.  With a
  // reduced dtype the single pass reads the reduced-precision copy of X and the
  // seeded test matrices are rounded to its format.
  if (pl.kron > 0) {
    rpet_kron_sketches(c, X, g, pl, seed, Omega, Omega_t, Omt, Ys, H);
  } else {
    const LpCopy lp = lp_make(c, X, g, pl.dtype);
    // Factor sketches Y_n = X_(n) Omega_n and their orthonormal bases Q_n
    for (int n = 0; n < N; ++n) {
      const float* W = (Omega != nullptr) ? Omega[n] : nullptr;
      if (lp.eb != 0 && W == nullptr) {
        lp_omega(c, lp, seed, (uint32_t)n, g.J(n), pl.K[n], Om);
        W = Om;
      }
      if (lp.eb != 0 && lp_sketch(c, lp, g, n, W, pl.K[n], Ys[n])) {
      } else if (W != nullptr) {
        op_sketch(c, mode_view(X, g, n), WView{W, g.L(n), g.J(n)}, pl.K[n], Ys[n], g.d[n]);
      } else {
        op_sketch_seeded(c, mode_view(X, g, n), pl.K[n], seed, (uint32_t)n, Ys[n], g.d[n], Om);
      }
      op_orth(c, Ys[n], g.d[n], pl.K[n], g.d[n]);
    }
    // core sketch H
    for (int n = 0; n < N; ++n)
      if (Omt[n] != nullptr) {
        if (lp.eb != 0) lp_omega(c, lp, seed, (uint32_t)(N + n), pl.S[n], (int)g.d[n], Omt[n]);
        else op_omega(c, seed, (uint32_t)(N + n), pl.S[n], (int)g.d[n], Omt[n]);
      }
    core_sketch_chain(c, X, g, pl.S, seed, Omega_t, Omt, H, &lp);
  }
  // recovered core C = H x_n (Omega~_n Q_n)^+ with the pseudo-inverse from the normal
  // equations (Omega~_n Q_n is a well-conditioned Gaussian-times-orthonormal
  // matrix): P^T = A (A^T A)^-1 = (A R^-1) R^-T, R^T R = A^T A
  Geom t = hs;
  const float* cur = H;
  int ping = 0;
  for (int n = 0; n < N; ++n) {
    const int K = pl.K[n], S = pl.S[n];
    const int64_t I = g.d[n];
    const float* om = (Omega_t != nullptr && Omega_t[n] != nullptr) ? Omega_t[n] : Omt[n];
    float* A = Pt[n];
    {
      // A(s, k) = sum_i Omega~(s, i) Q(i, k): the sketch of the S x I matrix
      // Omega~ (column-major) with W = Q, split over i
      View ov;
      ov.p = om;
      ov.L = 1;
      ov.I = S;
      ov.Rt = I;
      ov.s_i = 1;
      ov.s_r = S;
      op_sketch(c, ov, WView{Ys[n], 1, I}, K, A, S);
    }
    op_gram_matrix(c, A, S, K, S, Gd);
    c.launches += 2;
    if (!c.dry) c.check(launch_chol(Gd, K, Lf, nullptr, 0, 0, RHOSVD_EBREAKDOWN, c.st, c.s));
    if (!c.dry) c.check(launch_trsm_rows(A, S, K, S, Lf, 1, c.st, c.s));   // A (A^T A)^-1, in place
    float* dst = Cb[ping];
    ttm_mode(c, cur, t, n, A, 1, S, K, dst);   // M(s, k) = P^T(s, k)
    t.d[n] = K;
    cur = dst;
    ping ^= 1;
  }
  // truncation: a truncated HOSVD of the recovered core C (K_1 x ... x K_N)
  for (int n = 0; n < N; ++n) {
    const int K = pl.K[n], R = ranks[n];
    const int64_t L = cs.L(n), Rt = cs.Rt(n);
    View cv;
    cv.p = cur;
    cv.L = L;
    cv.I = K;
    cv.Rt = Rt;
    cv.s_i = L;
    cv.s_r = L * K;
    op_gram_df(c, cv, WView{cur, L * K, L}, K, Gd);
    c.launches += 1;
    if (!c.dry) c.check(launch_small_eig(Gd, K, R, Vb[n], ldu_of(K), nullptr, c.st, c.s));
    lift_factor(c, Ys[n], g.d[n], K, Vb[n], R, U[n]);
  }
  Geom tc = cs;
  const float* chain = cur;
  float* bufs[2] = {Cb[0], Cb[1]};
  int which = (cur == Cb[0]) ? 1 : 0;   // the buffer not holding C
  for (int n = 0; n < N; ++n) {
    float* dst = (n == N - 1) ? G : bufs[which];
    ttm_mode(c, chain, tc, n, Vb[n], 1, ldu_of(pl.K[n]), ranks[n], dst);
    tc.d[n] = ranks[n];
    chain = dst;
    which ^= 1;
  }
}

// Refinement: sweeps of RP-HOOI (Alg. 7) on the FP32 X, starting from the
// factors U[n] (I_n x R_n) of the decomposition.  For each mode n in turn
// S = X x_{p != n} U_p^T with the latest factors, and U_n is re-formed by
// Alg. 1 with q = 0 on S_(n) (sketch width min(R_n + p, I_n, J_n), truncation
// to R_n); the core is X x_1 U_1^T ... x_N U_N^T with the new factors.  Two
// full reads of X per sweep: S_1 is formed starting from the last mode, and
// T = X x_1 U_1^T (after U_1 is updated) serves every later mode, extended by
// one factor per mode as the sweep goes on.  Test matrices of sweep t, mode n
// are seeded on stream_id 2N + tN + n.
void run_refine(Ctx& c, const float* X, const Geom& g, const int32_t* ranks, const Plan& pl, uint64_t seed,
                float* const* U, float* G) {
  const int N = g.N;
  if (pl.refine <= 0 || N < 2) return;
  // sizes: the chains' intermediates, the per-mode S_n, Alg. 1's buffers
  size_t max_t = 1, max_jk = 1, max_ik = 1, max_kk = 1;
  int Kr[RHOSVD_MAX_MODES];
  for (int n = 0; n < N; ++n) {
    int64_t J = 1;
    for (int k = 0; k < N; ++k)
      if (k != n) J *= ranks[k];
    Kr[n] = (int)std::min<int64_t>(ranks[n] + pl.p, std::min<int64_t>(g.d[n], J));
    Kr[n] = std::max(Kr[n], (int)ranks[n]);
    max_jk = std::max<size_t>(max_jk, (size_t)J * Kr[n]);
    max_ik = std::max<size_t>(max_ik, (size_t)g.d[n] * Kr[n]);
    max_kk = std::max<size_t>(max_kk, (size_t)ldu_of(Kr[n]) * ranks[n]);
  }
  {
    Geom t = g;                                       // X x_{N-1} ... (chain of S_1)
    for (int p = N - 1; p >= 1; --p) {
      t.d[p] = ranks[p];
      max_t = std::max<size_t>(max_t, (size_t)t.numel());
    }
    t = g;                                            // T = X x_1 U_1^T and its extensions
    t.d[0] = ranks[0];
    max_t = std::max<size_t>(max_t, (size_t)t.numel());
  }
  Scope sc(c);
  float* Tb[2] = {c.take<float>(max_t), c.take<float>(max_t)};   // T and its extension (ping-pong)
  float* Cb[2] = {c.take<float>(max_t), c.take<float>(max_t)};   // the chain forming S_n
  float* Yb = c.take<float>(max_ik);
  float* Zb = c.take<float>(max_jk);
  float* Om = c.take<float>(max_jk);
  float* Ub = c.take<float>(max_kk);
  // chain: src (geometry t) x_p U_p^T for p = N-1 down to lo, p != skip; returns the result
  auto chain = [&](const float* src, Geom& t, int lo, int skip) -> const float* {
    const float* cur = src;
    int ping = 0;
    for (int p = N - 1; p >= lo; --p) {
      if (p == skip) continue;
      float* dst = Cb[ping];
      ttm_mode(c, cur, t, p, U[p], 1, g.d[p], ranks[p], dst);
      t.d[p] = ranks[p];
      cur = dst;
      ping ^= 1;
    }
    return cur;
  };
  for (int sweep = 0; sweep < pl.refine; ++sweep) {
    const uint32_t sb = (uint32_t)(2 * N + sweep * N);
    // mode 1: S_1 = X x_{p > 1} U_p^T
    Geom t = g;
    const float* s1 = chain(X, t, 1, -1);
    alg1_mode(c, s1, t, 0, Kr[0], ranks[0], 0, seed, nullptr, Yb, Zb, Om, Ub, sb);
    lift_factor(c, Yb, g.d[0], Kr[0], Ub, ranks[0], U[0]);
    // T = X x_1 U_1^T, then for n >= 2: S_n = T x_{p > n} U_p^T, T <- T x_n U_n^T
    Geom tg = g;
    int tp = 0;
    const float* T = X;
    {
      float* dst = (N == 1) ? G : Tb[tp];
      ttm_mode(c, X, tg, 0, U[0], 1, g.d[0], ranks[0], dst);
      tg.d[0] = ranks[0];
      T = dst;
      tp ^= 1;
    }
    for (int n = 1; n < N; ++n) {
      Geom ts = tg;
      const float* sn = chain(T, ts, n + 1, -1);
      alg1_mode(c, sn, ts, n, Kr[n], ranks[n], 0, seed, nullptr, Yb, Zb, Om, Ub, sb);
      lift_factor(c, Yb, g.d[n], Kr[n], Ub, ranks[n], U[n]);
      float* dst = (n == N - 1) ? G : Tb[tp];
      ttm_mode(c, T, tg, n, U[n], 1, g.d[n], ranks[n], dst);
      tg.d[n] = ranks[n];
      T = dst;
      tp ^= 1;
    }
  }
}

// ------------------------------------------------------------------ fixed accuracy

// Reads n doubles from the device (stream-ordered) and waits for the stream.
bool host_read(Ctx& c, const double* d, double* h, int n) {
  if (cudaMemcpyAsync(h, d, sizeof(double) * n, cudaMemcpyDeviceToHost, c.s) != cudaSuccess) return false;
  return cudaStreamSynchronize(c.s) == cudaSuccess;
}

// Fixed-accuracy R-STHOSVD: Alg. 8 with the blocked randomized QB with an
// error indicator in place of Alg. 1 (the fixed-precision range finders Sec. 5
// cites).  Per mode the tolerance is eps ||X||_F / sqrt(N), so that the
// sequential truncation keeps the total error within eps ||X||_F.  For the
// unfolding A = S_(n) of the current core the basis Q grows by blocks of b
// columns: Y = A Omega_i - Q (B Omega_i), Q_i = orth(Y) re-orthogonalised once
// against Q, B_i = Q_i^T A, and the indicator E = ||A||_F^2 - ||P_Q A||_F^2
// (equal to ||A - Q B||_F^2; the projected energy tr((Q^T Q)^-1 B B^T) to first
// order in Q^T Q - I: sum ||B_i||_F^2 less sum_ij (Q^T Q - I)_ij (B B^T)_ij) is
// read on the host after each block; the loop stops at E <= tol^2 (after at
// least one block) or kmax_n columns.  Then B = Ubar Sigma Vbar^T through
// the eigenvectors of B B^T, R_n = the smallest r with E + sum_{i>r} sigma_i^2
// <= tol^2 (at least 1), U_n = Q Ubar_R and S_(n) <- Ubar_R^T B.  Block i of
// mode n is drawn on stream_id 4096 + 256 n + i.  A dry run (sizing) takes every
// block and keeps kmax_n columns.
rhosvd_status run_fixed_accuracy(Ctx& c, const float* X, const Geom& g0, double eps, int block,
                                 const int32_t* kmax, uint64_t seed, int32_t* ranks_out, float* const* U,
                                 float* G) {
  const int N = g0.N;
  size_t max_s = 1, max_q = 1, max_bt = 1, max_om = 1, max_kk = 1;
  {
    Geom g = g0;
    for (int n = 0; n < N; ++n) {
      const int64_t J = g.J(n);
      max_q = std::max<size_t>(max_q, (size_t)g.d[n] * kmax[n]);
      max_bt = std::max<size_t>(max_bt, (size_t)J * kmax[n]);
      max_om = std::max<size_t>(max_om, (size_t)J * block);
      max_kk = std::max<size_t>(max_kk, (size_t)ldu_of(kmax[n]) * kmax[n]);
      g.d[n] = kmax[n];
      max_s = std::max<size_t>(max_s, (size_t)g.numel());
    }
  }
  float* Qb = c.take<float>(max_q);
  float* Bt = c.take<float>(max_bt);
  float* Om = c.take<float>(max_om);
  float* Cm = c.take<float>((size_t)RHOSVD_MAX_K * block);
  float* Tmp = c.take<float>(max_q);
  float* Ub = c.take<float>(max_kk);
  float* sv = c.take<float>(RHOSVD_MAX_K);
  double* Gd = c.take<double>((size_t)RHOSVD_MAX_K * RHOSVD_MAX_K);   // C = B B^T
  double* Gq = c.take<double>((size_t)RHOSVD_MAX_K * RHOSVD_MAX_K);   // M = Q^T Q
  double* pe = c.take<double>(2);
  float* Sb[2] = {c.take<float>(max_s), c.take<float>(max_s)};
  Geom g = g0;
  const float* cur = X;
  int ping = 0;
  double tol2 = 0.0;
  for (int n = 0; n < N; ++n) {
    const int64_t I = g.d[n], L = g.L(n), J = g.J(n);
    const View av = mode_view(cur, g, n);
    // ||A||_F^2 of the current core (a one-column Gram)
    op_gram_matrix(c, cur, g.numel(), 1, g.numel(), Gd);
    double a2 = 0.0;
    if (!c.dry && !host_read(c, Gd, &a2, 1)) return RHOSVD_ECUDA;
    if (n == 0) tol2 = eps * eps * a2 / N;
    double e = a2, sum_bb = 0.0;
    int kq = 0;
    for (int i = 0; kq < kmax[n]; ++i) {
      if (!c.dry && kq > 0 && e <= tol2) break;
      const int b = std::min(block, kmax[n] - kq);
      float* Y = Qb + (size_t)kq * I;
      op_omega(c, seed, (uint32_t)(4096 + 256 * n + i), J, b, Om);
      op_sketch(c, av, WView{Om, L, J}, b, Y, I);                            // A Omega_i
      if (kq > 0) {
        // Y -= Q (B Omega_i), B Omega_i = Bt^T Omega_i (kq x b)
        View btv{Bt, J, kq, 1, J, J * kq};
        op_sketch(c, btv, WView{Om, J, J}, b, Cm, kq);
        op_ttm(c, matrix_view(Qb, I, kq, I), Cm, 1, kq, b, OView{Tmp, I, 0});
        c.launches += 1;
        if (!c.dry) c.check(launch_axpy(Y, Tmp, -1.f, I * (int64_t)b, c.s));
      }
      op_orth(c, Y, I, b, I);
      if (kq > 0) {                                                           // once more against Q
        View qv{Qb, I, kq, 1, I, I * kq};
        op_sketch(c, qv, WView{Y, I, I}, b, Cm, kq);                          // Q^T Q_i
        op_ttm(c, matrix_view(Qb, I, kq, I), Cm, 1, kq, b, OView{Tmp, I, 0});
        c.launches += 1;
        if (!c.dry) c.check(launch_axpy(Y, Tmp, -1.f, I * (int64_t)b, c.s));
        op_orth(c, Y, I, b, I);
      }
      // B_i^T = A^T Q_i by the FP32 FMA TTM (round to nearest): the tensor cores'
      // truncating accumulation leaves B ~5e-7 low, which E would carry as
      // ~1e-6 ||A||^2 and so could not resolve eps below ~2e-3
      c.launches += 1;
      if (!c.dry) c.check(launch_ttm(av, Y, 1, I, b, OView{Bt + (size_t)kq * J, J, L}, nullptr, c.s));
      // E = ||A||^2 - ||P_Q A||^2 with ||P_Q A||^2 = tr(M^-1 C), M = Q^T Q,
      // C = B B^T: tr(C) = sum ||B_i||^2 from FP64-accurate one-column Grams,
      // less the first-order term sum_ij (M - I)_ij C_ij, for which an FP32 Gram
      // of B suffices.  Q is orthonormal only to FP32 storage (||M - I|| ~ 1e-6),
      // which the plain sum ||B_i||^2 would carry into E as ~1e-6 ||A||^2
      op_gram_matrix(c, Bt + (size_t)kq * J, J * (int64_t)b, 1, J * (int64_t)b, pe);
      kq += b;
      op_gram_matrix(c, Qb, I, kq, I, Gq);
      op_gram_matrix(c, Bt, J, kq, J, Gd, false);
      c.launches += 1;
      if (!c.dry) c.check(launch_proj_energy(Gq, Gd, kq, pe + 1, c.s));
      double h[2] = {0.0, 0.0};
      if (!c.dry && !host_read(c, pe, h, 2)) return RHOSVD_ECUDA;
      sum_bb += h[0];
      e = a2 - sum_bb + h[1];
    }
    // truncation: eigenvectors of B B^T (FP64-accurate Gram, all kq, descending) and the rank
    op_gram_matrix(c, Bt, J, kq, J, Gd);
    c.launches += 1;
    if (!c.dry) c.check(launch_small_eig(Gd, kq, kq, Ub, ldu_of(kq), sv, c.st, c.s));
    int r = kq;
    if (!c.dry) {
      float hs[RHOSVD_MAX_K];
      if (cudaMemcpyAsync(hs, sv, sizeof(float) * kq, cudaMemcpyDeviceToHost, c.s) != cudaSuccess ||
          cudaStreamSynchronize(c.s) != cudaSuccess)
        return RHOSVD_ECUDA;
      // smallest r with E + sum_{i >= r} sigma_i^2 <= tol^2 (0-based), tail[r] the suffix sums
      double tail[RHOSVD_MAX_K + 1];
      tail[kq] = 0.0;
      for (int t = kq - 1; t >= 0; --t) tail[t] = tail[t + 1] + (double)hs[t] * hs[t];
      const double res = std::max(e, 0.0);
      r = kq;
      for (int t = 0; t <= kq; ++t)
        if (res + tail[t] <= tol2) {
          r = t;
          break;
        }
      r = std::max(r, 1);
    }
    lift_factor(c, Qb, I, kq, Ub, r, U[n]);
    // sign convention (largest-magnitude entry of each factor column positive): the
    // next modes sketch the core in this mode's coordinates, so the convention
    // fixes which test matrix they effectively see
    c.launches += 1;
    if (!c.dry) c.check(launch_sign_canon(U[n], I, r, Ub, ldu_of(kq), kq, c.s));
    float* dst = (n == N - 1) ? G : Sb[ping];
    refold_core(c, Bt, g, n, kq, Ub, r, dst);
    g.d[n] = r;
    ranks_out[n] = r;
    cur = dst;
    ping ^= 1;
  }
  return RHOSVD_OK;
}

rhosvd_status finish(const Ctx& c) { return c.err == cudaSuccess ? RHOSVD_OK : RHOSVD_ECUDA; }

rhosvd_status begin(Ctx& c, void* ws, size_t ws_bytes, void* stream) {
  if (ws == nullptr || ws_bytes < sizeof(DevStatus) || (reinterpret_cast<uintptr_t>(ws) % ALIGN) != 0)
    return RHOSVD_EINVAL;
  c.dry = false;
  c.base = static_cast<char*>(ws);
  c.off = sizeof(DevStatus);
  c.high = c.off;
  c.s = static_cast<cudaStream_t>(stream);
  c.st = static_cast<DevStatus*>(ws);
  if (cudaMemsetAsync(ws, 0, sizeof(DevStatus), c.s) != cudaSuccess) return RHOSVD_ECUDA;
  return RHOSVD_OK;
}

Ctx dry_ctx() {
  Ctx c;
  c.dry = true;
  c.off = sizeof(DevStatus);
  c.high = c.off;
  return c;
}

size_t primitive_ws(const Geom& g, int Kmax) {
  // largest temporaries of the primitive calls: Z (J x K), Omega (J x K),
  // a core chain ping-pong, sketch partials and orth scratch
  Ctx c = dry_ctx();
  size_t max_jk = 1, max_n = (size_t)g.numel();
  for (int n = 0; n < g.N; ++n) max_jk = std::max<size_t>(max_jk, (size_t)g.J(n) * Kmax);
  c.take<float>(max_jk);
  c.take<float>(max_jk);
  c.take<float>(max_n);
  c.take<float>(max_n);
  size_t fixed = c.off;
  size_t extra = 0;
  for (int n = 0; n < g.N; ++n) {
    extra = std::max(extra, sketch_scratch_floats(g.d[n], Kmax, g.J(n)) * sizeof(double));
    SketchPlan pz = plan_sketch(Kmax, Kmax, g.J(n));
    extra = std::max(extra, sketch_partial_floats(pz, Kmax, Kmax) * sizeof(double));
  }
  extra += 4 * (size_t)RHOSVD_MAX_K * RHOSVD_MAX_K * sizeof(double) +
           (size_t)RHOSVD_MAX_K * RHOSVD_MAX_K * sizeof(float) + 8 * ALIGN;
  return fixed + extra;
}

}  // namespace
}  // namespace rhosvd

using namespace rhosvd;

extern "C" {

const char* rhosvd_status_string(rhosvd_status s) {
  switch (s) {
    case RHOSVD_OK: return "ok";
    case RHOSVD_EINVAL: return "invalid argument";
    case RHOSVD_ENOMEM: return "workspace too small";
    case RHOSVD_ECUDA: return "CUDA runtime error";
    case RHOSVD_ENONFINITE: return "non-finite value in the input or a sketch";
    case RHOSVD_EBREAKDOWN: return "orthonormalisation breakdown";
    case RHOSVD_ETIMEOUT: return "device wait timed out";
    case RHOSVD_EUNSUPPORTED: return "unsupported request";
  }
  return "unknown status";
}

rhosvd_status rhosvd_plan(const rhosvd_shape* shape, const int32_t* ranks, const rhosvd_opts* opts,
                          int32_t* K_out, int32_t* S_out, int64_t* J_out) {
  Geom g;
  rhosvd_status s = validate_shape(shape, g);
  if (s != RHOSVD_OK) return s;
  Plan pl;
  s = make_plan(g, ranks, opts, pl);
  if (s != RHOSVD_OK) return s;
  for (int n = 0; n < g.N; ++n) {
    if (K_out) K_out[n] = pl.K[n];
    if (S_out) S_out[n] = pl.S[n];
    if (J_out) J_out[n] = pl.J[n];
  }
  return RHOSVD_OK;
}

static size_t decompose_ws(const Geom& g, const int32_t* ranks, const rhosvd_opts* o, const Plan& pl,
                           const float* const* Omega, const float* const* Omega_t) {
  Ctx c = dry_ctx();
  float* U[RHOSVD_MAX_MODES] = {nullptr};
  if (o->algo == RHOSVD_ALGO_RSTHOSVD) run_rsthosvd(c, nullptr, g, ranks, pl, o->q, o->seed, Omega, U, nullptr);
  else if (o->algo == RHOSVD_ALGO_RHOSVD) run_rhosvd(c, nullptr, g, ranks, pl, o->q, o->seed, Omega, U, nullptr);
  else run_rpet(c, nullptr, g, ranks, pl, o->seed, Omega, Omega_t, U, nullptr);
  run_refine(c, nullptr, g, ranks, pl, o->seed, U, nullptr);
  return c.high;
}

int64_t rhosvd_launch_count(const rhosvd_shape* shape, const int32_t* ranks, const rhosvd_opts* opts) {
  Geom g;
  if (validate_shape(shape, g) != RHOSVD_OK) return -1;
  Plan pl;
  if (make_plan(g, ranks, opts, pl) != RHOSVD_OK) return -1;
  Ctx c = dry_ctx();
  float* U[RHOSVD_MAX_MODES] = {nullptr};
  if (opts->algo == RHOSVD_ALGO_RSTHOSVD) run_rsthosvd(c, nullptr, g, ranks, pl, opts->q, opts->seed, nullptr, U, nullptr);
  else if (opts->algo == RHOSVD_ALGO_RHOSVD) run_rhosvd(c, nullptr, g, ranks, pl, opts->q, opts->seed, nullptr, U, nullptr);
  else run_rpet(c, nullptr, g, ranks, pl, opts->seed, nullptr, nullptr, U, nullptr);
  run_refine(c, nullptr, g, ranks, pl, opts->seed, U, nullptr);
  return c.launches;
}

size_t rhosvd_workspace_size(const rhosvd_shape* shape, const int32_t* ranks, const rhosvd_opts* opts) {
  Geom g;
  if (validate_shape(shape, g) != RHOSVD_OK) return 0;
  Plan pl;
  if (make_plan(g, ranks, opts, pl) != RHOSVD_OK) return 0;
  return decompose_ws(g, ranks, opts, pl, nullptr, nullptr);
}

size_t rhosvd_primitive_workspace_size(const rhosvd_shape* shape, int32_t Kmax) {
  Geom g;
  if (validate_shape(shape, g) != RHOSVD_OK || Kmax < 1 || Kmax > RHOSVD_MAX_K) return 0;
  return primitive_ws(g, Kmax);
}

rhosvd_status rhosvd_omega(uint64_t seed, uint32_t stream_id, int64_t rows, int32_t cols, float* Omega,
                           int64_t ld, void* stream) {
  if (rows < 0 || cols < 0 || ld < rows || (Omega == nullptr && rows * (int64_t)cols > 0)) return RHOSVD_EINVAL;
  if (rows == 0 || cols == 0) return RHOSVD_OK;
  cudaError_t e = launch_omega(seed, stream_id, rows, cols, Omega, ld, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? RHOSVD_OK : RHOSVD_ECUDA;
}

rhosvd_status rhosvd_sketch(const float* X, const rhosvd_shape* shape, int32_t mode, int32_t K, uint64_t seed,
                            const float* Omega, float* Y, void* ws, size_t ws_bytes, void* stream) {
  Geom g;
  rhosvd_status s = validate_shape(shape, g);
  if (s != RHOSVD_OK) return s;
  if (X == nullptr || Y == nullptr || mode < 0 || mode >= g.N || K < 1 || K > RHOSVD_MAX_K) return RHOSVD_EINVAL;
  if (ws_bytes < primitive_ws(g, K)) return RHOSVD_ENOMEM;
  Ctx c;
  if ((s = begin(c, ws, ws_bytes, stream)) != RHOSVD_OK) return s;
  const int64_t J = g.J(mode);
  if (Omega == nullptr) {
    float* Om = c.take<float>((size_t)J * K);
    op_sketch_seeded(c, mode_view(X, g, mode), K, seed, (uint32_t)mode, Y, g.d[mode], Om);
  } else {
    op_sketch(c, mode_view(X, g, mode), WView{Omega, g.L(mode), J}, K, Y, g.d[mode]);
  }
  return finish(c);
}

rhosvd_status rhosvd_sketch_all(const float* X, const rhosvd_shape* shape, const int32_t* K, const int32_t* S,
                                uint64_t seed, const float* const* Omega, const float* const* Omega_tilde,
                                float* const* Y, float* H, void* ws, size_t ws_bytes, void* stream) {
  Geom g;
  rhosvd_status s = validate_shape(shape, g);
  if (s != RHOSVD_OK) return s;
  if (X == nullptr || K == nullptr || Y == nullptr || (H != nullptr && S == nullptr)) return RHOSVD_EINVAL;
  int kmax = 1;
  for (int n = 0; n < g.N; ++n) {
    if (K[n] < 1 || K[n] > RHOSVD_MAX_K || Y[n] == nullptr) return RHOSVD_EINVAL;
    if (H != nullptr && (S[n] < 1 || S[n] > (1 << 20))) return RHOSVD_EINVAL;
    kmax = std::max(kmax, (int)K[n]);
  }
  // core sketch chain needs two ping-pong tensors and the generated Omega~
  size_t need = primitive_ws(g, kmax);
  if (H != nullptr) {
    Geom t = g;
    size_t mt = 1, om = 0;
    for (int n = 0; n < g.N; ++n) {
      t.d[n] = S[n];
      mt = std::max<size_t>(mt, (size_t)t.numel());
      om += ((size_t)S[n] * g.d[n] * sizeof(float) + ALIGN);
    }
    need += 2 * (mt * sizeof(float) + ALIGN) + om;
  }
  if (ws_bytes < need) return RHOSVD_ENOMEM;
  Ctx c;
  if ((s = begin(c, ws, ws_bytes, stream)) != RHOSVD_OK) return s;
  {
    Scope sc(c);
    for (int n = 0; n < g.N; ++n) {
      const int64_t J = g.J(n);
      const float* W = (Omega != nullptr) ? Omega[n] : nullptr;
      Scope inner(c);
      if (W == nullptr) {
        float* Om = c.take<float>((size_t)J * K[n]);
        op_sketch_seeded(c, mode_view(X, g, n), K[n], seed, (uint32_t)n, Y[n], g.d[n], Om);
      } else {
        op_sketch(c, mode_view(X, g, n), WView{W, g.L(n), J}, K[n], Y[n], g.d[n]);
      }
    }
  }
  if (H != nullptr) {
    float* Omt[RHOSVD_MAX_MODES] = {nullptr};
    for (int n = 0; n < g.N; ++n) {
      if (Omega_tilde == nullptr || Omega_tilde[n] == nullptr) {
        Omt[n] = c.take<float>((size_t)S[n] * g.d[n]);
        op_omega(c, seed, (uint32_t)(g.N + n), S[n], (int)g.d[n], Omt[n]);
      }
    }
    int Si[RHOSVD_MAX_MODES];
    for (int n = 0; n < g.N; ++n) Si[n] = S[n];
    core_sketch_chain(c, X, g, Si, seed, Omega_tilde, Omt, H);
  }
  return finish(c);
}

rhosvd_status rhosvd_power(const float* X, const rhosvd_shape* shape, int32_t mode, int32_t K, float* Y_inout,
                           void* ws, size_t ws_bytes, void* stream) {
  Geom g;
  rhosvd_status s = validate_shape(shape, g);
  if (s != RHOSVD_OK) return s;
  if (X == nullptr || Y_inout == nullptr || mode < 0 || mode >= g.N || K < 1 || K > RHOSVD_MAX_K ||
      K > g.d[mode] || K > g.J(mode))
    return RHOSVD_EINVAL;
  if (ws_bytes < primitive_ws(g, K)) return RHOSVD_ENOMEM;
  Ctx c;
  if ((s = begin(c, ws, ws_bytes, stream)) != RHOSVD_OK) return s;
  const View xv = mode_view(X, g, mode);
  const int64_t I = g.d[mode], L = g.L(mode), J = g.J(mode);
  float* Zb = c.take<float>((size_t)J * K);
  op_ttm(c, xv, Y_inout, 1, I, K, OView{Zb, J, L});
  op_orth(c, Zb, J, K, J);
  op_sketch(c, xv, WView{Zb, L, J}, K, Y_inout, I);
  return finish(c);
}

rhosvd_status rhosvd_orth(float* Y, int64_t m, int32_t K, int64_t ld, int32_t* fallback_used, void* ws,
                          size_t ws_bytes, void* stream) {
  if (Y == nullptr || K < 1 || K > RHOSVD_MAX_K || m < K || ld < m) return RHOSVD_EINVAL;
  Geom g;
  g.N = 2;
  g.d[0] = m;
  g.d[1] = K;
  if (ws_bytes < primitive_ws(g, K)) return RHOSVD_ENOMEM;
  Ctx c;
  rhosvd_status s;
  if ((s = begin(c, ws, ws_bytes, stream)) != RHOSVD_OK) return s;
  op_orth(c, Y, m, K, ld);
  if (c.err != cudaSuccess) return RHOSVD_ECUDA;
  if (fallback_used != nullptr) {
    int32_t flags = 0;
    s = rhosvd_device_status(ws, ws_bytes, stream, &flags);
    *fallback_used = (flags & RHOSVD_FLAG_FALLBACK) ? 1 : 0;
    return s;
  }
  return RHOSVD_OK;
}

rhosvd_status rhosvd_core(const float* X, const rhosvd_shape* shape, const float* const* Q, const int32_t* K,
                          float* G, void* ws, size_t ws_bytes, void* stream) {
  Geom g;
  rhosvd_status s = validate_shape(shape, g);
  if (s != RHOSVD_OK) return s;
  if (X == nullptr || Q == nullptr || K == nullptr || G == nullptr) return RHOSVD_EINVAL;
  for (int n = 0; n < g.N; ++n) {
    if (K[n] < 1 || K[n] > g.d[n]) return RHOSVD_EINVAL;
    if (Q[n] == nullptr && K[n] != g.d[n]) return RHOSVD_EINVAL;
  }
  Geom t = g;
  size_t mt = 1;
  for (int n = 0; n < g.N; ++n) {
    t.d[n] = K[n];
    mt = std::max<size_t>(mt, (size_t)t.numel());
  }
  if (ws_bytes < sizeof(DevStatus) + 2 * (mt * sizeof(float) + ALIGN)) return RHOSVD_ENOMEM;
  Ctx c;
  if ((s = begin(c, ws, ws_bytes, stream)) != RHOSVD_OK) return s;
  float* Tb[2] = {c.take<float>(mt), c.take<float>(mt)};
  int last = -1;
  for (int n = 0; n < g.N; ++n)
    if (Q[n] != nullptr) last = n;
  Geom cur_g = g;
  const float* cur = X;
  int ping = 0;
  for (int n = 0; n < g.N; ++n) {
    if (Q[n] == nullptr) continue;
    float* dst = (n == last) ? G : Tb[ping];
    ttm_mode(c, cur, cur_g, n, Q[n], 1, g.d[n], K[n], dst);
    cur_g.d[n] = K[n];
    cur = dst;
    ping ^= 1;
  }
  if (last < 0 && !c.dry)
    c.check(cudaMemcpyAsync(G, X, sizeof(float) * g.numel(), cudaMemcpyDeviceToDevice, c.s));
  return finish(c);
}

rhosvd_status rhosvd_decompose(const float* X, const rhosvd_shape* shape, const int32_t* ranks,
                               const rhosvd_opts* opts, const float* const* Omega, const float* const* Omega_tilde,
                               float* const* U, float* G, void* ws, size_t ws_bytes, void* stream) {
  Geom g;
  rhosvd_status s = validate_shape(shape, g);
  if (s != RHOSVD_OK) return s;
  Plan pl;
  if ((s = make_plan(g, ranks, opts, pl)) != RHOSVD_OK) return s;
  if (X == nullptr || U == nullptr || G == nullptr) return RHOSVD_EINVAL;
  for (int n = 0; n < g.N; ++n)
    if (U[n] == nullptr) return RHOSVD_EINVAL;
  if (ws_bytes < decompose_ws(g, ranks, opts, pl, Omega, Omega_tilde)) return RHOSVD_ENOMEM;
  Ctx c;
  if ((s = begin(c, ws, ws_bytes, stream)) != RHOSVD_OK) return s;
  if (opts->algo == RHOSVD_ALGO_RSTHOSVD) run_rsthosvd(c, X, g, ranks, pl, opts->q, opts->seed, Omega, U, G);
  else if (opts->algo == RHOSVD_ALGO_RHOSVD) run_rhosvd(c, X, g, ranks, pl, opts->q, opts->seed, Omega, U, G);
  else run_rpet(c, X, g, ranks, pl, opts->seed, Omega, Omega_tilde, U, G);
  run_refine(c, X, g, ranks, pl, opts->seed, U, G);
  return finish(c);
}

static rhosvd_status validate_tol(const rhosvd_shape* shape, double eps, int32_t block, const int32_t* k_max,
                                  Geom& g) {
  rhosvd_status s = validate_shape(shape, g);
  if (s != RHOSVD_OK) return s;
  if (!(eps > 0.0 && eps < 1.0) || block < 1 || block > RHOSVD_MAX_K || k_max == nullptr) return RHOSVD_EINVAL;
  Geom t = g;
  for (int n = 0; n < g.N; ++n) {
    if (k_max[n] < 1 || k_max[n] > RHOSVD_MAX_K || k_max[n] > g.d[n] || k_max[n] > t.J(n)) return RHOSVD_EINVAL;
    t.d[n] = k_max[n];
  }
  return RHOSVD_OK;
}

size_t rhosvd_workspace_size_tol(const rhosvd_shape* shape, int32_t block, const int32_t* k_max) {
  Geom g;
  if (validate_tol(shape, 0.5, block, k_max, g) != RHOSVD_OK) return 0;
  Ctx c = dry_ctx();
  int32_t r[RHOSVD_MAX_MODES];
  float* U[RHOSVD_MAX_MODES] = {nullptr};
  run_fixed_accuracy(c, nullptr, g, 0.5, block, k_max, 0, r, U, nullptr);
  return c.high;
}

rhosvd_status rhosvd_decompose_tol(const float* X, const rhosvd_shape* shape, double eps, int32_t block,
                                   const int32_t* k_max, uint64_t seed, int32_t* ranks, float* const* U, float* G,
                                   void* ws, size_t ws_bytes, void* stream) {
  Geom g;
  rhosvd_status s = validate_tol(shape, eps, block, k_max, g);
  if (s != RHOSVD_OK) return s;
  if (X == nullptr || ranks == nullptr || U == nullptr || G == nullptr) return RHOSVD_EINVAL;
  for (int n = 0; n < g.N; ++n)
    if (U[n] == nullptr) return RHOSVD_EINVAL;
  if (ws_bytes < rhosvd_workspace_size_tol(shape, block, k_max)) return RHOSVD_ENOMEM;
  Ctx c;
  if ((s = begin(c, ws, ws_bytes, stream)) != RHOSVD_OK) return s;
  s = run_fixed_accuracy(c, X, g, eps, block, k_max, seed, ranks, U, G);
  if (s != RHOSVD_OK) return s;
  return finish(c);
}

rhosvd_status rhosvd_device_status(const void* ws, size_t ws_bytes, void* stream, int32_t* flags) {
  if (ws == nullptr || ws_bytes < sizeof(DevStatus)) return RHOSVD_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // The copy is ordered on the caller's stream and only that stream is waited
  // for: a plain cudaMemcpy would run on the legacy default stream, which waits
  // for every blocking stream of the device (other requests in flight).
  DevStatus h;
  if (cudaMemcpyAsync(&h, ws, sizeof(DevStatus), cudaMemcpyDeviceToHost, s) != cudaSuccess) return RHOSVD_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return RHOSVD_ECUDA;
  if (flags) *flags = h.flags;
  return static_cast<rhosvd_status>(h.code);
}

}  // extern "C"
