/*
 * rhosvd.h -- C ABI of the GB300 (sm_103a) randomized HOSVD / Tucker library.
 *
 * The library computes the hot path of randomized Tucker decomposition
 * (Ahmadi-Asl et al., "Randomized Algorithms for Computation of Tucker
 * Decomposition and Higher Order SVD (HOSVD)"): Gaussian mode-n sketches
 * Y_n = X_(n) Omega_n, power-iteration TTMs, thin orthonormalisation Y_n -> Q_n,
 * the core projection G = X x_1 Q_1^T ... x_N Q_N^T, and the single-pass
 * variant (R-PET) that sketches every mode and the core from one read of X.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Layout.   An N-way tensor X of sizes (I_1..I_N) is a dense FP32 array stored
 *           column-major, i_1 fastest (the column order of the n-unfolding,
 *           Sec. 2).  A torch tensor of shape (I_N, ..., I_1), contiguous, has
 *           this layout.  Matrices are column-major with the stated leading
 *           dimension.  Mode indices are 0-based (mode n is the paper's n+1).
 * Memory.   Every pointer named X, Y, Q, U, G, Omega, H or ws is a DEVICE
 *           pointer owned by the caller.  The library never allocates or frees
 *           device memory; it needs a caller-provided workspace `ws` of at
 *           least the size reported by the matching *_workspace_size query
 *           (256-byte aligned).  Host pointers are the shape/option structs,
 *           the int arrays (ranks, K, S) and the pointer arrays themselves
 *           (`const float* const*`), which are read before the call returns.
 * Streams.  `stream` is a cudaStream_t (NULL = legacy default stream).  All
 *           device work is enqueued on it; calls return without waiting for
 *           the GPU unless stated otherwise.
 * Errors.   Argument errors are detected on the host, before anything is
 *           enqueued, and returned synchronously (RHOSVD_EINVAL, RHOSVD_ENOMEM
 *           for a short workspace).  Conditions met on the GPU (non-finite
 *           values, breakdown of the orthonormalisation even after its
 *           Householder fallback, a bounded device wait that gave up) are
 *           recorded in a status word at the start of `ws` and returned by
 *           rhosvd_device_status(), which synchronises the stream.  No entry
 *           point exits, aborts or traps.  Calls with distinct workspaces are
 *           thread-safe; calls sharing a workspace must be stream-ordered.
 */
#ifndef RHOSVD_H
#define RHOSVD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RHOSVD_MAX_MODES 8
#define RHOSVD_MAX_K 128          /* largest sketch width K_n accepted */

typedef enum rhosvd_status {
  RHOSVD_OK = 0,
  RHOSVD_EINVAL = 1,        /* invalid argument; nothing was enqueued */
  RHOSVD_ENOMEM = 2,        /* workspace smaller than the size query reports */
  RHOSVD_ECUDA = 3,         /* a CUDA runtime call failed (launch or sync) */
  RHOSVD_ENONFINITE = 4,    /* a NaN/Inf reached a sketch or Gram matrix */
  RHOSVD_EBREAKDOWN = 5,    /* orthonormalisation failed even after the fallback */
  RHOSVD_ETIMEOUT = 6,      /* a bounded device-side wait gave up */
  RHOSVD_EUNSUPPORTED = 7   /* valid request outside what the library implements */
} rhosvd_status;

typedef enum rhosvd_algo {
  RHOSVD_ALGO_RHOSVD = 0,     /* RP-HOSVD, Alg. 6, factors by Alg. 1 on the original X */
  RHOSVD_ALGO_RSTHOSVD = 1,   /* R-STHOSVD, Alg. 8 (Alg. 1 on the shrinking core) */
  RHOSVD_ALGO_RPET = 2        /* R-PET, Alg. 9 (single pass over X) */
} rhosvd_algo;

/* Arithmetic of the sketch passes (the paper leaves it open).  RHOSVD_F32:
 * FP32 data, products in 3xTF32 with FP32 accumulation.  RHOSVD_BF16 and
 * RHOSVD_E4M3: the call first makes a reduced-precision copy of X (BF16, or
 * FP8 e4m3 with one power-of-two scale per frontal slice of the last mode,
 * chosen so that the slice's largest magnitude maps to at most 448), and the
 * passes listed under rhosvd_opts.dtype read that copy with BF16 (.kind::f16)
 * or e4m3 (.kind::f8f6f4) tensor-core MMAs and FP32 accumulation. */
typedef enum rhosvd_dtype {
  RHOSVD_F32 = 0,
  RHOSVD_BF16 = 1,
  RHOSVD_E4M3 = 2
} rhosvd_dtype;

/* bits of rhosvd_opts.flags */
#define RHOSVD_OPT_KRONECKER 1    /* R-PET with Kronecker-structured factor sketches (two reads of X) */

/* device status flags (bit set in the `flags` output of rhosvd_device_status) */
#define RHOSVD_FLAG_FALLBACK 1    /* a Householder fallback ran in some orthonormalisation */

typedef struct rhosvd_shape {
  int32_t N;                          /* number of modes, 1..RHOSVD_MAX_MODES */
  int64_t dims[RHOSVD_MAX_MODES];     /* I_1..I_N, each >= 1 */
} rhosvd_shape;

typedef struct rhosvd_opts {
  int32_t algo;                       /* rhosvd_algo */
  int32_t p;                          /* oversampling p >= 0 (Remark 1) */
  int32_t q;                          /* power iterations q >= 0 (Remark 1) */
  int32_t flags;                      /* RHOSVD_OPT_* bits, else 0.  RHOSVD_OPT_KRONECKER
                                         (R-PET only): the factor sketch of mode n is
                                         Y_n = (X x_{p != n} Phi_p^T)_(n), i.e. X_(n) times the
                                         Kronecker product of Gaussian matrices Phi_p (I_p x k)
                                         (the memory-efficient test matrices of Sec. 5.1), with
                                         k the smallest width such that k^(N-1) >= max K_n;
                                         every K_n becomes k^(N-1).  Phi_p is drawn on stream_id
                                         10N + p, or taken from Omega[p] (I_p x k, ld I_p).  All
                                         sketches then come from two reads of X: one product
                                         over the last mode with [Omega~_N^T Phi_N] and one over
                                         the first with Phi_1. */
  uint64_t seed;                      /* seed of the Gaussian test matrices */
  int32_t K[RHOSVD_MAX_MODES];        /* R-PET factor sketch widths, 0 => R_n + p */
  int32_t S[RHOSVD_MAX_MODES];        /* R-PET core sketch widths, 0 => 2 K_n + 1 */
  int32_t dtype;                      /* rhosvd_dtype of the sketch passes: for R-PET the
                                         single pass (every factor sketch and the first
                                         core-sketch product), for RP-HOSVD and R-STHOSVD
                                         the power-iteration products of mode 1; test
                                         matrices drawn from the seed are rounded to the
                                         format.  Passes whose layout the reduced-precision
                                         kernels do not take run in FP32. */
  int32_t refine_iters;               /* sweeps of RP-HOOI (Alg. 7) on the FP32 X after the
                                         decomposition, 0..8: for each mode in turn,
                                         S = X x_{p != n} U_p^T and U_n from Alg. 1 (q = 0,
                                         oversampling p) on S_(n); test matrices of sweep t,
                                         mode n from the seed on stream_id 2N + tN + n; the
                                         core is X x_1 U_1^T ... x_N U_N^T. */
} rhosvd_opts;

/* ---------------------------------------------------------------- sizing */

/* Sketch widths a decomposition uses.  K_out[n] = min(R_n + p, I_n, J_n)
 * where J_n is the number of columns of the unfolding that mode n sketches
 * (prod_{k != n} I_k for RP-HOSVD and R-PET, prod_{k<n} R_k prod_{k>n} I_k for
 * R-STHOSVD); for R-PET the opts.K/opts.S overrides apply and S_out[n] is the
 * core sketch width (S_n >= K_n).  J_out[n] receives J_n.  Any output
 * pointer may be NULL.  Returns RHOSVD_EINVAL on an invalid request. */
rhosvd_status rhosvd_plan(const rhosvd_shape* shape, const int32_t* ranks, const rhosvd_opts* opts,
                          int32_t* K_out, int32_t* S_out, int64_t* J_out);

/* Workspace bytes rhosvd_decompose needs for this request (0 on invalid input). */
size_t rhosvd_workspace_size(const rhosvd_shape* shape, const int32_t* ranks, const rhosvd_opts* opts);

/* Number of kernel launches one rhosvd_decompose of this request enqueues
 * with seed-drawn test matrices (-1 on invalid input); for profiling. */
int64_t rhosvd_launch_count(const rhosvd_shape* shape, const int32_t* ranks, const rhosvd_opts* opts);

/* Workspace bytes the primitive calls (sketch, sketch_all, power, orth, core)
 * need on a tensor of this shape with sketch widths up to Kmax. */
size_t rhosvd_primitive_workspace_size(const rhosvd_shape* shape, int32_t Kmax);

/* ---------------------------------------------------------------- primitives */

/* Gaussian test matrix (Omega of Alg. 1; Omega_n of Alg. 6 and Alg. 9):
 * Omega(j, k), j < rows, k < cols, written at Omega[j + k*ld] (ld >= rows).
 * Entry (j,k) is a deterministic function of (seed, stream_id, j, k):
 * Philox4x32-10 (Salmon et al. 2011) on counter (j mod 2^32, j div 2^32,
 * k div 4, stream_id) with key (seed mod 2^32, seed div 2^32), its four words
 * turned into four normals by Box-Muller on 24-bit uniforms.  Inside
 * rhosvd_decompose mode n draws Omega_n on stream_id n and the R-PET core
 * sketch Omega~_n on stream_id N + n. */
rhosvd_status rhosvd_omega(uint64_t seed, uint32_t stream_id, int64_t rows, int32_t cols,
                           float* Omega, int64_t ld, void* stream);

/* Mode-n sketch Y = X_(n) Omega (the first product of Alg. 1,
 * the factor sketches of Alg. 6 and Alg. 9).  Omega is J_n x K with leading dimension J_n
 * (J_n = prod_{k != mode} I_k); if Omega is NULL it is drawn from
 * (seed, stream_id = mode) as in rhosvd_omega.  Y is I_mode x K, ld = I_mode. */
rhosvd_status rhosvd_sketch(const float* X, const rhosvd_shape* shape, int32_t mode, int32_t K,
                            uint64_t seed, const float* Omega, float* Y,
                            void* ws, size_t ws_bytes, void* stream);

/* Mode-n sketch without a workspace (the paper has no counterpart; this is a
 * deployment variant of rhosvd_sketch).  For callers that cannot allocate
 * device memory where they need the sketch -- code inside another framework's
 * memory pool, plug-ins handed only their input and output buffers, loops
 * where a cudaMalloc and its implicit synchronisation are not allowed.
 * Computes Y = X_(n) Omega exactly like rhosvd_sketch with an explicit Omega
 * (J_n x K, ld J_n; must not be NULL -- there is nowhere to draw it) and Y
 * (I_mode x K, ld I_mode).  The split-K partial sums live in a fixed 4 MiB
 * device array (2^20 floats) that every GPU which loads the library holds
 * until the process exits; the call allocates nothing.  Requests with
 * I_mode * K > 2^20 return RHOSVD_EINVAL before anything is enqueued.
 * The first call on a device looks up that array's device address (a
 * cudaGetSymbolAddress on the current device), so make the first call on each
 * device before any stream capture.  All calls on a device share the one
 * array and each call overwrites it: calls whose work may overlap on the GPU
 * (different streams, no ordering between them) race and give wrong results;
 * order them on one stream or with events. */
rhosvd_status rhosvd_sketch_noalloc(const float* X, const rhosvd_shape* shape, int32_t mode, int32_t K,
                                    const float* Omega, float* Y, void* stream);

/* Every sketch R-PET needs (Alg. 9: factor and core sketches): Y[n] = X_(n) Omega_n
 * (I_n x K[n], ld = I_n) for all n, and, if H is not NULL, the core sketch
 * H = X x_1 Omega~_1 ... x_N Omega~_N (S[0] x ... x S[N-1], column-major) with
 * Omega~_n of size S[n] x I_n (ld = S[n]).  NULL Omega / Omega_tilde arrays
 * (or NULL entries) are drawn from the seed on stream_ids n and N + n. */
rhosvd_status rhosvd_sketch_all(const float* X, const rhosvd_shape* shape, const int32_t* K,
                                const int32_t* S, uint64_t seed,
                                const float* const* Omega, const float* const* Omega_tilde,
                                float* const* Y, float* H, void* ws, size_t ws_bytes, void* stream);

/* One power iteration of Alg. 1 in its stable form (the remark after
 * Alg. 1): on entry Y_inout holds an I_n x K matrix Q with orthonormal
 * columns; the call forms Z = orth(X_(n)^T Q) (J_n x K) and writes the new
 * sketch X_(n) Z into Y_inout (not orthonormalised; call rhosvd_orth). */
rhosvd_status rhosvd_power(const float* X, const rhosvd_shape* shape, int32_t mode, int32_t K,
                           float* Y_inout, void* ws, size_t ws_bytes, void* stream);

/* Thin orthonormalisation Y = QR, Q overwriting Y (the orthonormal basis of Alg. 1).  Y is
 * m x K, leading dimension ld >= m, K <= RHOSVD_MAX_K, m >= K.  Method:
 * CholeskyQR2 (Yamamoto et al. 2015) with an FP64-accurate Gram; if a
 * Cholesky pivot is non-positive or too small, a Householder QR (the LAPACK
 * geqr2/org2r sequence) runs instead.  If fallback_used is not NULL the call
 * synchronises the stream and stores 1 there when the fallback ran. */
rhosvd_status rhosvd_orth(float* Y, int64_t m, int32_t K, int64_t ld, int32_t* fallback_used,
                          void* ws, size_t ws_bytes, void* stream);

/* Core projection G = X x_1 Q_1^T x_2 ... x_N Q_N^T (Eq. "Core"; the core of
 * Alg. 6).  Q[n] is I_n x K[n] with ld = I_n; a NULL Q[n] skips mode n
 * (requires K[n] == I_n, the small-mode remark of Sec. 4).  G is
 * K[0] x ... x K[N-1], column-major. */
rhosvd_status rhosvd_core(const float* X, const rhosvd_shape* shape, const float* const* Q,
                          const int32_t* K, float* G, void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------- driver */

/* Full randomized Tucker decomposition [[G; U_1..U_N]] of X with multilinear
 * rank (R_1..R_N) by the algorithm in opts->algo (Alg. 6 + Alg. 1, Alg. 8, or
 * Alg. 9 with a truncated HOSVD of the recovered core).  U[n] is I_n x R_n
 * (ld = I_n) with orthonormal columns; G is R_1 x ... x R_N column-major.
 * Omega (nullable, or NULL entries) supplies explicit test matrices with the
 * sizes rhosvd_plan reports (J_n x K_n, ld = J_n); missing ones are drawn
 * from opts->seed.  Omega_tilde likewise supplies the R-PET core sketches
 * (S_n x I_n, ld = S_n).  Requires 1 <= R_n <= min(I_n, J_n). */
rhosvd_status rhosvd_decompose(const float* X, const rhosvd_shape* shape, const int32_t* ranks,
                               const rhosvd_opts* opts, const float* const* Omega,
                               const float* const* Omega_tilde, float* const* U, float* G,
                               void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------- fixed accuracy */

/* Workspace bytes rhosvd_decompose_tol needs (0 on invalid input). */
size_t rhosvd_workspace_size_tol(const rhosvd_shape* shape, int32_t block, const int32_t* k_max);

/* Fixed-accuracy R-STHOSVD: Alg. 8 with a fixed-precision range finder in
 * place of Alg. 1 (the rank-revealing randomized algorithms Sec. 5 cites for
 * adaptive use), returning ranks chosen so that ||X - [[G; U]]||_F <= eps ||X||_F.
 * Reading of the tolerance split (Eqs. DT1 / SubPro disagree): every mode gets
 * tol = eps ||X||_F / sqrt(N).  Per mode, on the unfolding A of the current
 * core: blocked randomized QB with an error indicator -- blocks of `block`
 * Gaussian columns (block i of mode n drawn from (seed, stream_id 4096 +
 * 256 n + i)), Y = A Omega_i - Q (B Omega_i), Q_i = orth(Y) re-orthogonalised
 * against Q, B_i = Q_i^T A (FP32 FMA arithmetic, rounded to nearest: the
 * tensor cores' truncating accumulation would leave B ~5e-7 low and E with an
 * error ~1e-6 ||A||^2), E = ||A||^2 - ||P_Q A||^2 (= ||A - Q B||^2), with the
 * projected energy tr((Q^T Q)^-1 B B^T) taken to first order in Q^T Q - I (the
 * FP32 Q is orthonormal to ~1e-6, which the plain sum ||B_i||^2 would carry
 * into E as an error ~1e-6 ||A||^2), until E <= tol^2 (after at least one
 * block) or k_max[n] columns; then R_n = the smallest rank r (>= 1) whose truncated SVD
 * of B keeps E + sum_{i > r} sigma_i^2 <= tol^2, U_n = Q Ubar_r, and the core
 * shrinks to Ubar_r^T B.  U[n] must hold I_n x k_max[n] floats (ld I_n) and G
 * prod k_max[n]; on return ranks[n] (host) holds R_n, U[n] its first R_n
 * columns and G the R_1 x ... x R_N core.  1 <= k_max[n] <= min(I_n, 128),
 * 0 < eps < 1, 1 <= block <= 128.  The ranks depend on the data: the call reads
 * the indicator on the host after every block (it synchronises `stream` that
 * often and returns when the work is done); it cannot be captured in a graph. */
rhosvd_status rhosvd_decompose_tol(const float* X, const rhosvd_shape* shape, double eps, int32_t block,
                                   const int32_t* k_max, uint64_t seed, int32_t* ranks, float* const* U,
                                   float* G, void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------- batches */

/* One tensor of a batch: device pointers owned by the caller. */
typedef struct rhosvd_batch_item {
  const float* X;                     /* I_1 x ... x I_N, column-major (read only) */
  float* G;                           /* R_1 x ... x R_N core, column-major (written) */
  float* U[RHOSVD_MAX_MODES];         /* U[n]: I_n x R_n factor, ld I_n (written) */
  int64_t dims[RHOSVD_MAX_MODES];     /* I_1..I_N, each in 1..256 */
  int32_t ranks[RHOSVD_MAX_MODES];    /* R_1..R_N */
  int32_t N;                          /* number of modes, 1..RHOSVD_MAX_MODES */
} rhosvd_batch_item;

/* Sizes and launch configuration of a batch (filled by rhosvd_batch_plan_create,
 * updated by rhosvd_batch_tune; a plain struct the caller keeps). */
typedef struct rhosvd_batch_plan {
  int32_t n_items, q, p;
  int32_t threads;                    /* threads per CTA: 128, 256 or 512 */
  int32_t jc;                         /* columns of S_(n) per streamed tile: 32 or 64 */
  int32_t ctas_per_sm;                /* persistent CTAs per SM, 1..4 */
  int32_t imax, kmax;                 /* largest mode size and sketch width of the batch */
  int32_t sms, max_ctas;
  uint64_t seed;
  int64_t zb_floats, s_floats;        /* per-CTA scratch: a J x K matrix, two core buffers */
  size_t ws_bytes;                    /* workspace the batch needs */
} rhosvd_batch_plan;

/* Batched R-STHOSVD (Alg. 8 with Alg. 1 per mode, q power iterations,
 * oversampling p) of many independent small tensors in ONE persistent launch:
 * each CTA takes the next tensor from a work queue (largest work first) and
 * decomposes it by itself in FP32 on the CUDA cores -- sketch and TTMs through
 * shared-memory tiles with the test matrices generated in the kernel (the same
 * values as rhosvd_decompose with the same seed: mode n on stream_id n), CGS2
 * for the bases Q, one shifted CholeskyQR pass for the intermediate Z,
 * two-sided Jacobi on B B^T for the truncation.  Restrictions: opts.algo =
 * RHOSVD_ALGO_RSTHOSVD, dtype F32, no refinement or flags, q <= 8, every
 * I_n <= 256 and every sketch width K_n = min(R_n + p, I_n, J_n) <= 32.
 * Accuracy: the truncation's eigenvectors come from the FP32 Gram B B^T, so the
 * subspace error grows as u (sigma_1 / sigma_R)^2 (u = 2^-24); suited to cores
 * with sigma_1 / sigma_R below about 100.
 *
 * rhosvd_batch_plan_create (host only) validates the items and fills `plan`
 * (sizes, a default launch configuration, plan->ws_bytes).
 * rhosvd_batch_upload copies the item table and the work order into `ws`
 * (>= plan->ws_bytes, 256-byte aligned) and waits for `stream`; call it again
 * whenever an item's pointers change.
 * rhosvd_batch_run launches the batch on `stream` (a memset and one kernel;
 * capturable in a CUDA graph, no synchronisation).  Device errors (non-finite
 * values) are recorded in the status block at the start of `ws`.
 * rhosvd_batch_tune runs every launchable configuration (threads x tile
 * columns x CTAs per SM) twice on the uploaded batch, times the second run
 * with CUDA events on `stream` (it synchronises), keeps the fastest in `plan`
 * and returns its time in best_ms (nullable).  The outputs hold a complete
 * decomposition afterwards. */
rhosvd_status rhosvd_batch_plan_create(const rhosvd_batch_item* items, int32_t n_items, const rhosvd_opts* opts,
                                       rhosvd_batch_plan* plan);
rhosvd_status rhosvd_batch_upload(const rhosvd_batch_plan* plan, const rhosvd_batch_item* items, void* ws,
                                  size_t ws_bytes, void* stream);
rhosvd_status rhosvd_batch_run(const rhosvd_batch_plan* plan, void* ws, size_t ws_bytes, void* stream);
rhosvd_status rhosvd_batch_tune(rhosvd_batch_plan* plan, void* ws, size_t ws_bytes, void* stream, float* best_ms);

/* Read the device status word kept at the start of `ws` with a copy ordered
 * on `stream`, wait for that stream (and no other), and return the first error
 * recorded there by earlier calls (RHOSVD_OK if none); `flags` (nullable)
 * receives the RHOSVD_FLAG_* bits.  The word is cleared at the start of every
 * rhosvd_decompose and primitive call. */
rhosvd_status rhosvd_device_status(const void* ws, size_t ws_bytes, void* stream, int32_t* flags);

/* Static description of a status code. */
const char* rhosvd_status_string(rhosvd_status status);

#ifdef __cplusplus
}
#endif

#endif /* RHOSVD_H */
