"""Deterministic and randomized Tucker algorithms of Secs. 3-5, plain FP64.

Each function follows the paper's steps in its order and notation; dense
linear algebra is delegated to NumPy/LAPACK (QR = Householder, SVD = gesdd).
Random test matrices are inputs (explicit arrays), never drawn here, so the
GPU path and this oracle can be run on identical Omegas.

Readings taken where the paper is silent or garbled:
* sketch width K_n = min(R_n + p, I_n, J_n) with J_n the number of columns of
  the unfolding being sketched (oversampling of Remark 1 applied to Alg. 6);
* the power iteration of Alg. 1 is evaluated as subspace iteration with
  an orthonormalisation after every product (the stability note after Alg. 1):
  Z = orth(A^T Q), Q = orth(A Z), q times;
* Alg. 8 starts from S = X (it prints S = X_(n));
* the final truncation of R-PET is a truncated HOSVD of the small recovered core,
  whose factors are lifted through Q_n;
* fixed accuracy: the tolerance eps is relative and split evenly over the modes,
  tol = eps ||X||_F / sqrt(N) per mode (Eqs. DT1 and SubPro disagree on the
  split), which bounds the ST-HOSVD error by eps ||X||_F.
"""
from __future__ import annotations

from typing import Callable, Sequence

import numpy as np

from .tensor import fold, multi_ttm, ttm, unfold


def orth(y: np.ndarray) -> np.ndarray:
    """Orthonormal basis of range(Y) from the economic QR Y = QR (Sec. 3.1)."""
    q, _ = np.linalg.qr(np.asarray(y, dtype=np.float64), mode="reduced")
    return q


def sketch_width(r: int, p: int, i_n: int, j_n: int) -> int:
    """K_n = min(R_n + p, I_n, J_n)."""
    return int(min(r + p, i_n, j_n))


def brsvd(a: np.ndarray, r: int, q: int, omega: np.ndarray, return_q: bool = False):
    """Algorithm 1 (basic randomized SVD with oversampling and power iteration).

    a      I x J data matrix
    r      target rank R
    q      number of power iterations
    omega  J x K Gaussian test matrix, K = R + p (drawn by the caller)

    Returns U = Q Ubar(:, 1:R) (I x R) and Ubar(:, 1:R)^T B = S V^T (R x J),
    the latter being the projected unfolding used by STHOSVD (the shortcut
    stated after Alg. 4).
    """
    a = np.asarray(a, dtype=np.float64)
    y = a @ np.asarray(omega, dtype=np.float64)          # sketch A Omega
    qm = orth(y)                                         # its orthonormal basis
    for _ in range(q):                                   # power iteration, (A A^T)^q A Omega
        z = orth(a.T @ qm)
        qm = orth(a @ z)
    b = qm.T @ a                                         # projection B = Q^T A
    ubar, _, _ = np.linalg.svd(b, full_matrices=False)   # SVD of the small B
    ubar_r = ubar[:, :r]
    u = qm @ ubar_r                                      # lift: U = Q Ubar_R
    out = (u, ubar_r.T @ b)
    if return_q:
        out = out + (qm,)
    return out


def leading_left_singular_vectors(a: np.ndarray, r: int) -> np.ndarray:
    """Leading r left singular vectors of A (LAPACK SVD).  For a very wide A the
    SVD is taken of the triangular factor of A^T = Q R (A = R^T Q^T has the same
    left singular vectors), which avoids forming the huge right factor."""
    a = np.asarray(a, dtype=np.float64)
    if a.shape[1] > 8 * a.shape[0]:
        a = np.linalg.qr(a.T, mode="r").T
    u, _, _ = np.linalg.svd(a, full_matrices=False)
    return u[:, :r]


def thosvd(x: np.ndarray, ranks: Sequence[int]):
    """Truncated HOSVD (Sec. 4): Q^(n) = leading R_n left singular vectors of X_(n),
    S = X x_1 Q^(1)T ... x_N Q^(N)T (Eq. "Core")."""
    us = [leading_left_singular_vectors(unfold(x, n), ranks[n]) for n in range(x.ndim)]
    return multi_ttm(x, us, transpose=True), us


def sthosvd(x: np.ndarray, ranks: Sequence[int]):
    """Algorithm 4 (STHOSVD), fixed-rank form, ascending mode order."""
    s = np.asarray(x, dtype=np.float64)
    us = []
    for n in range(s.ndim):
        u = leading_left_singular_vectors(unfold(s, n), ranks[n])   # factor of the current core
        s = ttm(s, u.T, n)                                           # shrink mode n
        us.append(u)
    return s, us


def hooi_sweep(x: np.ndarray, us: Sequence[np.ndarray], ranks: Sequence[int]):
    """One outer iteration of Algorithm 5 (HOOI): for each n in turn,
    Z = X x_{p != n} Q^(p)T with the latest factors, Q^(n) = leading R_n left
    singular vectors of Z_(n); then S = X x_1 Q^(1)T ... x_N Q^(N)T."""
    us = list(us)
    for n in range(x.ndim):
        mats = [None if p == n else us[p].T for p in range(x.ndim)]
        z = multi_ttm(x, mats)
        us[n] = leading_left_singular_vectors(unfold(z, n), ranks[n])
    return multi_ttm(x, us, transpose=True), us


def hooi(x: np.ndarray, ranks: Sequence[int], sweeps: int = 20):
    """HOOI initialised by the truncated HOSVD (Alg. 5), a fixed number of sweeps."""
    _, us = thosvd(x, ranks)
    g = None
    for _ in range(sweeps):
        g, us = hooi_sweep(x, us, ranks)
    return g, us


def rp_hooi_sweep(x: np.ndarray, us: Sequence[np.ndarray], ranks: Sequence[int],
                  omegas: Sequence[np.ndarray]):
    """One sweep of Algorithm 7 (RP-HOOI), in its order: for each n in turn,
    S = X x_{p != n} Q^(p)T with the latest factors, and Q^(n) from a random
    projection of S_(n).  The factor step is Algorithm 1 with q = 0: the sketch
    S_(n) Omega^(n) with K_n = min(R_n + p, I_n, J_n) columns, its orthonormal
    basis, and the truncation to R_n through the SVD of the projected matrix
    (the oversampling reading taken for Alg. 6 as well).  omegas[n] is
    J_n x K_n with J_n = prod_{p != n} R_p.  The core is the last S times
    Q^(N)T, i.e. X x_1 Q^(1)T ... x_N Q^(N)T with the new factors.
    Used as the refinement sweep after a single-pass or reduced-precision run."""
    x = np.asarray(x, dtype=np.float64)
    us = [np.asarray(u, dtype=np.float64) for u in us]
    s = x
    for n in range(x.ndim):
        mats = [None if k == n else us[k].T for k in range(x.ndim)]
        s = multi_ttm(x, mats)
        us[n] = brsvd(unfold(s, n), ranks[n], 0, omegas[n])[0]
    return ttm(s, us[-1].T, x.ndim - 1), us


def rp_hooi_omega_shapes(dims: Sequence[int], ranks: Sequence[int], p: int):
    """Sizes (J_n, K_n) of the test matrices of one RP-HOOI sweep: J_n = prod_{k != n} R_k."""
    shapes = []
    for n in range(len(dims)):
        j_n = int(np.prod([int(ranks[k]) for k in range(len(dims)) if k != n], dtype=np.int64))
        shapes.append((j_n, sketch_width(int(ranks[n]), p, int(dims[n]), j_n)))
    return shapes


def rhosvd(x: np.ndarray, ranks: Sequence[int], q: int, omegas: Sequence[np.ndarray]):
    """Algorithm 6 (RP-HOSVD) with each factor from Algorithm 1 on the original X:
    Q^(n) from X_(n) Omega^(n) (J_n = prod_{k != n} I_k rows), then
    S = X x_1 Q^(1)T ... x_N Q^(N)T."""
    us = [brsvd(unfold(x, n), ranks[n], q, omegas[n])[0] for n in range(x.ndim)]
    return multi_ttm(x, us, transpose=True), us


def rsthosvd(x: np.ndarray, ranks: Sequence[int], q: int, omegas: Sequence[np.ndarray]):
    """Algorithm 8 (R-STHOSVD): S = X; for n = 1..N apply Alg. 1 to S_(n) with target
    rank R_n (Omega^(n) has prod_{k<n} R_k prod_{k>n} I_k rows) and set
    S = S x_n Q^(n)T, i.e. S_(n) = Ubar_R^T B."""
    s = np.asarray(x, dtype=np.float64)
    us = []
    for n in range(s.ndim):
        u, sn = brsvd(unfold(s, n), ranks[n], q, omegas[n])
        dims = list(s.shape)
        dims[n] = ranks[n]
        s = fold(sn, n, dims)
        us.append(u)
    return s, us


def randqb_ei(a: np.ndarray, tol: float, block: int, k_max: int, omega_block: Callable[[int, int, int], np.ndarray],
              q: int = 0):
    """Fixed-precision range finder (the blocked randomized QB with an error
    indicator that Secs. 3 and 5 cite for rank-revealing, "fixed-precision"
    randomized algorithms).

    The basis grows by blocks of `block` columns.  Block i starts from the
    Gaussian test block omega_block(i, J, b) (J x b, an input like every test
    matrix here): Y = A Omega_i - Q (B Omega_i) is the part of A Omega_i outside
    the current basis, optionally refined by q subspace-iteration steps against
    the same deflated operator, then orthonormalised and orthogonalised once
    more against Q.  With B_i = Q_i^T A appended to B, the indicator
    E = ||A||_F^2 - sum_i ||B_i||_F^2 equals ||A - Q B||_F^2 = ||(I - Q Q^T) A||_F^2
    (Q orthonormal, B = Q^T A).  The loop stops once E <= tol^2 or Q holds k_max
    columns.  Returns Q (I x K), B (K x J) and the list of indicator values after
    each block."""
    a = np.asarray(a, dtype=np.float64)
    m, j = a.shape
    k_max = int(min(k_max, m, j))
    qm = np.zeros((m, 0))
    bm = np.zeros((0, j))
    e = float(np.sum(a * a))
    history = []
    i = 0
    while e > tol * tol and qm.shape[1] < k_max:
        b = int(min(block, k_max - qm.shape[1]))
        om = np.asarray(omega_block(i, j, b), dtype=np.float64)
        y = a @ om - qm @ (bm @ om)
        for _ in range(q):                                  # power steps on (I - QQ^T) A = A - Q B
            w = orth(y)
            z = orth(a.T @ w - bm.T @ (qm.T @ w))
            y = a @ z - qm @ (bm @ z)
        qi = orth(y)
        qi = orth(qi - qm @ (qm.T @ qi))                    # re-orthogonalisation
        bi = qi.T @ a
        qm = np.hstack([qm, qi])
        bm = np.vstack([bm, bi])
        e = e - float(np.sum(bi * bi))
        history.append(e)
        i += 1
    return qm, bm, history


def truncation_rank(sigma: np.ndarray, residual: float, tol: float) -> int:
    """Smallest r with residual + sum_{i > r} sigma_i^2 <= tol^2 (sigma descending):
    the rank-revealing truncation of B = Ubar Sigma Vbar^T after a QB step."""
    tail = np.concatenate([np.cumsum((sigma ** 2)[::-1])[::-1], [0.0]])   # tail[r] = sum_{i >= r} sigma_i^2
    for r in range(len(sigma) + 1):
        if residual + tail[r] <= tol * tol:
            return r
    return len(sigma)


def rsthosvd_fixed_accuracy(x: np.ndarray, eps: float, block: int, k_max: Sequence[int],
                            omega_block: Callable[[int, int, int, int], np.ndarray], q: int = 0):
    """R-STHOSVD with fixed accuracy (Alg. 8 with the fixed-precision range finder
    in place of Alg. 1, as Sec. 5 suggests).  Reading of the garbled tolerance
    split (Eqs. DT1 and SubPro): each mode gets tol = eps ||X||_F / sqrt(N), so
    that the sequential-truncation error identity gives
    ||X - X_hat||_F <= eps ||X||_F.  For mode n: S_(n) -> (Q, B, E) by
    randqb_ei, B = Ubar Sigma Vbar^T, R_n = truncation_rank(Sigma, E, tol),
    U^(n) = Q Ubar_R, S_(n) <- Ubar_R^T B.  omega_block(n, i, J, b) is block i of
    mode n.  Returns the core, the factors and the ranks."""
    s = np.asarray(x, dtype=np.float64)
    n_modes = s.ndim
    tol = eps * float(np.linalg.norm(s)) / np.sqrt(n_modes)
    us, ranks = [], []
    for n in range(n_modes):
        a = unfold(s, n)
        qm, bm, hist = randqb_ei(a, tol, block, k_max[n], lambda i, j, b, n=n: omega_block(n, i, j, b), q=q)
        e = hist[-1] if hist else float(np.sum(a * a))
        if qm.shape[1] == 0:                                # the whole mode fits the tolerance at rank 0
            r = 0
            ubar = np.zeros((0, 0))
        else:
            ubar, sig, _ = np.linalg.svd(bm, full_matrices=False)
            r = truncation_rank(sig, max(e, 0.0), tol)
        u = qm @ ubar[:, :r] if r > 0 else np.zeros((a.shape[0], 0))
        if r > 0:
            # sign convention: each factor column's largest-magnitude entry positive
            # (factors are defined up to column signs; the later modes sketch the core
            # in this mode's coordinates, so the convention fixes their test matrices)
            flip = np.where(u[np.argmax(np.abs(u), axis=0), np.arange(r)] < 0, -1.0, 1.0)
            u = u * flip
            ubar = ubar[:, :r] * flip
        sn = ubar[:, :r].T @ bm if r > 0 else np.zeros((0, a.shape[1]))
        dims = list(s.shape)
        dims[n] = r
        s = fold(sn, n, dims)
        us.append(u)
        ranks.append(r)
    return s, us, ranks


def pinv_lstsq(a: np.ndarray) -> np.ndarray:
    """Moore-Penrose pseudo-inverse of a full-column-rank A by least squares."""
    a = np.asarray(a, dtype=np.float64)
    sol, *_ = np.linalg.lstsq(a, np.eye(a.shape[0]), rcond=None)
    return sol


def rpet(x: np.ndarray, ranks: Sequence[int], omegas: Sequence[np.ndarray],
         omegas_tilde: Sequence[np.ndarray]):
    """Algorithm 9 (R-PET, single pass over X).

    omegas[n]        J_n x K_n factor sketch matrices (J_n = prod_{k != n} I_k)
    omegas_tilde[n]  S_n x I_n core sketch matrices, R_n <= K_n <= S_n
    Steps: Y_n = X_(n) Omega_n; Q^(n) = QR(Y_n); H = X x_1 Omega~_1 ... x_N Omega~_N;
    S = H x_1 (Omega~_1 Q^(1))^+ ... x_N (Omega~_N Q^(N))^+; truncate with a
    truncated HOSVD of S: S ~ G x_n V_n, U_n = Q^(n) V_n.
    Returns (G, U, extras) with extras holding Y, Q, H and the untruncated core.
    """
    x = np.asarray(x, dtype=np.float64)
    ys = [unfold(x, n) @ np.asarray(omegas[n], dtype=np.float64) for n in range(x.ndim)]
    qs = [orth(y) for y in ys]
    h = multi_ttm(x, [np.asarray(o, dtype=np.float64) for o in omegas_tilde])
    c = multi_ttm(h, [pinv_lstsq(np.asarray(omegas_tilde[n], np.float64) @ qs[n])
                      for n in range(x.ndim)])
    g, vs = thosvd(c, ranks)
    us = [qs[n] @ vs[n] for n in range(x.ndim)]
    return g, us, {"Y": ys, "Q": qs, "H": h, "C": c}


def kronecker_test_matrix(phis: Sequence[np.ndarray], n: int) -> np.ndarray:
    """The structured test matrix of the memory-efficient sketch of Sec. 5.1:
    Omega_n = Phi_N kron ... kron Phi_1 with Phi_n left out, in the reversed order
    of the unfolding (Eq. "TuckerUnfold"), so that X_(n) Omega_n equals the
    n-unfolding of X x_{p != n} Phi_p^T.  phis[p] is I_p x k_p."""
    m = np.ones((1, 1))
    for p in reversed(range(len(phis))):
        if p != n:
            m = np.kron(m, np.asarray(phis[p], dtype=np.float64))
    return m


def omega_shapes(algo: str, dims: Sequence[int], ranks: Sequence[int], p: int,
                 K: Sequence[int] | None = None, S: Sequence[int] | None = None):
    """Sizes (rows, cols) of the Gaussian test matrices each algorithm consumes.

    rhosvd / rpet: J_n = prod_{k != n} I_k rows; rsthosvd: prod_{k<n} R_k prod_{k>n} I_k.
    rpet also returns the core sketch sizes (S_n, I_n)."""
    dims = [int(d) for d in dims]
    ranks = [int(r) for r in ranks]
    nmodes = len(dims)
    shapes = []
    cur = list(dims)
    for n in range(nmodes):
        j_n = int(np.prod([cur[k] for k in range(nmodes) if k != n], dtype=np.int64))
        k_n = int(K[n]) if K is not None else sketch_width(ranks[n], p, dims[n], j_n)
        shapes.append((j_n, k_n))
        if algo == "rsthosvd":
            cur[n] = ranks[n]
    if algo == "rpet":
        tilde = [(int(S[n]) if S is not None else 2 * shapes[n][1] + 1, dims[n]) for n in range(nmodes)]
        return shapes, tilde
    return shapes
