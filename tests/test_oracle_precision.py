"""What reduced precision costs the randomized decompositions (FP64 oracle, CPU).

* R-STHOSVD on the 512^3 workload with BF16 power iterates: the products of the
  power steps computed on a BF16-rounded copy of the unfolding (round to nearest
  even), first sketch and projection exact.  On mode 1 E stays within 3%
  (measured +2.2%); on every mode it does not; one exact power step after the
  BF16 ones restores E.
* The same workload under the device's FP32 arithmetic: every large product as a
  truncating 3xTF32 split with FP32 accumulation, every orthonormalisation as
  the device's CholeskyQR (one pass for the intermediate bases, two for the
  final one), and the truncation's eigenvectors by the device's route (Cholesky factor of B B^T, then FP32
  one-sided Jacobi that stops once no column cosine exceeds 2e-6).  E stays
  within 0.3% of exact (measured +0.17%; with exact eigenvectors +0.015%, so
  the stopping threshold costs most of it).  A larger excess on the device is
  not arithmetic.
* The same workload with every tensor-core product accumulated toward zero
  instead of to nearest: the core comes out 1.3e-5 short and E rises by about
  2%, the size of the excess measured on the GPU.
* The same workload with both tall Grams of a mode in FP32 (a shifted FP32
  CholeskyQR for the intermediate basis Z, an FP32 B B^T for the truncation):
  E agrees with the exact run to 1e-6 relative.
* R-PET on the 128^4 workload, the single pass reading a BF16 or a per-slice
  e4m3 copy of X: E grows 2x and 25x, with or without an exact core pass.
About twelve minutes of CPU: opt-in with RHOSVD_SLOW=1."""
import numpy as np
import pytest

from oracle import algorithms as A
from oracle import metrics as M
from oracle import tensor as T
from oracle.precision import bf16_round, e4m3_round
from workloads import WORKLOADS, gaussian_matrix


def test_bf16_round_is_correct():
    # the BF16 spacing at 1 is 2^-7
    v = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -3.14159, 1e-30], dtype=np.float32)
    r = bf16_round(v)
    assert r[0] == 1.0
    assert r[1] == 1.0                                  # half a spacing: tie to the even neighbour
    assert r[2] == 1.0 + 2.0 ** -6                      # 1.5 spacings: tie to the even neighbour above
    assert r[3] == 1.0 + 2.0 ** -7                      # 0.75 of a spacing: nearest
    assert r[4] == -3.140625
    assert abs(r[5] / 1e-30 - 1) <= 2.0 ** -8


def _brsvd(a, r, q, omega, bf16_power, exact_refine):
    ab = bf16_round(a) if bf16_power else a
    qm = A.orth(a @ omega)
    for _ in range(q):
        qm = A.orth(ab @ A.orth(ab.T @ qm))
    for _ in range(exact_refine):
        qm = A.orth(a @ A.orth(a.T @ qm))
    b = qm.T @ a
    ubar, _, _ = np.linalg.svd(b, full_matrices=False)
    return qm @ ubar[:, :r], ubar[:, :r].T @ b


def _rsthosvd(x, ranks, q, omegas, bf16_modes=(), exact_refine=0):
    s = x
    us = []
    for n in range(s.ndim):
        u, sn = _brsvd(T.unfold(s, n), ranks[n], q, omegas[n], n in bf16_modes, exact_refine if n in bf16_modes else 0)
        dims = list(s.shape)
        dims[n] = ranks[n]
        s = T.fold(sn, n, dims)
        us.append(u)
    return s, us


@pytest.mark.slow
def test_bf16_power_products_on_mode_one_keep_the_error():
    w = WORKLOADS["decay512_rsthosvd"]
    x = np.asfortranarray(w.tensor().astype(np.float32).astype(np.float64))
    shapes = A.omega_shapes(w.algo, w.dims, w.ranks, w.p)
    omegas = [gaussian_matrix(w.omega_seed + n, r, c).astype(np.float64) for n, (r, c) in enumerate(shapes)]
    e = {}
    for label, kw in [("exact", {}), ("mode1", dict(bf16_modes=(0,))), ("all", dict(bf16_modes=(0, 1, 2))),
                      ("mode1+refine", dict(bf16_modes=(0,), exact_refine=1))]:
        g, us = _rsthosvd(x, w.ranks, w.q, omegas, **kw)
        e[label] = M.rel_error(x, g, us)
    assert e["mode1"] <= 1.03 * e["exact"]
    assert e["all"] > 2 * e["exact"]
    assert abs(e["mode1+refine"] - e["exact"]) <= 1e-3 * e["exact"]


def _trunc_tf32(a):
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    return (u & np.uint32(0xFFFFE000)).view(np.float32)


def _mm3(a, b):
    """3xTF32 product with FP32 accumulation: a_hi b_hi + a_hi b_lo + a_lo b_hi, each
    part truncated to TF32 as the tensor core reads it."""
    a32, b32 = np.ascontiguousarray(a, dtype=np.float32), np.ascontiguousarray(b, dtype=np.float32)
    ah, bh = _trunc_tf32(a32), _trunc_tf32(b32)
    al, bl = _trunc_tf32(a32 - ah), _trunc_tf32(b32 - bh)
    return (ah @ bh + (ah @ bl + al @ bh)).astype(np.float64)


def test_truncating_tf32_split_is_exact_in_its_parts():
    x = np.random.default_rng(0).standard_normal(1000).astype(np.float32)
    hi = _trunc_tf32(x)
    lo = x - hi
    assert np.all(hi + lo == x)                        # the remainder is exact in FP32
    assert np.all(np.abs(lo) < np.abs(x) * 2.0 ** -10)  # and below the TF32 spacing


def _jacobi_columns_f32(l, jtol=2e-6, max_sweeps=30):
    """One-sided Jacobi (Hestenes 1958) on the columns of l in FP32: round-robin
    (circle) pairs, the rotation that zeroes a pair's inner product, and a stop
    once no pair's cosine exceeds jtol in a whole sweep. Returns the columns
    normalised and ordered by decreasing norm, and the number of sweeps."""
    f = np.float32
    x = np.array(l, dtype=f)
    k = x.shape[1]
    n = k + (k & 1)
    w = np.arange(n // 2)
    for sweep in range(max_sweeps):
        norms = np.einsum("ij,ij->j", x, x)
        rotated = False
        for s in range(n - 1):
            a = np.where(w == 0, 0, (w - 1 + s) % (n - 1) + 1)
            b = (n - 2 - w + s) % (n - 1) + 1
            p, q = np.minimum(a, b), np.maximum(a, b)
            p, q = p[q < k], q[q < k]
            gamma = np.einsum("ij,ij->j", x[:, p], x[:, q])
            alpha, beta = norms[p], norms[q]
            hit = (gamma != 0) & (np.abs(gamma) > f(jtol) * np.sqrt(alpha) * np.sqrt(beta))
            if not hit.any():
                continue
            p, q, gamma, alpha, beta = p[hit], q[hit], gamma[hit], alpha[hit], beta[hit]
            zeta = (beta - alpha) / (f(2) * gamma)
            t = np.copysign(f(1) / (np.abs(zeta) + np.sqrt(zeta * zeta + f(1))), zeta).astype(f)
            c = (f(1) / np.sqrt(t * t + f(1))).astype(f)
            sn = c * t
            xp, xq = x[:, p].copy(), x[:, q].copy()
            x[:, p], x[:, q] = c * xp - sn * xq, sn * xp + c * xq
            norms[p], norms[q] = np.maximum(alpha - t * gamma, f(0)), beta + t * gamma
            rotated = True
        if not rotated:
            break
    nc = np.sqrt(np.einsum("ij,ij->j", x, x))
    order = np.argsort(-nc, kind="stable")
    return (x[:, order] / nc[order]).astype(np.float64), sweep + 1


def test_jacobi_columns_gives_the_left_singular_vectors():
    rng = np.random.default_rng(3)
    u0, _ = np.linalg.qr(rng.standard_normal((20, 20)))
    sig = 0.7 ** np.arange(20)
    l = np.linalg.cholesky((u0 * sig ** 2) @ u0.T)     # L L^T = U S^2 U^T: left vectors of L are U
    u, sweeps = _jacobi_columns_f32(l)
    assert sweeps < 30
    assert np.abs(np.abs(np.sum(u[:, :10] * u0[:, :10], axis=0)) - 1).max() < 1e-5
    assert np.abs(u.T @ u - np.eye(20)).max() < 5e-6


def _cholqr_device(y, passes):
    """CholeskyQR as the device runs it: pass 0 from an FP64-accurate Gram and
    Cholesky, pass 1 from an FP32 Gram summed over 64-row tiles and an FP32
    Cholesky; the factor rounded to FP32 and applied in FP32 (a triangular
    solve, or for tall matrices the product with an FP32 R^-1 as a truncating
    3xTF32 GEMM)."""
    from scipy.linalg import solve_triangular
    q = np.asarray(y, dtype=np.float32)
    m, k = q.shape
    for p in range(passes):
        q64 = q.astype(np.float64)
        if p == 0:
            g = q64.T @ q64
        else:
            g = sum((q[i:i + 64].T @ q[i:i + 64]).astype(np.float64) for i in range(0, m, 64))
        lo = (np.linalg.cholesky(g) if p == 0 else np.linalg.cholesky(g.astype(np.float32))).astype(np.float32)
        if m >= 32768:
            rinv = solve_triangular(lo, np.eye(k, dtype=np.float32), lower=True).T.astype(np.float32)
            q = _mm3(q, rinv).astype(np.float32)
        else:
            q = solve_triangular(lo, q.T, lower=True).T.astype(np.float32)
    return q.astype(np.float64)


def _brsvd_device(a, r, q, omega):
    qm = _cholqr_device(_mm3(a, omega), 1 if q > 0 else 2)
    for it in range(q):
        z = _cholqr_device(_mm3(a.T, qm), 1)
        qm = _cholqr_device(_mm3(a, z), 1 if it + 1 < q else 2)
    qm = qm.astype(np.float32).astype(np.float64)
    b = _mm3(qm.T, a)
    ubar = _jacobi_columns_f32(np.linalg.cholesky(b @ b.T))[0][:, :r]
    return _mm3(qm, ubar), _mm3(ubar.T, b)


@pytest.mark.slow
def test_emulated_device_arithmetic_keeps_the_error():
    w = WORKLOADS["decay512_rsthosvd"]
    x = np.asfortranarray(w.tensor().astype(np.float32).astype(np.float64))
    shapes = A.omega_shapes(w.algo, w.dims, w.ranks, w.p)
    omegas = [gaussian_matrix(w.omega_seed + n, r, c).astype(np.float64) for n, (r, c) in enumerate(shapes)]
    g, us = _rsthosvd(x, w.ranks, w.q, omegas)
    e_exact = M.rel_error(x, g, us)
    s, us = x, []
    for n in range(3):
        u, sn = _brsvd_device(T.unfold(s, n), w.ranks[n], w.q, omegas[n])
        dims = list(s.shape)
        dims[n] = w.ranks[n]
        s = T.fold(sn, n, dims)
        us.append(u)
    e_dev = M.rel_error(x, s, us)
    print(f"E exact {e_exact:.6e}, emulated device {e_dev:.6e} ({e_dev / e_exact - 1:+.3%}), "
          f"factors orthonormal to {max(M.orthonormality(u) for u in us):.1e}")
    assert e_dev <= 1.003 * e_exact


def _shifted_cholqr_range(z, c):
    """One CholeskyQR pass from an FP32 Gram with a diagonal shift c u tr(G):
    the shift keeps the Cholesky from breaking down at any condition number,
    and the result keeps range(Z) (R is invertible), which is all an
    intermediate basis of the power iteration needs."""
    z32 = np.asarray(z, dtype=np.float32)
    g = (z32.T @ z32).astype(np.float64)
    r = np.linalg.cholesky(g + c * 2.0 ** -24 * np.trace(g) * np.eye(g.shape[0])).T.astype(np.float32)
    return np.linalg.solve(r.T.astype(np.float64), z32.T.astype(np.float64)).T.astype(np.float32).astype(np.float64)


@pytest.mark.slow
def test_fp32_grams_keep_the_error():
    """The 512^3 workload with the two tall Grams of a mode in FP32 instead of
    FP64-accurate: the intermediate basis Z by a shifted FP32 CholeskyQR, and the
    truncation's B B^T accumulated in FP32. E agrees with the exact run to
    1e-6 relative, so both Grams could run at FP32 speed on this workload.
    (The truncation Gram still needs FP64 accuracy when lambda_R / lambda_1
    approaches the FP32 unit roundoff.)"""
    w = WORKLOADS["decay512_rsthosvd"]
    x = np.asfortranarray(w.tensor().astype(np.float32).astype(np.float64))
    shapes = A.omega_shapes(w.algo, w.dims, w.ranks, w.p)
    omegas = [gaussian_matrix(w.omega_seed + n, r, c).astype(np.float64) for n, (r, c) in enumerate(shapes)]
    e = {}
    for label in ("exact", "fp32"):
        s, us = x, []
        for n in range(3):
            a = T.unfold(s, n)
            qm = A.orth(a @ omegas[n])
            for _ in range(w.q):
                z = a.T @ qm
                qm = A.orth(a @ (A.orth(z) if label == "exact" else _shifted_cholqr_range(z, 100.0)))
            b = qm.T @ a
            if label == "exact":
                g = b @ b.T
            else:
                b32 = b.astype(np.float32)
                g = (b32 @ b32.T).astype(np.float64)
            ub = np.linalg.eigh(g)[1][:, ::-1][:, :w.ranks[n]]
            dims = list(s.shape)
            dims[n] = w.ranks[n]
            s = T.fold(ub.T @ b, n, dims)
            us.append(qm @ ub)
        e[label] = M.rel_error(x, s, us)
    print(f"E exact {e['exact']:.7e}, with FP32 Grams {e['fp32']:.7e}")
    assert abs(e["fp32"] - e["exact"]) <= 1e-6 * e["exact"]


def _rz32(s):
    """Round FP64 values to FP32 toward zero."""
    f = s.astype(np.float32)
    over = np.abs(f.astype(np.float64)) > np.abs(s)
    f[over] = np.nextafter(f[over], np.float32(0))
    return f


def _mm3_rz(a, b, splits=1):
    """The 3xTF32 product as an accumulator that rounds toward zero: per K step of
    8, the parts hi*hi, hi*lo and lo*hi are each added to an FP32 accumulator with
    round-toward-zero (each 8-term partial exact); the K range is cut into
    `splits` contiguous parts, summed exactly (the split-K reduction)."""
    a32, b32 = np.asarray(a, np.float32), np.asarray(b, np.float32)
    ah, bh = _trunc_tf32(a32), _trunc_tf32(b32)
    al, bl = _trunc_tf32(a32 - ah), _trunc_tf32(b32 - bh)
    k = a32.shape[1]
    total = np.zeros((a32.shape[0], b32.shape[1]))
    bounds = np.linspace(0, k, splits + 1).astype(int)
    for s0, s1 in zip(bounds[:-1], bounds[1:]):
        acc = np.zeros_like(total, dtype=np.float32)
        for c in range(s0, s1, 8):
            c1 = min(c + 8, s1)
            for x, y in ((ah, bh), (ah, bl), (al, bh)):
                acc = _rz32(acc.astype(np.float64) + x[:, c:c1].astype(np.float64) @ y[c:c1].astype(np.float64))
        total += acc
    return total


@pytest.mark.slow
def test_round_toward_zero_accumulation_reproduces_the_excess():
    """The device path of the 512^3 workload with every tensor-core product
    accumulated toward zero (the rest as in the device emulation above): the core
    comes out about 1.3e-5 short of X x_n U_n^T, and E rises by about 2%, close to
    the excess measured on the GPU, while the subspaces and orthonormality stay
    at the round-to-nearest figures.  Whether tcgen05 accumulates this way is
    what test_tensor_core_accumulation_is_unbiased measures on the GPU."""
    w = WORKLOADS["decay512_rsthosvd"]
    x = np.asfortranarray(w.tensor().astype(np.float32).astype(np.float64))
    shapes = A.omega_shapes(w.algo, w.dims, w.ranks, w.p)
    omegas = [gaussian_matrix(w.omega_seed + n, r, c).astype(np.float64) for n, (r, c) in enumerate(shapes)]
    g0, us0 = _rsthosvd(x, w.ranks, w.q, omegas)
    e0 = M.rel_error(x, g0, us0)
    s, us = x, []
    for n in range(3):
        a = T.unfold(s, n)
        sp = max(1, min(152, a.shape[1] // 16))           # the sketch's split over CTAs
        qm = _cholqr_device(_mm3_rz(a, omegas[n], sp), 1)
        z = _cholqr_device(_mm3_rz(a.T, qm), 1)
        qm = _cholqr_device(_mm3_rz(a, z, sp), 2)
        b = _mm3_rz(qm.T, a)
        ub = _jacobi_columns_f32(np.linalg.cholesky(b @ b.T))[0][:, :w.ranks[n]]
        dims = list(s.shape)
        dims[n] = w.ranks[n]
        s = T.fold(_mm3_rz(ub.T, b), n, dims)
        us.append(_mm3_rz(qm, ub))
    e = M.rel_error(x, s, us)
    g_t = T.multi_ttm(x, us, transpose=True)
    scale = float(np.sum(s * g_t) / np.sum(g_t * g_t) - 1)
    print(f"E {e / e0 - 1:+.3%} over exact, core scale - 1 {scale:+.2e}")
    assert 0.01 < e / e0 - 1 < 0.04
    assert -3e-5 < scale < -5e-6


def test_e4m3_round_is_correct():
    v = np.array([1.0, 1.0625, 1.1875, 3.3, 448.0, 500.0, 2.0 ** -9, 3 * 2.0 ** -10, -0.3])
    r = e4m3_round(v)
    assert r[0] == 1.0
    assert r[1] == 1.0                 # halfway between 1 and 1.125: tie to even
    assert r[2] == 1.25                # halfway between 1.125 and 1.25: tie to even
    assert r[3] == 3.25                # spacing 0.25 in [2, 4)
    assert r[4] == 448.0 and r[5] == 448.0
    assert r[6] == 2.0 ** -9           # smallest subnormal
    assert r[7] == 2.0 ** -8           # 1.5 subnormal spacings: tie to even (2)
    assert r[8] == -0.3125             # spacing 2^-5 in [0.25, 0.5)


def _per_slice(x, fn):
    out = np.empty_like(x)
    for k in range(x.shape[-1]):
        sl = x[..., k]
        sc = 448.0 / np.abs(sl).max()
        out[..., k] = fn(sl * sc) / sc
    return out


@pytest.mark.slow
def test_reduced_precision_single_pass_loses_accuracy():
    """R-PET on the 128^4 workload (noise 1e-3) with the single pass reading a BF16
    or a per-slice-scaled e4m3 copy of X: the quantisation noise (1.7e-3 and
    2.7e-2 relative) exceeds the data's, and E grows 2x and 25x; an exact FP32
    core pass over the found factors does not bring it back."""
    w = WORKLOADS["lowrank128x4_rpet"]
    x = np.asfortranarray(w.tensor().astype(np.float32).astype(np.float64))
    n_modes = x.ndim
    om = [gaussian_matrix(w.omega_seed + n, int(np.prod(w.dims)) // w.dims[n], w.K[n]).astype(np.float64)
          for n in range(n_modes)]
    ot = [gaussian_matrix(w.omega_seed + 100 + n, w.S[n], w.dims[n]).astype(np.float64) for n in range(n_modes)]
    e = {}
    for label, xq in [("fp32", x), ("bf16", bf16_round(x).reshape(x.shape, order="A")),
                      ("e4m3", _per_slice(x, e4m3_round))]:
        g, us, _ = A.rpet(np.asfortranarray(xq), w.ranks, om, ot)
        e[label] = M.rel_error(x, g, us)
        e[label + "+core"] = M.rel_error(x, T.multi_ttm(x, us, transpose=True), us)
    assert e["bf16"] > 1.5 * e["fp32"] and e["bf16+core"] > 1.5 * e["fp32+core"]
    assert e["e4m3"] > 10 * e["fp32"] and e["e4m3+core"] > 10 * e["fp32+core"]
