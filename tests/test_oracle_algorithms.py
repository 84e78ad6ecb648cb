"""Pins for the oracle's algorithms (Secs. 3-5) against closed forms, invariants,
special cases that reduce to LAPACK, exact recovery and the paper's bounds."""
import math

import numpy as np
import pytest

from oracle import algorithms as A
from oracle import metrics as M
from oracle import tensor as T
from workloads import gaussian_matrix, lowrank_tensor, random_tensor


def _omegas(algo, dims, ranks, p, seed=0, K=None, S=None):
    shapes = A.omega_shapes(algo, dims, ranks, p, K=K, S=S)
    if algo == "rpet":
        fs, ts = shapes
        om = [gaussian_matrix(seed + n, r, c).astype(np.float64) for n, (r, c) in enumerate(fs)]
        ot = [gaussian_matrix(seed + 100 + n, r, c).astype(np.float64) for n, (r, c) in enumerate(ts)]
        return om, ot
    return [gaussian_matrix(seed + n, r, c).astype(np.float64) for n, (r, c) in enumerate(shapes)]


# ----------------------------------------------------------------------------- orth / Alg. 1

def test_orth_is_orthonormal_and_spans():
    y = np.random.default_rng(0).standard_normal((50, 7))
    q = A.orth(y)
    assert M.orthonormality(q) < 1e-14
    np.testing.assert_allclose(q @ (q.T @ y), y, atol=1e-13)


def test_orth_rank_deficient_still_orthonormal():
    rng = np.random.default_rng(1)
    y = rng.standard_normal((40, 3)) @ rng.standard_normal((3, 6))
    q = A.orth(y)
    assert q.shape == (40, 6) and M.orthonormality(q) < 1e-13
    np.testing.assert_allclose(q @ (q.T @ y), y, atol=1e-12)


def _decaying_matrix(m, n, seed, decay=0.7):
    rng = np.random.default_rng(seed)
    u, _ = np.linalg.qr(rng.standard_normal((m, min(m, n))))
    v, _ = np.linalg.qr(rng.standard_normal((n, min(m, n))))
    s = decay ** np.arange(min(m, n))
    return (u * s) @ v.T, s


@pytest.mark.parametrize("q", [1, 2])
def test_power_iteration_spans_explicit_power(q):
    """Power iteration of Alg. 1: range(Q) = range((A A^T)^q A Omega) (Remark 1 closed form)."""
    a, _ = _decaying_matrix(60, 40, 2, decay=0.9)
    om = np.random.default_rng(3).standard_normal((40, 8))
    _, _, qm = A.brsvd(a, 5, q, om, return_q=True)
    y = a @ om
    for _ in range(q):
        y = a @ (a.T @ y)
    assert M.max_principal_sine(qm, y) < 1e-8


def test_power_iteration_spectrum_identity():
    """(A A^T)^q A = U S^(2q+1) V^T (Remark 1)."""
    a, s = _decaying_matrix(30, 20, 4, decay=0.8)
    u, sv, vt = np.linalg.svd(a, full_matrices=False)
    lhs = a @ a.T @ a @ a.T @ a
    np.testing.assert_allclose(lhs, (u * sv ** 5) @ vt, atol=1e-12)


def test_brsvd_recovers_exact_low_rank():
    rng = np.random.default_rng(5)
    a = rng.standard_normal((80, 6)) @ rng.standard_normal((6, 120))
    u, sv = A.brsvd(a, 6, 0, rng.standard_normal((120, 9)))
    np.testing.assert_allclose(u @ sv, a, atol=1e-11 * np.abs(a).max())
    assert M.orthonormality(u) < 1e-13


@pytest.mark.parametrize("q", [0, 1])
def test_halko_expected_error_bound(q):
    """E||A - QQ^T A||_2 <= (1 + sqrt(R/(P-1)) + e sqrt(R+P)/P sqrt(min(I,J)-R))^(1/(2q+1)) sigma_{R+1}
    (the bound quoted after Alg. 1 with k = R), averaged over 40 Gaussian draws."""
    a, s = _decaying_matrix(120, 90, 6, decay=0.85)
    r, p = 8, 5
    bound = (1 + math.sqrt(r / (p - 1)) + math.e * math.sqrt(r + p) / p * math.sqrt(min(a.shape) - r)) \
        ** (1.0 / (2 * q + 1)) * s[r]
    errs = []
    for t in range(40):
        om = np.random.default_rng(100 + t).standard_normal((90, r + p))
        _, _, qm = A.brsvd(a, r, q, om, return_q=True)
        errs.append(np.linalg.norm(a - qm @ (qm.T @ a), 2))
    assert np.mean(errs) <= bound
    # Q has R+P columns, so no draw beats the optimal rank-(R+P) error sigma_{R+P+1}
    assert min(errs) >= s[r + p] * (1 - 1e-12)


# ----------------------------------------------------------------------------- deterministic Tucker

def test_thosvd_core_all_orthogonal_and_pseudo_diagonal():
    """Full-rank HOSVD core: mode-n slices mutually orthogonal, slice norms = sigma_i(X_(n)),
    non-increasing (Sec. 4)."""
    x = random_tensor((5, 6, 7), 11)
    g, us = A.thosvd(x, (5, 6, 7))
    for n in range(3):
        gram = T.unfold(g, n) @ T.unfold(g, n).T
        sv = np.linalg.svd(T.unfold(x, n), compute_uv=False)
        np.testing.assert_allclose(np.diag(gram), sv ** 2, rtol=1e-12)
        off = gram - np.diag(np.diag(gram))
        assert np.max(np.abs(off)) < 1e-12 * sv[0] ** 2
        assert np.all(np.diff(np.diag(gram)) <= 1e-12)
    np.testing.assert_allclose(T.reconstruct(g, us), x, atol=1e-12)


def test_sthosvd_shortcut_lambda_vt():
    """S x_n Q^(n)T has unfolding Lambda V^T (the remark before Alg. 4)."""
    x = random_tensor((6, 7, 8), 12)
    ranks = (3, 4, 5)
    s = x
    for n in range(3):
        u, sv, vt = np.linalg.svd(T.unfold(s, n), full_matrices=False)
        proj = T.ttm(s, u[:, :ranks[n]].T, n)
        np.testing.assert_allclose(T.unfold(proj, n), sv[:ranks[n], None] * vt[:ranks[n]], atol=1e-12)
        s = proj
    g, _ = A.sthosvd(x, ranks)
    np.testing.assert_allclose(np.abs(g), np.abs(s), atol=1e-12)


def test_quasi_optimality_and_hooi_monotone():
    """||X - X_THOSVD|| <= sqrt(N) ||X - X_best|| <= sqrt(N) ||X - X_HOOI|| (Sec. 4), and
    HOOI does not increase the error of its HOSVD start."""
    x = lowrank_tensor((12, 13, 14), (4, 4, 4), 13, noise=0.3)
    ranks = (3, 3, 3)
    g_t, u_t = A.thosvd(x, ranks)
    g_s, u_s = A.sthosvd(x, ranks)
    g_h, u_h = A.hooi(x, ranks, sweeps=30)
    e_t, e_s, e_h = (M.rel_error(x, g, u) for g, u in ((g_t, u_t), (g_s, u_s), (g_h, u_h)))
    assert e_h <= e_t + 1e-14
    assert e_t <= math.sqrt(3) * e_h
    assert e_s <= math.sqrt(3) * e_h


# ----------------------------------------------------------------------------- randomized Tucker

@pytest.mark.parametrize("algo", ["rhosvd", "rsthosvd", "rpet"])
@pytest.mark.parametrize("q", [0, 1])
def test_exact_recovery_noise_free(algo, q):
    """Noise-free tensor of exact multilinear rank, K >= R: relative error <= 1e-12
    (the noiseless row of Table 1 reports ~1e-13..1e-12)."""
    dims, ranks = (30, 40, 50), (4, 5, 6)
    x = lowrank_tensor(dims, ranks, 14, noise=0.0, factors="gaussian")
    if algo == "rpet":
        K = tuple(r + 2 for r in ranks)
        S = tuple(2 * k + 1 for k in K)
        om, ot = _omegas("rpet", dims, ranks, 2, K=K, S=S)
        g, us, _ = A.rpet(x, ranks, om, ot)
    else:
        om = _omegas(algo, dims, ranks, 3)
        g, us = getattr(A, algo)(x, ranks, q, om)
    assert M.rel_error(x, g, us) <= 1e-12
    for u in us:
        assert M.orthonormality(u) < 1e-13


def test_exact_recovery_four_way():
    dims, ranks = (9, 10, 11, 12), (2, 3, 3, 4)
    x = lowrank_tensor(dims, ranks, 15, noise=0.0, factors="gaussian")
    for algo in ("rhosvd", "rsthosvd"):
        g, us = getattr(A, algo)(x, ranks, 1, _omegas(algo, dims, ranks, 2))
        assert M.rel_error(x, g, us) <= 1e-12


def test_exact_recovery_eight_way():
    """The largest order the library accepts (8 modes), including modes kept
    whole (R_n = I_n) and a rank-1 mode: all three algorithms recover a
    noise-free tensor of exact multilinear rank."""
    dims, ranks = (4, 3, 5, 2, 3, 4, 2, 3), (2, 3, 2, 1, 2, 2, 2, 2)
    x = lowrank_tensor(dims, ranks, 19, noise=0.0, factors="gaussian")
    for algo in ("rhosvd", "rsthosvd"):
        g, us = getattr(A, algo)(x, ranks, 1, _omegas(algo, dims, ranks, 1))
        assert M.rel_error(x, g, us) <= 1e-12
    rng = np.random.default_rng(19)
    om = [rng.standard_normal((int(np.prod(dims)) // d, min(r + 1, d))) for d, r in zip(dims, ranks)]
    ot = [rng.standard_normal((min(r + 1, d) + 1, d)) for d, r in zip(dims, ranks)]
    g, us, _ = A.rpet(x, ranks, om, ot)
    assert M.rel_error(x, g, us) <= 1e-10


def test_full_width_sketch_equals_deterministic():
    """K_n >= I_n: range(X_(n) Omega) = range(X_(n)) a.s., so RP-HOSVD = truncated HOSVD
    and R-STHOSVD = STHOSVD (same subspaces, same error)."""
    x = random_tensor((8, 9, 10), 16)
    ranks = (3, 4, 5)
    om = _omegas("rhosvd", x.shape, ranks, 100)
    assert all(c == i for (_, c), i in zip(A.omega_shapes("rhosvd", x.shape, ranks, 100), x.shape))
    g_r, u_r = A.rhosvd(x, ranks, 0, om)
    g_t, u_t = A.thosvd(x, ranks)
    for a, b in zip(u_r, u_t):
        assert M.max_principal_sine(a, b) < 1e-10
    assert M.rel_error(x, g_r, u_r) == pytest.approx(M.rel_error(x, g_t, u_t), rel=1e-10)
    om = _omegas("rsthosvd", x.shape, ranks, 100)
    g_r, u_r = A.rsthosvd(x, ranks, 0, om)
    g_s, u_s = A.sthosvd(x, ranks)
    for a, b in zip(u_r, u_s):
        assert M.max_principal_sine(a, b) < 1e-10
    assert M.rel_error(x, g_r, u_r) == pytest.approx(M.rel_error(x, g_s, u_s), rel=1e-10)


def test_pythagoras_and_error_split():
    """||X||^2 = ||X x_n QQ^T||^2 + ||X x_n (I - QQ^T)||^2 for orthonormal Q, and
    ||X - X x_1 Q1Q1^T ... x_N QNQN^T||^2 <= sum_n ||X - X x_n QnQn^T||^2 (Sec. 5.1)."""
    x = lowrank_tensor((15, 16, 17), (4, 5, 6), 17, noise=0.2)
    ranks = (3, 4, 5)
    _, us = A.rhosvd(x, ranks, 1, _omegas("rhosvd", x.shape, ranks, 2))
    nx2 = np.sum(x ** 2)
    parts = []
    for n, u in enumerate(us):
        p = u @ u.T
        a = T.ttm(x, p, n)
        b = T.ttm(x, np.eye(x.shape[n]) - p, n)
        assert np.sum(a ** 2) + np.sum(b ** 2) == pytest.approx(nx2, rel=1e-13)
        parts.append(np.sum(b ** 2))
    full = x - T.multi_ttm(x, [u @ u.T for u in us])
    assert np.sum(full ** 2) <= sum(parts) * (1 + 1e-12)


def test_rpet_identity_core_sketch_is_tucker_projection():
    """With S_n = I_n and Omega~_n = I, (Omega~_n Q_n)^+ = Q_n^T, so the recovered core is
    X x_1 Q_1^T ... x_N Q_N^T exactly."""
    x = lowrank_tensor((10, 11, 12), (3, 3, 3), 18, noise=0.1)
    ranks = (3, 3, 3)
    K = (5, 5, 5)
    om, _ = _omegas("rpet", x.shape, ranks, 2, K=K, S=(10, 11, 12))
    ot = [np.eye(i) for i in x.shape]
    g, us, ex = A.rpet(x, ranks, om, ot)
    np.testing.assert_allclose(ex["C"], T.multi_ttm(x, ex["Q"], transpose=True), atol=1e-12)
    np.testing.assert_allclose(ex["H"], x)


# ----------------------------------------------------------------------------- planted mistakes

def test_planted_mistakes_fail_exact_recovery(monkeypatch):
    """Plausible mistakes planted in the oracle are caught by the exact-recovery pin."""
    dims, ranks = (20, 21, 22), (3, 4, 5)
    x = lowrank_tensor(dims, ranks, 19, noise=0.0, factors="gaussian")
    om = _omegas("rhosvd", dims, ranks, 2)

    real_svd = np.linalg.svd

    def trailing_vectors_svd(a, full_matrices=True, compute_uv=True):
        u, s, vt = real_svd(a, full_matrices=full_matrices)
        return u[:, ::-1], s[::-1], vt[::-1]

    monkeypatch.setattr(A.np.linalg, "svd", trailing_vectors_svd)
    g, us = A.rhosvd(x, ranks, 0, om)
    monkeypatch.setattr(A.np.linalg, "svd", real_svd)
    assert M.rel_error(x, g, us) > 1e-3

    # transposed operand instead of the pseudo-inverse in R-PET's core recovery
    K = tuple(r + 2 for r in ranks)
    omf, omt = _omegas("rpet", dims, ranks, 2, K=K, S=tuple(2 * k + 1 for k in K))
    monkeypatch.setattr(A, "pinv_lstsq", lambda a: np.asarray(a).T)
    g, us, _ = A.rpet(x, ranks, omf, omt)
    assert M.rel_error(x, g, us) > 1e-3


# ----------------------------------------------------------------------------- metrics

def test_metrics_closed_forms():
    th = 0.3
    a = np.array([[1.0], [0.0], [0.0]])
    b = np.array([[math.cos(th)], [math.sin(th)], [0.0]])
    assert M.max_principal_sine(a, b) == pytest.approx(math.sin(th), rel=1e-14)
    assert M.max_principal_sine(a, 3 * a) < 1e-15
    x = random_tensor((4, 5, 6), 20)
    eye = [np.eye(d) for d in x.shape]
    assert M.rel_error(x, x, eye) == 0.0
    assert M.rel_error(x, 0.5 * x, eye) == pytest.approx(0.5, rel=1e-14)
    assert M.rel_error(x, -x, eye) == pytest.approx(2.0, rel=1e-14)
    assert M.orthonormality(np.eye(5)[:, :3]) == 0.0
    assert M.compression_ratio((10, 10, 10), (2, 2, 2)) == pytest.approx(1000 / (8 + 60))
