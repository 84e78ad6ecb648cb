"""Pins for the oracle's fixed-accuracy path: the blocked range finder with an
error indicator, the rank-revealing truncation and fixed-accuracy R-STHOSVD.

Each pin checks the arithmetic against something it does not share: the
indicator against the residual computed from scratch, the truncation rank
against a brute-force search, the error guarantee ||X - X_hat|| <= eps ||X||
that the tolerance split implies, exact recovery of tensors of known
multilinear rank, and a single full-width block against the deterministic
fixed-accuracy ST-HOSVD built on LAPACK's SVD."""
import numpy as np
import pytest

from oracle import algorithms as A
from oracle import metrics as M
from oracle import tensor as T
from workloads import gaussian_matrix, lowrank_tensor


def _omega(seed):
    """Test blocks as inputs: block i of mode n is a seeded Gaussian J x b matrix."""
    def f(n, i, j, b):
        return gaussian_matrix(seed + 1000 * n + i, j, b).astype(np.float64)
    return f


def _residual(a, q):
    return float(np.linalg.norm(a - q @ (q.T @ a)) ** 2)


@pytest.mark.parametrize("q_power", [0, 1])
def test_error_indicator_equals_residual(q_power):
    rng = np.random.default_rng(3)
    a = rng.standard_normal((60, 15)) @ np.diag(0.7 ** np.arange(15)) @ rng.standard_normal((15, 90))
    a += 1e-3 * rng.standard_normal(a.shape)
    qm, bm, hist = A.randqb_ei(a, 0.0, 4, 40, lambda i, j, b: gaussian_matrix(50 + i, j, b).astype(np.float64),
                               q=q_power)
    assert qm.shape == (60, 40) and bm.shape == (40, 90) and len(hist) == 10
    assert M.orthonormality(qm) < 1e-12
    np.testing.assert_allclose(bm, qm.T @ a, atol=1e-12)
    # the indicator after each block is the residual of the basis built so far
    for i, e in enumerate(hist):
        qi = qm[:, : 4 * (i + 1)]
        assert abs(e - _residual(a, qi)) <= 1e-10 * float(np.sum(a * a)), (i, e, _residual(a, qi))


def test_range_finder_stops_at_the_tolerance():
    rng = np.random.default_rng(4)
    a = rng.standard_normal((80, 30)) @ np.diag(0.8 ** np.arange(30)) @ rng.standard_normal((30, 70))
    tol = 1e-2 * np.linalg.norm(a)
    qm, _, hist = A.randqb_ei(a, tol, 3, 80, lambda i, j, b: gaussian_matrix(60 + i, j, b).astype(np.float64))
    assert hist[-1] <= tol ** 2                        # stopped because the indicator met the tolerance
    assert all(e > tol ** 2 for e in hist[:-1])        # and not before
    assert _residual(a, qm) <= tol ** 2 * (1 + 1e-9)


def test_truncation_rank_is_the_smallest_admissible():
    rng = np.random.default_rng(5)
    for _ in range(50):
        sig = np.sort(rng.exponential(1.0, size=12))[::-1]
        res = float(rng.uniform(0, 0.5))
        tol = float(rng.uniform(0.3, 3.0))
        r = A.truncation_rank(sig, res, tol)
        brute = next((k for k in range(13) if res + float(np.sum(sig[k:] ** 2)) <= tol * tol), 12)
        assert r == brute


def test_exact_multilinear_rank_is_recovered():
    dims, ranks = (30, 26, 22), (4, 6, 5)
    x = lowrank_tensor(dims, ranks, seed=11, noise=0.0)
    g, us, found = A.rsthosvd_fixed_accuracy(x, 1e-6, 3, [20, 20, 20], _omega(7))
    assert found == list(ranks)
    assert M.rel_error(x, g, us) <= 1e-9
    for u in us:
        assert M.orthonormality(u) < 1e-12


@pytest.mark.parametrize("eps", [1e-1, 3e-2, 1e-2, 3e-3])
def test_error_guarantee_holds(eps):
    dims, ranks = (40, 36, 32), (12, 10, 8)
    x = lowrank_tensor(dims, ranks, seed=12, noise=1e-3)
    g, us, found = A.rsthosvd_fixed_accuracy(x, eps, 4, list(dims), _omega(8), q=1)
    err = M.rel_error(x, g, us)
    assert err <= eps * (1 + 1e-9), (err, eps, found)
    # smaller tolerances never need smaller ranks on the same inputs
    if eps > 3e-3:
        _, _, tighter = A.rsthosvd_fixed_accuracy(x, eps / 3, 4, list(dims), _omega(8), q=1)
        assert all(t >= f for t, f in zip(tighter, found))


def _deterministic_fixed_accuracy(x, eps):
    """ST-HOSVD with ranks from each unfolding's own singular values (LAPACK SVD)."""
    s = np.asarray(x, dtype=np.float64)
    tol = eps * np.linalg.norm(s) / np.sqrt(s.ndim)
    us, ranks = [], []
    for n in range(s.ndim):
        u, sig, _ = np.linalg.svd(T.unfold(s, n), full_matrices=False)
        r = next(k for k in range(len(sig) + 1) if float(np.sum(sig[k:] ** 2)) <= tol ** 2)
        us.append(u[:, :r])
        ranks.append(r)
        s = T.ttm(s, u[:, :r].T, n)
    return s, us, ranks


def test_full_width_block_matches_deterministic_sthosvd():
    dims, ranks = (18, 16, 14), (6, 5, 4)
    x = lowrank_tensor(dims, ranks, seed=13, noise=1e-2)
    eps = 5e-3
    # one block as wide as the mode captures the whole range: E = 0 and the
    # truncation sees the unfolding's own singular values
    g, us, found = A.rsthosvd_fixed_accuracy(x, eps, 64, list(dims), _omega(9))
    gd, ud, rd = _deterministic_fixed_accuracy(x, eps)
    assert found == rd
    for u, v in zip(us, ud):
        assert M.max_principal_sine(u, v) <= 1e-8
    assert abs(M.rel_error(x, g, us) - M.rel_error(x, gd, ud)) <= 1e-12
