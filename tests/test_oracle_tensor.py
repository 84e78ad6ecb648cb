"""Pins for the multilinear primitives of the oracle (Sec. 2), by brute force."""
import itertools

import numpy as np
import pytest

from oracle import tensor as T

SHAPES = [(3, 4, 5), (2, 3, 2, 4), (5, 1, 3), (4, 3)]


def _rand(shape, seed=0):
    return np.random.default_rng(seed).standard_normal(shape)


def _brute_unfold(x, n):
    """X_(n)(i_n, j), j = sum_{k != n} i_k J_k, J_k = prod_{m<k, m != n} I_m (0-based)."""
    dims = x.shape
    cols = int(np.prod([d for k, d in enumerate(dims) if k != n]))
    out = np.zeros((dims[n], cols))
    for idx in itertools.product(*[range(d) for d in dims]):
        j = 0
        for k in range(len(dims)):
            if k == n:
                continue
            jk = 1
            for m in range(k):
                if m != n:
                    jk *= dims[m]
            j += idx[k] * jk
        out[idx[n], j] = x[idx]
    return out


@pytest.mark.parametrize("shape", SHAPES)
def test_unfold_matches_index_formula(shape):
    x = _rand(shape)
    for n in range(len(shape)):
        np.testing.assert_array_equal(T.unfold(x, n), _brute_unfold(x, n))


@pytest.mark.parametrize("shape", SHAPES)
def test_fold_inverts_unfold(shape):
    x = _rand(shape, 1)
    for n in range(len(shape)):
        np.testing.assert_array_equal(T.fold(T.unfold(x, n), n, shape), x)


def test_unfold_pin_catches_row_major_flattening():
    """A C-order flattening (a plausible transposition mistake) fails the index pin."""
    x = _rand((3, 4, 5))
    wrong = np.reshape(np.moveaxis(x, 1, 0), (4, -1), order="C")
    assert not np.array_equal(wrong, _brute_unfold(x, 1))


@pytest.mark.parametrize("shape", SHAPES)
def test_ttm_matches_elementwise_sum(shape):
    x = _rand(shape, 2)
    for n in range(len(shape)):
        b = _rand((3, shape[n]), 3 + n)
        got = T.ttm(x, b, n)
        want_shape = list(shape)
        want_shape[n] = 3
        want = np.zeros(want_shape)
        for idx in itertools.product(*[range(d) for d in want_shape]):
            s = 0.0
            for i_n in range(shape[n]):
                src = list(idx)
                src[n] = i_n
                s += x[tuple(src)] * b[idx[n], i_n]
            want[idx] = s
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)


def test_ttm_product_rule():
    """X x_n B x_n A = X x_n (A B) (Eq. TMM-M)."""
    x = _rand((4, 5, 6), 4)
    b = _rand((3, 5), 5)
    a = _rand((2, 3), 6)
    lhs = T.ttm(T.ttm(x, b, 1), a, 1)
    rhs = T.ttm(x, a @ b, 1)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("shape,ranks", [((4, 5, 6), (2, 3, 4)), ((3, 4, 2, 5), (2, 2, 2, 3))])
def test_tucker_unfolding_kronecker_identity(shape, ranks):
    """X = S x_1 Q1 ... x_N QN  <=>  X_(n) = Q^(n) S_(n) (Q^(N) (x) ... (x) Q^(n+1) (x) Q^(n-1) (x) ... (x) Q^(1))^T
    (Eq. TuckerUnfold, reverse Kronecker order)."""
    s = _rand(ranks, 7)
    qs = [_rand((i, r), 8 + k) for k, (i, r) in enumerate(zip(shape, ranks))]
    x = T.reconstruct(s, qs)
    for n in range(len(shape)):
        others = [qs[k] for k in reversed(range(len(shape))) if k != n]
        rhs = qs[n] @ T.unfold(s, n) @ T.kron_chain(others).T
        np.testing.assert_allclose(T.unfold(x, n), rhs, rtol=1e-12, atol=1e-12)


def test_kronecker_identity_catches_forward_order():
    """Forward Kronecker order (a plausible mistake) does not satisfy the identity."""
    shape, ranks = (4, 5, 6), (2, 3, 4)
    s = _rand(ranks, 7)
    qs = [_rand((i, r), 8 + k) for k, (i, r) in enumerate(zip(shape, ranks))]
    x = T.reconstruct(s, qs)
    n = 0
    fwd = [qs[k] for k in range(3) if k != n]
    rhs = qs[n] @ T.unfold(s, n) @ T.kron_chain(fwd).T
    assert not np.allclose(T.unfold(x, n), rhs)


def test_multi_ttm_skips_none_and_transposes():
    x = _rand((3, 4, 5), 9)
    m = _rand((4, 2), 10)
    np.testing.assert_allclose(T.multi_ttm(x, [None, m, None], transpose=True), T.ttm(x, m.T, 1))
