"""Pins of the oracle's reduced-precision formats and of its RP-HOOI
refinement sweep (Alg. 7).

Formats (oracle/precision.py) against their definitions by brute force:
every one of the 256 e4m3 codes decoded from its bit fields is a fixed point
of the rounding, and rounding picks the nearest code with ties to an even
mantissa; BF16 rounding picks the nearest value with 7 stored mantissa bits;
the per-slice scales are the smallest powers of two that bring each frontal
slice inside the e4m3 range.

RP-HOOI: with sketch widths that cover every column of S_(n) the sweep is
exactly the HOOI sweep of Alg. 5; started from the true factors of a
noise-free tensor of exact multilinear rank it recovers the tensor; after a
single-pass R-PET it lowers the error to within a small factor of the
converged HOOI error.
"""
import numpy as np
import pytest

from oracle import algorithms as A
from oracle import metrics as M
from oracle import precision as P
from workloads import gaussian_matrix, lowrank_tensor


def _e4m3_codes():
    """All finite e4m3 values from the bit fields: sign, 4 exponent bits (bias 7),
    3 mantissa bits; exponent field 0 is subnormal; S.1111.111 is NaN."""
    vals = []
    for code in range(256):
        s, e, m = code >> 7, (code >> 3) & 15, code & 7
        if e == 15 and m == 7:
            continue
        v = (m / 8.0) * 2.0 ** -6 if e == 0 else (1 + m / 8.0) * 2.0 ** (e - 7)
        vals.append((-v if s else v, m))
    return vals


def test_e4m3_codes_are_fixed_points_and_span_448():
    vals = _e4m3_codes()
    v = np.array([a for a, _ in vals])
    assert np.array_equal(P.e4m3_round(v), v)
    assert v.max() == 448.0 and np.min(v[v > 0]) == 2.0 ** -9
    assert len(set(v.tolist())) == 253                 # +0 and -0 coincide


def test_e4m3_round_is_nearest_with_ties_to_even():
    vals = _e4m3_codes()
    grid = np.array(sorted({a for a, _ in vals}))
    mant = {a: m for a, m in vals}
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(-460, 460, 4000), rng.normal(0, 0.05, 4000),
                        (grid[:-1] + grid[1:]) / 2])      # every midpoint: a tie
    r = P.e4m3_round(x)
    for xi, ri in zip(x, r):
        xc = min(max(xi, -448.0), 448.0)
        d = np.abs(grid - xc)
        best = grid[d == d.min()]
        if len(best) == 1:
            assert ri == best[0], (xi, ri, best)
        else:
            even = [b for b in best if mant[b] % 2 == 0]
            assert ri == even[0], (xi, ri, best)


def test_bf16_round_is_nearest_representable():
    rng = np.random.default_rng(2)
    x = (rng.standard_normal(3000) * 10.0 ** rng.uniform(-20, 20, 3000)).astype(np.float32)
    r = P.bf16_round(x)
    u = x.view(np.uint32)
    lo = (u & 0xFFFF0000).view(np.float32).astype(np.float64)
    hi = ((u & 0xFFFF0000) + 0x10000).view(np.float32).astype(np.float64)
    xd = x.astype(np.float64)
    for xi, ri, a, b, ua in zip(xd, r, lo, hi, u):
        da, db = abs(xi - a), abs(xi - b)
        if da < db:
            assert ri == a
        elif db < da:
            assert ri == b
        else:                                              # tie: the even 16-bit pattern
            assert ri == (a if ((ua >> 16) & 1) == 0 else b)
    # 7 stored mantissa bits: every rounded value has a zero low half
    assert np.all((r.astype(np.float32).view(np.uint32) & 0xFFFF) == 0)


def test_slice_scales_are_minimal_powers_of_two():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((6, 5, 7)) * np.array([1e-3, 1.0, 448.0, 449.0, 1e5, 3.5, 0.0])
    s = P.slice_scales(x)
    amax = np.abs(x).reshape(-1, 7, order="F").max(axis=0)
    for k in range(7):
        e = np.log2(s[k])
        assert e == int(e)
        assert amax[k] / s[k] <= 448.0
        if amax[k] > 0:
            assert amax[k] / (s[k] / 2) > 448.0           # the next smaller power would overflow
    assert s[6] == 1.0
    xq, s2 = P.quantize(x, "e4m3")
    assert np.array_equal(s, s2)
    assert np.all(np.abs(xq - x) <= np.abs(x) / 16 + s * 2.0 ** -10)   # half a spacing of 3 mantissa bits


def _omegas(dims, ranks, p, seed):
    return [gaussian_matrix(seed + n, j, k).astype(np.float64)
            for n, (j, k) in enumerate(A.rp_hooi_omega_shapes(dims, ranks, p))]


def test_rp_hooi_with_full_width_sketches_is_the_hooi_sweep():
    dims, ranks = (14, 12, 10), (3, 4, 2)
    x = lowrank_tensor(dims, ranks, seed=31, noise=0.05)
    _, u0 = A.thosvd(x, ranks)
    u0 = [np.linalg.qr(u + 0.3 * np.random.default_rng(n).standard_normal(u.shape))[0] for n, u in enumerate(u0)]
    om = _omegas(dims, ranks, p=40, seed=400)              # K_n = J_n: the sketch sees every column
    assert all(o.shape[1] == o.shape[0] or o.shape[1] == d for o, d in zip(om, dims))
    g_r, u_r = A.rp_hooi_sweep(x, u0, ranks, om)
    g_h, u_h = A.hooi_sweep(x, u0, ranks)
    for a, b in zip(u_r, u_h):
        assert M.max_principal_sine(a, b) <= 1e-10
    assert abs(M.rel_error(x, g_r, u_r) - M.rel_error(x, g_h, u_h)) <= 1e-12


def test_rp_hooi_from_true_factors_recovers_exact_rank():
    dims, ranks = (20, 18, 16, 6), (4, 3, 5, 2)
    x = lowrank_tensor(dims, ranks, seed=32)
    _, u_true = A.thosvd(x, ranks)
    g, us = A.rp_hooi_sweep(x, u_true, ranks, _omegas(dims, ranks, 5, 500))
    assert M.rel_error(x, g, us) <= 1e-12
    assert max(M.orthonormality(u) for u in us) <= 1e-12


def test_rp_hooi_refines_a_single_pass_result():
    dims, ranks = (30, 28, 26), (4, 5, 3)
    x = lowrank_tensor(dims, ranks, seed=33, noise=1e-2)
    K, S = [r + 6 for r in ranks], [2 * (r + 6) + 1 for r in ranks]
    om = [gaussian_matrix(600 + n, int(np.prod(dims)) // dims[n], K[n]).astype(np.float64) for n in range(3)]
    ot = [gaussian_matrix(700 + n, S[n], dims[n]).astype(np.float64) for n in range(3)]
    g0, u0, _ = A.rpet(x, ranks, om, ot)
    e0 = M.rel_error(x, g0, u0)
    g1, u1 = A.rp_hooi_sweep(x, u0, ranks, _omegas(dims, ranks, 10, 800))
    e1 = M.rel_error(x, g1, u1)
    g_h, u_h = A.hooi(x, ranks, sweeps=10)
    e_h = M.rel_error(x, g_h, u_h)
    assert e1 < e0
    assert e1 <= 1.01 * e_h
    # the core of the sweep is the projection of X onto its factors
    from oracle import tensor as T
    assert np.allclose(g1, T.multi_ttm(x, u1, transpose=True), atol=1e-12 * np.linalg.norm(x))


def test_kronecker_test_matrix_is_the_mode_product_sketch():
    """X_(n) (Phi_N kron ... kron Phi_1, without Phi_n) equals the n-unfolding of
    X x_{p != n} Phi_p^T, computed by mode products; the forward Kronecker order
    does not (a transposed ordering is caught)."""
    from oracle import tensor as T
    rng = np.random.default_rng(9)
    dims, k = (5, 4, 3, 6), 2
    x = rng.standard_normal(dims)
    phis = [rng.standard_normal((d, k)) for d in dims]
    for n in range(4):
        om = A.kronecker_test_matrix(phis, n)
        assert om.shape == (int(np.prod(dims)) // dims[n], k ** 3)
        via_ttm = T.unfold(T.multi_ttm(x, [None if p == n else phis[p].T for p in range(4)]), n)
        assert np.allclose(T.unfold(x, n) @ om, via_ttm, atol=1e-12)
        fwd = np.ones((1, 1))
        for p in range(4):
            if p != n:
                fwd = np.kron(fwd, phis[p])
        assert not np.allclose(T.unfold(x, n) @ fwd, via_ttm, atol=1e-6)
