"""Pins for the seeded input generators shared by the oracle and the CUDA path:
the relative noise level, the exact multilinear rank of the signal, the decay
scaling of the core, determinism, the closed-form tensors of Sec. 8, and the
column-major flat layout handed to the library."""
import numpy as np
import pytest

from oracle import tensor as T
from workloads import (WORKLOADS, device_layout, function_tensor, gaussian_matrix, hilbert_tensor,
                       lowrank_tensor)


@pytest.mark.parametrize("eta", [1e-1, 1e-3, 1e-4])
def test_noise_is_at_the_stated_relative_level(eta):
    x, xs = lowrank_tensor((20, 18, 16), (4, 5, 3), seed=3, noise=eta, return_signal=True)
    assert abs(np.linalg.norm(x - xs) / np.linalg.norm(xs) - eta) <= 1e-12 * eta


def test_signal_has_the_stated_multilinear_rank():
    dims, ranks = (20, 18, 16, 9), (4, 5, 3, 2)
    _, xs = lowrank_tensor(dims, ranks, seed=4, noise=1e-3, return_signal=True)
    for n in range(len(dims)):
        s = np.linalg.svd(T.unfold(xs, n), compute_uv=False)
        assert np.sum(s > 1e-12 * s[0]) == ranks[n]


def test_orthonormal_factors_keep_the_core_norm_and_decay_scales_it():
    dims, ranks = (15, 14, 13), (3, 4, 2)
    rng = np.random.default_rng(5)
    core = rng.standard_normal(ranks)                     # the generator's first draw
    _, xs = lowrank_tensor(dims, ranks, seed=5, return_signal=True)
    assert abs(np.linalg.norm(xs) - np.linalg.norm(core)) <= 1e-12 * np.linalg.norm(core)
    _, xd = lowrank_tensor(dims, ranks, seed=5, decay=0.5, return_signal=True)
    scaled = core * 0.5 ** np.indices(ranks).sum(axis=0)
    assert abs(np.linalg.norm(xd) - np.linalg.norm(scaled)) <= 1e-12 * np.linalg.norm(scaled)


def test_generators_are_deterministic_and_column_major():
    a = lowrank_tensor((9, 8, 7), (2, 3, 2), seed=6, noise=1e-2)
    b = lowrank_tensor((9, 8, 7), (2, 3, 2), seed=6, noise=1e-2)
    np.testing.assert_array_equal(a, b)
    assert a.flags["F_CONTIGUOUS"]
    flat = device_layout(a)
    assert flat.dtype == np.float32 and flat.shape == (9 * 8 * 7,)
    # i_1 fastest: element (i, j, k) at i + 9 j + 72 k
    assert flat[1 + 9 * 2 + 72 * 3] == np.float32(a[1, 2, 3])


def test_gaussian_matrix_is_fp32_column_major_and_standard():
    g = gaussian_matrix(7, 4000, 25)
    assert g.dtype == np.float32 and g.shape == (4000, 25) and g.flags["F_CONTIGUOUS"]
    np.testing.assert_array_equal(g, gaussian_matrix(7, 4000, 25))
    assert abs(float(g.mean())) < 0.01 and abs(float(g.var()) - 1.0) < 0.02


def test_closed_form_tensors():
    f = function_tensor(6)
    assert f[0, 0, 0] == pytest.approx(3.0 ** -0.2)
    assert f[1, 2, 3] == pytest.approx((2 ** 5 + 3 ** 5 + 4 ** 5) ** -0.2)
    h = hilbert_tensor((4, 5, 6))
    assert h[0, 0, 0] == 1.0 and h[3, 4, 5] == pytest.approx(1.0 / 13.0)


def test_workloads_match_their_descriptions():
    w = WORKLOADS["decay512_rsthosvd"]
    assert w.dims == (512, 512, 512) and w.ranks == (32, 32, 32) and w.p == 10 and w.q == 1
    assert w.noise == 1e-4 and w.decay == 0.9 and w.algo == "rsthosvd"
    r = WORKLOADS["lowrank128x4_rpet"]
    assert r.dims == (128,) * 4 and r.ranks == (16,) * 4 and r.algo == "rpet"
