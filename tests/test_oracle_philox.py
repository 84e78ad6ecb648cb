"""Pins for the oracle's Gaussian generator (Philox4x32-10 + Box-Muller)."""
import math

import numpy as np
import pytest

from oracle import philox

# Known-answer vectors published with the Random123 library for philox4x32-10:
# (counter c0..c3, key k0..k1) -> output words.
KAT = [
    ((0x00000000, 0x00000000, 0x00000000, 0x00000000), (0x00000000, 0x00000000),
     (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF), (0xFFFFFFFF, 0xFFFFFFFF),
     (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


@pytest.mark.parametrize("ctr,key,want", KAT)
def test_philox_known_answers(ctr, key, want):
    out = philox.philox4x32_10(*[np.array([c], dtype=np.uint64) for c in ctr], *key)
    assert tuple(int(w[0]) for w in out) == want


def test_box_muller_closed_forms():
    # w0 = 0xFFFFFFFF -> u1 = 1 -> radius 0; w0 = 0, w1 = 0 -> u1 = 2^-24, angle 0
    z0, z1 = philox._box_muller(np.array([0xFFFFFFFF], np.uint32), np.array([123456], np.uint32))
    assert z0[0] == 0.0 and z1[0] == 0.0
    z0, z1 = philox._box_muller(np.array([0], np.uint32), np.array([0], np.uint32))
    assert z0[0] == pytest.approx(math.sqrt(2 * 24 * math.log(2)), rel=1e-15)
    assert z1[0] == 0.0
    # a quarter turn: a1 = 2^22 -> u2 = 1/4
    z0, z1 = philox._box_muller(np.array([0], np.uint32), np.array([1 << 30], np.uint32))
    assert abs(z0[0]) < 1e-15 and z1[0] == pytest.approx(math.sqrt(2 * 24 * math.log(2)), rel=1e-15)


def test_omega_entry_uses_counter_layout():
    """Entry (j, k) comes from counter (j, 0, k div 4, stream) and word k mod 4."""
    seed, stream = 0x1234_5678_9ABC_DEF0, 3
    om = philox.omega(seed, stream, 7, 9)
    j, k = 5, 6
    w = philox.philox4x32_10(np.array([j], np.uint64), np.array([0], np.uint64),
                             np.array([k // 4], np.uint64), np.array([stream], np.uint64),
                             seed & 0xFFFFFFFF, seed >> 32)
    z2, z3 = philox._box_muller(w[2], w[3])
    assert om[j, k] == np.float32(z2[0])


def test_omega_prefix_and_stream_independence():
    a = philox.omega(7, 0, 100, 10)
    b = philox.omega(7, 0, 60, 3)
    np.testing.assert_array_equal(a[:60, :3], b)
    c = philox.omega(7, 1, 100, 10)
    d = philox.omega(8, 0, 100, 10)
    assert not np.any(a == c) or np.mean(a == c) < 0.01
    assert np.mean(a == d) < 0.01


def test_omega_is_standard_normal():
    z = philox.omega(2024, 0, 1 << 16, 8).astype(np.float64).ravel()
    n = z.size
    assert abs(z.mean()) < 5 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    # chi-square goodness of fit on 20 equiprobable bins of N(0,1)
    from scipy.stats import norm, chi2
    edges = norm.ppf(np.linspace(0, 1, 21))
    counts, _ = np.histogram(z, bins=edges)
    stat = np.sum((counts - n / 20) ** 2 / (n / 20))
    assert stat < chi2.ppf(0.999, 19)
    # columns uncorrelated
    m = philox.omega(2024, 0, 1 << 14, 8).astype(np.float64)
    cc = np.corrcoef(m.T)
    assert np.max(np.abs(cc - np.eye(8))) < 5 / math.sqrt(1 << 14)
