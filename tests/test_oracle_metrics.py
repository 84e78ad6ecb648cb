"""Pins of the oracle's accuracy measures (Sec. 8) against closed forms and
against the noisy-tensor experiment the paper reports.

* SNR [dB] = 10 log10(||X||^2 / ||gamma N||^2): signal-to-noise ratios of
  known power ratios, and the noise level the seeded generator produces
  (relative Frobenius noise eta gives -20 log10(eta) dB).
* Fit = 1 - E: exact reconstruction has fit 1, the zero approximation fit 0,
  and for the low-rank-plus-Gaussian-noise template at 20 dB the paper reports
  a fit of about 90% for the truncated HOSVD, the sequentially truncated HOSVD
  and their randomized variants (Sec. 8.1.1, noisy case).
* compression_ratio: the entry counts of X, of the core and of the factors.
"""
import numpy as np
import pytest

from oracle import algorithms as A
from oracle import metrics as M
from workloads import gaussian_matrix, lowrank_tensor


def test_snr_db_of_known_power_ratios():
    rng = np.random.default_rng(3)
    s = rng.standard_normal((7, 5, 3))
    assert M.snr_db(s, s) == pytest.approx(0.0, abs=1e-12)
    assert M.snr_db(s, 0.1 * s) == pytest.approx(20.0, abs=1e-10)
    assert M.snr_db(10 * s, s) == pytest.approx(20.0, abs=1e-10)
    assert M.snr_db(s, 1e-3 * s) == pytest.approx(60.0, abs=1e-9)
    # power ratio 100 / 1 with unrelated arrays: 20 dB
    a = np.zeros(4); a[0] = 10.0
    b = np.zeros(9); b[5] = 1.0
    assert M.snr_db(a, b) == pytest.approx(20.0, abs=1e-12)


@pytest.mark.parametrize("eta,db", [(1e-1, 20.0), (1e-3, 60.0), (1e-4, 80.0)])
def test_generator_noise_level_matches_snr_definition(eta, db):
    x, xs = lowrank_tensor((20, 18, 16), (3, 4, 2), seed=11, noise=eta, return_signal=True)
    assert M.snr_db(xs, x - xs) == pytest.approx(db, abs=1e-9)


def test_fit_closed_forms():
    x = lowrank_tensor((12, 10, 8), (3, 2, 4), seed=5)
    g, u = A.thosvd(x, (3, 2, 4))
    assert M.fit(M.rel_error(x, g, u)) == pytest.approx(1.0, abs=1e-12)
    assert M.fit(M.rel_error(x, np.zeros_like(g), u)) == pytest.approx(0.0, abs=1e-15)
    assert M.fit(0.25) == 0.75


def test_fit_at_20_db_is_about_90_percent():
    """The paper's noisy experiment: a random low-multilinear-rank tensor with
    Gaussian noise at 20 dB decomposed by THOSVD, STHOSVD and their randomized
    variants (q = 2, P = 10) gives a fit of about 90% for all of them.  A rank
    (4, 8, 6) tensor of size 60^3 stands in for the 1000^3 one: its Tucker
    subspaces hold 0.1% of the noise, so the fit sits just above 0.9."""
    dims, ranks = (60, 60, 60), (4, 8, 6)
    x = lowrank_tensor(dims, ranks, seed=21, noise=0.1)
    fits = []
    g, u = A.thosvd(x, ranks)
    fits.append(M.fit(M.rel_error(x, g, u)))
    g, u = A.sthosvd(x, ranks)
    fits.append(M.fit(M.rel_error(x, g, u)))
    for algo in ("rhosvd", "rsthosvd"):
        om = [gaussian_matrix(300 + n, r, c).astype(np.float64)
              for n, (r, c) in enumerate(A.omega_shapes(algo, dims, ranks, 10))]
        g, u = getattr(A, algo)(x, ranks, 2, om)
        fits.append(M.fit(M.rel_error(x, g, u)))
    for f in fits:
        assert 0.895 <= f <= 0.91, fits
    assert max(fits) - min(fits) <= 1e-3, fits


def test_compression_ratio_counts_entries():
    assert M.compression_ratio((10, 20, 30), (2, 3, 4)) == pytest.approx(6000 / (24 + 20 + 60 + 120))
    assert M.compression_ratio((5,), (5,)) == pytest.approx(5 / 30)
