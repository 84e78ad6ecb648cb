"""Accuracy measures used to compare decompositions (Sec. 8).

Factors of a Tucker decomposition are defined only up to column signs and
rotations inside repeated singular values, so comparisons use subspaces and
reconstructions, never factor entries.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np

from .tensor import reconstruct


def rel_error(x: np.ndarray, core: np.ndarray, factors: Sequence[np.ndarray]) -> float:
    """E = ||X - Xhat||_F / ||X||_F with the residual formed explicitly in FP64
    (Eq. "Relativeerror"); ||X||^2 - ||G||^2 would cancel at small E."""
    x = np.asarray(x, dtype=np.float64)
    xhat = reconstruct(np.asarray(core, np.float64), [np.asarray(u, np.float64) for u in factors])
    return float(np.linalg.norm((x - xhat).ravel()) / np.linalg.norm(x.ravel()))


def principal_sines(ua: np.ndarray, ub: np.ndarray) -> np.ndarray:
    """Sines of the principal angles between range(Ua) and range(Ub): the
    singular values of (I - Qa Qa^T) Qb for orthonormal bases Qa, Qb."""
    qa, _ = np.linalg.qr(np.asarray(ua, dtype=np.float64))
    qb, _ = np.linalg.qr(np.asarray(ub, dtype=np.float64))
    resid = qb - qa @ (qa.T @ qb)
    return np.linalg.svd(resid, compute_uv=False)


def max_principal_sine(ua: np.ndarray, ub: np.ndarray) -> float:
    return float(np.max(principal_sines(ua, ub), initial=0.0))


def orthonormality(u: np.ndarray) -> float:
    """max |U^T U - I|."""
    u = np.asarray(u, dtype=np.float64)
    return float(np.max(np.abs(u.T @ u - np.eye(u.shape[1])), initial=0.0))


def fit(e: float) -> float:
    """Fit = 1 - E (Sec. 8)."""
    return 1.0 - e


def snr_db(signal: np.ndarray, noise: np.ndarray) -> float:
    """SNR [dB] = 10 log10(||X||^2 / ||gamma N||^2) (Sec. 8)."""
    return float(10 * np.log10(np.sum(np.square(signal)) / np.sum(np.square(noise))))


def compression_ratio(dims: Sequence[int], core_shape: Sequence[int]) -> float:
    """#entries of X over #entries of core + factors (Sec. 8)."""
    full = float(np.prod(dims, dtype=np.float64))
    small = float(np.prod(core_shape, dtype=np.float64)) + float(sum(i * r for i, r in zip(dims, core_shape)))
    return full / small
