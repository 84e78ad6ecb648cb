"""Multilinear primitives of Sec. 2, written out from their definitions.

Tensors are NumPy arrays of shape (I_1, ..., I_N); mode indices are 0-based in
code (mode n here is the paper's mode n+1).
"""
from __future__ import annotations

from typing import Sequence

import numpy as np


def unfold(x: np.ndarray, n: int) -> np.ndarray:
    """n-unfolding X_(n) of Sec. 2: X_(n)(i_n, j) = X(i_1, ..., i_N) with
    j = sum_{k != n} i_k J_k (0-based) and J_k = prod_{m < k, m != n} I_m.

    Moving mode n to the front and flattening the remaining modes with the
    lowest mode fastest (Fortran order) enumerates j exactly as the formula does.
    """
    x = np.asarray(x)
    return np.reshape(np.moveaxis(x, n, 0), (x.shape[n], -1), order="F")


def fold(m: np.ndarray, n: int, dims: Sequence[int]) -> np.ndarray:
    """Inverse of ``unfold``: rebuild the tensor of sizes ``dims`` from M = X_(n)."""
    dims = tuple(int(d) for d in dims)
    front = (dims[n],) + dims[:n] + dims[n + 1:]
    return np.moveaxis(np.reshape(m, front, order="F"), 0, n)


def ttm(x: np.ndarray, b: np.ndarray, n: int) -> np.ndarray:
    """n-mode product X x_n B of Sec. 2 for B of size J x I_n:
    (X x_n B)(i_1..j..i_N) = sum_{i_n} X(i_1..i_n..i_N) B(j, i_n).
    Computed through the unfolding: (X x_n B)_(n) = B X_(n)."""
    dims = list(x.shape)
    dims[n] = b.shape[0]
    return fold(b @ unfold(x, n), n, dims)


def multi_ttm(x: np.ndarray, mats: Sequence[np.ndarray | None], transpose: bool = False) -> np.ndarray:
    """X x_1 M_1 x_2 ... x_N M_N (M_n^T when ``transpose``); ``None`` skips a mode."""
    t = x
    for n, m in enumerate(mats):
        if m is None:
            continue
        t = ttm(t, m.T if transpose else m, n)
    return t


def reconstruct(core: np.ndarray, factors: Sequence[np.ndarray]) -> np.ndarray:
    """Tucker model [[S; Q^(1), ..., Q^(N)]] = S x_1 Q^(1) ... x_N Q^(N) (Sec. 4)."""
    return multi_ttm(core, factors)


def kron_chain(mats: Sequence[np.ndarray]) -> np.ndarray:
    """Kronecker product M_1 (x) M_2 (x) ... in the given order."""
    out = np.ones((1, 1))
    for m in mats:
        out = np.kron(out, m)
    return out
