"""Seeded synthetic tensors shaped like the paper's experiments (Sec. 8, Test 1).

Storage convention used everywhere in this project: an N-way tensor with sizes
(I_1, ..., I_N) is stored column-major, i_1 fastest, which is the order the
n-unfolding of Sec. 2 enumerates its columns in.  In NumPy this is an array of
shape (I_1, ..., I_N) in Fortran order; the flat buffer handed to the CUDA
library is ``X.ravel(order="F")``.

Recipes (the numbers are the workload definitions, the construction is the
paper's low-multilinear-rank template of Sec. 8.1.1 resized):

* ``lowrank_tensor``: X_s = G x_1 U_1 ... x_N U_N with a core G whose entries
  are i.i.d. N(0,1), optionally scaled by decay**(i_1+...+i_N) (0-based), and
  factors U_n that are either orthonormal (Q of the QR of an I_n x R_n Gaussian
  matrix) or plain Gaussian.  Noise is added at a relative Frobenius level eta:
  X = X_s + gamma*N with gamma = eta*||X_s||_F/||N||_F, so SNR = -20 log10(eta) dB
  (the noise model of Sec. 8, Eq. "noisytensor").
* ``function_tensor``: X(i,j,k) = (i^5 + j^5 + k^5)^(-1/5), 1-based (Sec. 8.1.2).
* ``hilbert_tensor``: X(i_1..i_N) = 1/(i_1 + ... + i_N - N + 1), 1-based (Sec. 8.1.4).
* ``gaussian_matrix``: explicit i.i.d. N(0,1) test matrices Omega, rounded to
  FP32, so that the CUDA path and the oracle consume identical values.
"""
from __future__ import annotations

import dataclasses
from typing import Sequence

import numpy as np

__all__ = [
    "Workload", "lowrank_tensor", "function_tensor", "hilbert_tensor",
    "gaussian_matrix", "gaussian_matrices", "device_layout", "workload",
    "WORKLOADS", "random_tensor",
]


def _multilinear(core: np.ndarray, factors: Sequence[np.ndarray]) -> np.ndarray:
    """Assemble core x_1 U_1 ... x_N U_N with library tensordots (input construction only)."""
    t = core
    for n, u in enumerate(factors):
        t = np.moveaxis(np.tensordot(u, t, axes=([1], [n])), 0, n)
    return np.asfortranarray(t)


def lowrank_tensor(dims: Sequence[int], ranks: Sequence[int], seed: int, noise: float = 0.0,
                   decay: float | None = None, factors: str = "orthonormal",
                   return_signal: bool = False):
    """Low-multilinear-rank tensor plus relative Frobenius noise, FP64, Fortran order."""
    dims = tuple(int(d) for d in dims)
    ranks = tuple(int(r) for r in ranks)
    rng = np.random.default_rng(seed)
    core = rng.standard_normal(ranks)
    if decay is not None:
        grid = np.indices(ranks).sum(axis=0)
        core = core * decay ** grid
    us = []
    for i_n, r_n in zip(dims, ranks):
        g = rng.standard_normal((i_n, r_n))
        if factors == "orthonormal":
            g, _ = np.linalg.qr(g)
        us.append(g)
    xs = _multilinear(np.asfortranarray(core), us)
    if noise > 0:
        # draw the noise in FP32 to keep large workloads fast; the scale is exact in FP64
        nz = rng.standard_normal(dims, dtype=np.float32).astype(np.float64)
        nz = np.asfortranarray(nz)
        gamma = noise * np.linalg.norm(xs.ravel(order="K")) / np.linalg.norm(nz.ravel(order="K"))
        x = xs + gamma * nz
        x = np.asfortranarray(x)
    else:
        x = xs
    if return_signal:
        return x, xs
    return x


def random_tensor(dims: Sequence[int], seed: int) -> np.ndarray:
    """Dense i.i.d. N(0,1) tensor (full multilinear rank), Fortran order."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal(tuple(dims)))


def function_tensor(n: int) -> np.ndarray:
    """X(i,j,k) = 1/(i^5+j^5+k^5)^(1/5) with 1-based indices."""
    i = np.arange(1, n + 1, dtype=np.float64) ** 5
    s = i[:, None, None] + i[None, :, None] + i[None, None, :]
    return np.asfortranarray(s ** (-0.2))


def hilbert_tensor(dims: Sequence[int]) -> np.ndarray:
    """X(i_1..i_N) = 1/(i_1+...+i_N - N + 1) with 1-based indices."""
    dims = tuple(int(d) for d in dims)
    s = np.zeros(dims)
    for n, d in enumerate(dims):
        shape = [1] * len(dims)
        shape[n] = d
        s = s + np.arange(d, dtype=np.float64).reshape(shape)
    return np.asfortranarray(1.0 / (s + 1.0))


def gaussian_matrix(seed: int, rows: int, cols: int) -> np.ndarray:
    """rows x cols i.i.d. N(0,1) FP32 matrix, column-major (Fortran order)."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((cols, rows), dtype=np.float32).T)


def gaussian_matrices(seed: int, shapes: Sequence[tuple[int, int]]) -> list[np.ndarray]:
    """One independent Gaussian matrix per (rows, cols), seeds seed, seed+1, ..."""
    return [gaussian_matrix(seed + t, r, c) for t, (r, c) in enumerate(shapes)]


def device_layout(x: np.ndarray) -> np.ndarray:
    """Flat FP32 buffer of a tensor in the column-major storage order."""
    return np.asfortranarray(x, dtype=np.float32).ravel(order="F")


@dataclasses.dataclass(frozen=True)
class Workload:
    """One decomposition problem: tensor recipe plus algorithm parameters."""
    name: str
    dims: tuple
    ranks: tuple
    algo: str           # "rhosvd" (Alg. 6 + Alg. 1), "rsthosvd" (Alg. 8), "rpet" (Alg. 9)
    p: int              # oversampling
    q: int              # power iterations
    noise: float
    decay: float | None
    seed: int           # data seed
    omega_seed: int = 0
    K: tuple | None = None   # explicit sketch widths (R-PET)
    S: tuple | None = None   # core sketch widths (R-PET)

    def tensor(self, return_signal: bool = False):
        return lowrank_tensor(self.dims, self.ranks, self.seed, self.noise, self.decay,
                              return_signal=return_signal)


WORKLOADS = {
    # 100^3 FP64 low-rank tensor, rank 10, 1e-3 noise; randomized HOSVD, p=5, q=0
    "lowrank100_rhosvd": Workload("lowrank100_rhosvd", (100, 100, 100), (10, 10, 10), "rhosvd",
                                  5, 0, 1e-3, None, 1001),
    # 512^3 FP32 low-rank tensor, rank 32 with 0.9^(i+j+k) core decay, 1e-4 noise; R-STHOSVD p=10 q=1
    "decay512_rsthosvd": Workload("decay512_rsthosvd", (512, 512, 512), (32, 32, 32), "rsthosvd",
                                  10, 1, 1e-4, 0.9, 1002),
    # 128^4 low-rank tensor, rank 16, 1e-3 noise; single-pass R-PET, K=26, S=40
    "lowrank128x4_rpet": Workload("lowrank128x4_rpet", (128, 128, 128, 128), (16, 16, 16, 16), "rpet",
                                  10, 0, 1e-3, None, 1003, K=(26,) * 4, S=(40,) * 4),
}


def workload(name: str) -> Workload:
    return WORKLOADS[name]
