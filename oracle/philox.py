"""Counter-based Gaussian test matrices: Philox4x32-10 + Box-Muller.

The paper draws Omega_n from a Gaussian distribution (Alg. 1, Alg. 6,
Alg. 9) and leaves the generator open.  This project fixes one so that a
decomposition is reproducible from a 64-bit seed; the GPU library implements the
same definition independently in CUDA.

Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC 2011): a 128-bit counter (c0,c1,c2,c3) and a 64-bit key (k0,k1)
go through 10 rounds.  One round multiplies c0 and c2 by the constants
M0 = 0xD2511F53 and M1 = 0xCD9E8D57 into 64-bit products (hi, lo) and outputs
(hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); between rounds the key is advanced
by the Weyl constants (0x9E3779B9, 0xBB67AE85).

Entry (j, k) of a rows x cols matrix drawn on ``stream`` uses counter
(j mod 2^32, j div 2^32, k div 4, stream) and key (seed mod 2^32, seed div 2^32).
The four output words w0..w3 give four normals by Box-Muller on 24-bit
uniforms (G. E. P. Box, M. E. Muller, 1958):
    a = w >> 8 (24 bits), u1 = (a0 + 1) 2^-24 in (0, 1], u2 = a1 2^-24 in [0, 1)
    z0 = sqrt(-2 ln u1) cos(2 pi u2),  z1 = sqrt(-2 ln u1) sin(2 pi u2)
and likewise (w2, w3) -> (z2, z3); column k takes z_(k mod 4).  Values are
evaluated in FP64 and rounded once to FP32, the precision the GPU stores.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0: int, k1: int):
    """Vectorised Philox4x32-10 on uint32 counter arrays; returns four uint32 arrays."""
    c0 = np.asarray(c0, dtype=np.uint64) & MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & MASK32
    k0 = int(k0) & 0xFFFFFFFF
    k1 = int(k1) & 0xFFFFFFFF
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & 0xFFFFFFFF
            k1 = (k1 + W1) & 0xFFFFFFFF
        p0 = M0 * c0          # < 2^64, exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1, hi0 ^ c3 ^ np.uint64(k1), lo0)
    return (c0.astype(np.uint32), c1.astype(np.uint32), c2.astype(np.uint32), c3.astype(np.uint32))


def _box_muller(wa, wb):
    a = (wa >> np.uint32(8)).astype(np.float64)
    b = (wb >> np.uint32(8)).astype(np.float64)
    u1 = (a + 1.0) * 2.0 ** -24
    u2 = b * 2.0 ** -24
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)


def omega(seed: int, stream: int, rows: int, cols: int) -> np.ndarray:
    """rows x cols Gaussian matrix (FP32 values, Fortran order) from (seed, stream)."""
    seed = int(seed)
    k0, k1 = seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF
    j = np.arange(rows, dtype=np.uint64)
    groups = (cols + 3) // 4
    out = np.empty((rows, 4 * groups), dtype=np.float64, order="F")
    for g in range(groups):
        w0, w1, w2, w3 = philox4x32_10(j & MASK32, j >> np.uint64(32),
                                       np.full(rows, g, dtype=np.uint64),
                                       np.full(rows, stream, dtype=np.uint64), k0, k1)
        z0, z1 = _box_muller(w0, w1)
        z2, z3 = _box_muller(w2, w3)
        out[:, 4 * g + 0] = z0
        out[:, 4 * g + 1] = z1
        out[:, 4 * g + 2] = z2
        out[:, 4 * g + 3] = z3
    return np.asfortranarray(out[:, :cols].astype(np.float32))
