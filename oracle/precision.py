"""Reduced-precision number formats and the per-slice scaling of X (TEST
INFRASTRUCTURE ONLY, like the rest of ``oracle``).

The reduced-precision form of the hot path keeps a copy of X in BF16 or in FP8
e4m3 and runs its sketch contractions on that copy with FP32 accumulation.
The oracle needs the formats only to build the inputs both sides share: the
test matrices of a reduced-precision run are themselves rounded to the
format, so that the GPU's products are exact in it and the oracle can be given
the identical values.  Definitions:

* BF16: the upper 16 bits of an FP32 value (8 exponent bits, 7 stored mantissa
  bits), round to nearest, ties to even.
* FP8 e4m3 (the OCP 8-bit "E4M3" format): 4 exponent bits with bias 7, 3
  mantissa bits, subnormals with spacing 2^-9, largest finite value 448, no
  infinities; round to nearest, ties to even, saturating at +-448.
* per-slice scale of X (e4m3 only): X is cut into its frontal slices along the
  last mode, and slice k is stored as e4m3(X[..., k] / s_k) with s_k the
  smallest power of two for which the slice's largest magnitude divided by s_k
  is at most 448.  A power of two keeps s_k * e4m3 value exact in FP32 and BF16.
  BF16 has the exponent range of FP32 and needs no scale.
"""
from __future__ import annotations

import numpy as np

E4M3_MAX = 448.0


def bf16_round(a) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned in FP64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    r = ((u + (((u >> 16) & 1) + 0x7FFF)) & 0xFFFF0000).view(np.float32).astype(np.float64)
    return r.reshape(np.shape(a))


def e4m3_round(a) -> np.ndarray:
    """Round to FP8 e4m3 (bias 7, 3 mantissa bits, largest 448, subnormal spacing
    2^-9), ties to even, saturating at 448; returned in FP64."""
    a = np.asarray(a, dtype=np.float64)
    m = np.minimum(np.abs(a), E4M3_MAX)
    e = np.maximum(np.floor(np.log2(np.maximum(m, 2.0 ** -9))), -6.0)
    step = 2.0 ** (e - 3)
    return np.sign(a) * np.minimum(np.round(m / step) * step, E4M3_MAX)


def round_to(a, dtype: str) -> np.ndarray:
    """Values of `a` rounded to 'f32', 'bf16' or 'e4m3', in FP64."""
    if dtype == "f32":
        return np.asarray(a, dtype=np.float32).astype(np.float64)
    if dtype == "bf16":
        return bf16_round(a)
    if dtype == "e4m3":
        return e4m3_round(a)
    raise ValueError(dtype)


def slice_scales(x: np.ndarray) -> np.ndarray:
    """Power-of-two scale per frontal slice of the last mode: the smallest 2^e
    with max|X[..., k]| / 2^e <= 448 (2^0 for an all-zero slice)."""
    x = np.asarray(x, dtype=np.float64)
    amax = np.max(np.abs(x.reshape(-1, x.shape[-1], order="F")), axis=0)
    e = np.where(amax > 0, np.ceil(np.log2(np.where(amax > 0, amax, 1.0) / E4M3_MAX)), 0.0)
    s = 2.0 ** e
    # ceil(log2) can land one short when amax / 448 sits just above a power of two
    s = np.where(amax / s > E4M3_MAX, 2 * s, s)
    return s


def quantize(x: np.ndarray, dtype: str):
    """The reduced-precision copy of X as the GPU keeps it, dequantized to FP64:
    (values, per-slice scales).  'bf16' rounds every entry (scales 1); 'e4m3'
    rounds X[..., k] / s_k and multiplies back."""
    x = np.asarray(x, dtype=np.float64)
    if dtype == "bf16":
        return bf16_round(x.astype(np.float32)).reshape(x.shape), np.ones(x.shape[-1])
    if dtype == "e4m3":
        s = slice_scales(x)
        return np.asfortranarray(e4m3_round(x / s) * s), s
    if dtype == "f32":
        return x, np.ones(x.shape[-1])
    raise ValueError(dtype)
