"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This package only draws and assembles input data (tensors and explicit Gaussian
test matrices).  It contains none of the decomposition arithmetic, so both the
CUDA path and the FP64 oracle can consume its outputs without sharing code.
"""
from .synthetic import *  # noqa: F401,F403
