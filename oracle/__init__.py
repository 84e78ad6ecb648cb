"""FP64 CPU oracle for the randomized HOSVD / Tucker hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library never
calls it and shares no code with it: the oracle is a plain, slow restatement of
the paper's definitions and algorithms (NumPy, FP64, LAPACK through NumPy), used
to check the GPU results.

Modules
-------
tensor      n-unfolding, folding and n-mode products (Sec. 2)
philox      Philox4x32-10 counter generator + Box-Muller (the Gaussian test
            matrices the GPU draws from a seed)
algorithms  orth, Alg. 1 (randomized SVD with oversampling and power iteration),
            truncated HOSVD, STHOSVD (Alg. 4), one HOOI sweep (Alg. 5),
            RP-HOSVD (Alg. 6), R-STHOSVD (Alg. 8), R-PET (Alg. 9)
metrics     relative error (Eq. "Relativeerror", explicit residual), principal
            angles between subspaces, orthonormality

Every function is pinned by tests under ``tests/test_oracle_*.py`` against
brute force, closed forms, invariants or the values printed in Table 1.
"""
