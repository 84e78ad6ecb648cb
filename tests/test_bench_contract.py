"""The benchmark's reference arm (the FP64 oracle on the host cores) keeps the
JSON-line contract: one line from rank 0 with the metric, unit, step counts,
CPU-baseline and end-to-end objects; nothing from the other ranks."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(extra_env=None, *args):
    env = dict(os.environ)
    env.update(extra_env or {})
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "lowrank100_rhosvd",
           "--steps", "2", "--warmup", "3", *args]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _bench()
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["steps"] == 2 and d["steps_requested"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["value"] > 0
    assert abs(d["ms_per_step"] - 1e3 / d["value"]) <= 1e-6 * d["ms_per_step"]
    assert d["config"]["workload"] == "lowrank100_rhosvd"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_is_silent_on_other_ranks():
    r = _bench({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, "--gpus", "2")
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [l for l in r.stdout.splitlines() if l.strip().startswith("{")], r.stdout


def test_accuracy_report_separates_subspace_and_orthonormality():
    """The error gate on a small decomposition: the oracle's own result passes with
    zero sines, and factors scaled off orthonormality (same subspaces) keep
    E_lsq_core at the oracle's E while E_transpose_core grows."""
    import numpy as np
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    from oracle import algorithms as A
    from oracle import tensor as T
    from workloads import gaussian_matrix, lowrank_tensor
    dims, ranks = (14, 12, 10), (3, 4, 2)
    x = lowrank_tensor(dims, ranks, 5, noise=1e-3)
    om = [gaussian_matrix(40 + n, r, c).astype(np.float64)
          for n, (r, c) in enumerate(A.omega_shapes("rsthosvd", dims, ranks, 4))]
    g, us = A.rsthosvd(x, ranks, 1, om)
    rep = bench.accuracy_report(x, g, us, g, us)
    assert rep["pass"] and rep["E_gpu"] == rep["E_oracle"]
    assert max(rep["sine_per_mode"]) < 1e-7 and max(rep["orthonormality_per_mode"]) < 1e-12
    assert abs(rep["E_lsq_core"] - rep["E_oracle"]) < 1e-9 and abs(rep["E_transpose_core"] - rep["E_oracle"]) < 1e-9
    assert abs(rep["core_scale_minus_1"]) < 1e-12 and max(map(abs, rep["column_norm_minus_1_per_mode"])) < 1e-12
    short = bench.accuracy_report(x, g * (1 - 1e-3), us, g, us)          # a uniformly shortened core
    assert abs(short["core_scale_minus_1"] + 1e-3) < 1e-12
    bent = [u * (1 + 1e-3 * np.arange(u.shape[1])) for u in us]       # same columns' directions, wrong lengths
    rep = bench.accuracy_report(x, T.multi_ttm(x, bent, transpose=True), bent, g, us)
    assert max(rep["sine_per_mode"]) < 1e-7
    # column k of mode n has length 1 + 1e-3 k: the largest departure is mode 2's last column
    assert abs(max(rep["orthonormality_per_mode"]) - (1.003 ** 2 - 1)) < 1e-9
    assert abs(rep["E_lsq_core"] - rep["E_oracle"]) < 1e-10
    assert rep["E_transpose_core"] > 1.5 * rep["E_oracle"]
    assert rep["E_gpu"] == rep["E_transpose_core"] and not rep["pass"]
