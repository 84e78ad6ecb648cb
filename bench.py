"""Benchmark: randomized Tucker decompositions per second on one GB300 per rank.

Default workload: 512^3 FP32 tensor of multilinear rank (32,32,32) with a
0.9^(i+j+k) core decay and 1e-4 relative noise, decomposed by R-STHOSVD
(Alg. 8) with oversampling p = 10 and q = 1 power iteration, test matrices
drawn on the device from seed 0.  One step = one full decomposition (all
modes: Omega generation, sketches, power-iteration TTMs, orthonormalisations,
projections, truncations, core).  X (512 MiB) is larger than L2, so no flush is
needed between steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on the host cores instead (the comparison arm of this project).
``--serve N`` runs the serving loop (paper_2001_07124_gb300/serving.py) on N
Poisson-arriving requests (200 req/s; cubic sizes log-uniform in [64, 768] on
multiples of 64; ranks uniform in 8..64; R-STHOSVD p = 10, q = 1; 150 GB device
budget) with 4 slots and, for comparison, with 1 slot; its JSON line reports
p50/p99 latency and decomps/s (not the benchmark line).
``--batch N`` decomposes N independent small tensors (mode sizes uniform in
[16, 96], ranks uniform in [4, 16] capped at the mode size, p = 5, q = 1,
low rank plus 1e-3 noise) with a per-tensor launch loop and with
rhosvd.BatchGraph (CUDA graphs of 512 decompositions on 16 parallel branches);
its JSON line reports both rates (not the benchmark line).
``--primitive sketch|power|orth`` times one C-ABI primitive on the workload's
mode-1 shapes instead (a kernel micro-benchmark for profiling; its line is not
the benchmark line): sketch = rhosvd_sketch(X, mode 1, Omega_1), power =
rhosvd_power (TTM, CholeskyQR2 of Z, sketch), orth = rhosvd_orth of a J_1 x K_1
Gaussian matrix.
Multi-GPU: every rank decomposes its own tensor (independent replicas, no
data-path collective); value = all decompositions / slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

_CORES = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, str(_CORES))

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import WORKLOADS, device_layout  # noqa: E402

_ALGO_NAMES = {"rhosvd": "RP-HOSVD", "rsthosvd": "R-STHOSVD", "rpet": "R-PET"}


def slowest_rank_ms(local_ms: float, dist=None, device="cpu") -> float:
    """The timed region's length for the whole job: every rank contributes its own
    elapsed time and all of them receive the maximum (one all-reduce)."""
    if dist is None:
        return float(local_ms)
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(steps: int, world: int, elapsed_ms: float) -> float:
    """Whole-job units per second: every rank's steps over the slowest rank's time
    (replicas: each rank decomposes its own tensor, so the work grows with N)."""
    return world * steps / (elapsed_ms / 1e3)


def replica_workload(w, rank: int):
    """The workload a rank decomposes: the same shapes with its own data seed."""
    import dataclasses
    return dataclasses.replace(w, seed=w.seed + rank)


def _l2_note(w) -> str:
    mib = 4 * int(np.prod(w.dims)) / 2 ** 20
    if mib * 2 ** 20 > 129e6:
        return f"input {mib:.0f} MiB > 129 MB L2"
    return f"input {mib:.1f} MiB fits in L2 (not flushed)"


def metric_name(w, dtype="f32", refine=0, kron=False) -> str:
    """Metric label of a workload, e.g. decomps/s (R-STHOSVD 512^3 FP32, rank 32, p=10, q=1)."""
    d = w.dims
    shape = f"{d[0]}^{len(d)}" if len(set(d)) == 1 else "x".join(str(v) for v in d)
    r = w.ranks
    rank = str(r[0]) if len(set(r)) == 1 else "(" + ",".join(str(v) for v in r) + ")"
    par = f"K={w.K[0]}, S={w.S[0]}" if w.algo == "rpet" and w.K else f"p={w.p}, q={w.q}"
    extra = ", Kronecker factor sketches" if kron else ""
    extra += "" if dtype == "f32" else f", {dtype.upper()} sketch passes"
    extra += f", {refine} RP-HOOI sweep" + ("s" if refine > 1 else "") if refine else ""
    return f"decomps/s ({_ALGO_NAMES[w.algo]} {shape} FP32, rank {rank}, {par}{extra})"
UNIT = "decomps/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        except OSError:
            pass
        finally:
            if self.path:
                try:
                    os.unlink(self.path)
                except OSError:
                    pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


def _traffic_for(kernel_src: str, key: str):
    """DRAM bytes per launch from the committed ncu summary, valid only for the
    kernel source it was captured on (null otherwise)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        data = json.load(open(path))
    except (OSError, ValueError):
        return None
    h = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
    ent = data.get(key)
    if not ent or ent.get("source_sha") != h:
        return None
    return ent.get("bytes_per_launch")


def accuracy_report(x32, g_gpu, u_gpu, g_or, u_or, tol=1e-5, max_sine=1e-4) -> dict:
    """The error gate of a bench line: E_gpu against E_oracle (explicit FP64
    residuals on the same FP32 input) and the largest principal-angle sine between
    the two sets of factors. Beside it, what separates the causes of an excess:
    per mode the factors' orthonormality, mean column length and sine; the scale
    of the device's core against X x_n U_n^T (a systematic shortening of the
    products shows there); and E for two FP64 cores of the device's factors,
    X x_n pinv(U_n) (subspaces only) and X x_n U_n^T (what the device's
    projection computes in exact arithmetic)."""
    from oracle import metrics as M
    from oracle import tensor as T
    e_gpu = M.rel_error(x32, g_gpu, u_gpu)
    e_or = M.rel_error(x32, g_or, u_or)
    sines = [M.max_principal_sine(a, b) for a, b in zip(u_gpu, u_or)]
    sine = max(sines)
    g_t = T.multi_ttm(x32, u_gpu, transpose=True)
    return {"E_gpu": e_gpu, "E_oracle": e_or, "max_principal_sine": sine,
            "pass": bool(abs(e_gpu - e_or) <= tol and sine <= max_sine),
            "sine_per_mode": sines,
            "orthonormality_per_mode": [M.orthonormality(u) for u in u_gpu],
            "column_norm_minus_1_per_mode": [float(np.mean(np.linalg.norm(u, axis=0)) - 1) for u in u_gpu],
            "core_scale_minus_1": float(np.sum(g_gpu * g_t) / np.sum(g_t * g_t) - 1),
            "E_lsq_core": M.rel_error(x32, T.multi_ttm(x32, [np.linalg.pinv(u) for u in u_gpu]), u_gpu),
            "E_transpose_core": M.rel_error(x32, g_t, u_gpu)}


def oracle_decompose(w, x32, dtype="f32", refine=0, kron=False):
    """Time one oracle decomposition (FP64 NumPy) with the generator's own test
    matrices (rounded to the format of a reduced-precision run, as the device
    rounds its own) and the same number of RP-HOOI sweeps."""
    from oracle import algorithms as A
    from oracle import philox
    from oracle.precision import round_to
    shapes = A.omega_shapes(w.algo, w.dims, w.ranks, w.p, K=w.K, S=w.S)
    N = len(w.dims)
    rnd = (lambda a: round_to(a, dtype)) if (dtype != "f32" and w.algo == "rpet") else (lambda a: a)
    t0 = time.perf_counter()
    if w.algo == "rpet" and kron:
        # Kronecker-structured factor sketches: Phi_p on stream_id 10N + p, k from the plan's K_n = k^(N-1)
        fs, ts = shapes
        from paper_2001_07124_gb300 import rhosvd as R
        Kp, Sp, _ = R.rhosvd_plan(w.dims, w.ranks, "rpet", w.p, w.q, K=w.K, S=w.S, kron=True)
        k = int(round(Kp[0] ** (1.0 / (N - 1))))
        phis = [philox.omega(w.omega_seed, 10 * N + p, w.dims[p], k).astype(np.float64) for p in range(N)]
        om = [A.kronecker_test_matrix(phis, n) for n in range(N)]
        ot = [philox.omega(w.omega_seed, N + n, Sp[n], w.dims[n]).astype(np.float64) for n in range(N)]
        t0 = time.perf_counter()
        g, u, _ = A.rpet(x32, w.ranks, om, ot)
    elif w.algo == "rpet":
        fs, ts = shapes
        om = [rnd(philox.omega(w.omega_seed, n, r, c).astype(np.float64)) for n, (r, c) in enumerate(fs)]
        ot = [rnd(philox.omega(w.omega_seed, N + n, r, c).astype(np.float64)) for n, (r, c) in enumerate(ts)]
        g, u, _ = A.rpet(x32, w.ranks, om, ot)
    else:
        om = [philox.omega(w.omega_seed, n, r, c).astype(np.float64) for n, (r, c) in enumerate(shapes)]
        g, u = getattr(A, w.algo)(x32, w.ranks, w.q, om)
    for t in range(refine):
        ref = [philox.omega(w.omega_seed, 2 * N + t * N + n, j, k).astype(np.float64)
               for n, (j, k) in enumerate(A.rp_hooi_omega_shapes(w.dims, w.ranks, w.p))]
        g, u = A.rp_hooi_sweep(x32, u, w.ranks, ref)
    return time.perf_counter() - t0, g, u


def run_reference(args, w, rank):
    if rank != 0:
        return
    x = w.tensor()
    x32 = np.asfortranarray(x.astype(np.float32).astype(np.float64))
    del x
    # one oracle decomposition takes about a second on 512^3: the warm-up steps
    # time it, and the timed steps are capped so that the run stays near two
    # minutes whatever --steps asks for (the rate does not depend on the count)
    t_warm = [oracle_decompose(w, x32)[0] for _ in range(max(1, min(args.warmup, 3)))]
    steps = max(1, min(args.steps, int(120.0 / max(min(t_warm), 1e-3))))
    times = [oracle_decompose(w, x32)[0] for _ in range(steps)]
    total = sum(times)
    value = steps / total
    line = {
        "impl": "reference", "metric": metric_name(w), "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": steps, "steps_requested": args.steps, "warmup": len(t_warm), "ms_per_step": 1e3 * total / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded low-rank tensor, seeded Philox test matrices)",
        "config": {"workload": w.name, "dims": list(w.dims), "ranks": list(w.ranks), "p": w.p, "q": w.q,
                   "algo": w.algo, "l2_flush": _l2_note(w)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": _CORES, "kind": "oracle",
                         "sample": f"full workload, {steps} decompositions"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_serving(args):
    """Poisson request stream through the serving loop, 4 slots vs 1 slot."""
    import torch
    import paper_2001_07124_gb300 as pkg
    from paper_2001_07124_gb300 import serving
    pkg.build()
    rng = np.random.default_rng(1005)
    n = args.serve
    rate = float(args.serve_rate)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n))
    sizes = np.clip(np.rint(np.exp(rng.uniform(np.log(64), np.log(768), size=n)) / 64) * 64, 64, 768).astype(int)
    ranks = np.minimum(rng.integers(8, 65, size=n), sizes)
    # half of the requests are fixed-accuracy ones (eps 1e-2 on a core with a 0.9^(i+j+k)
    # decay and 1e-4 noise; ranks found on the device), half fixed-rank
    fixed_acc = (np.arange(n) % 2) == 1
    # one low-rank-plus-noise tensor per size and kind, drawn on the device and kept in pinned host memory
    pool = {}
    pool_acc = {}
    g = torch.Generator(device="cuda")
    for I in sorted(set(sizes.tolist())):
        g.manual_seed(1005 + I)
        r = 64
        core = torch.randn(r, r, r, device="cuda", generator=g)
        U = [torch.linalg.qr(torch.randn(I, r, device="cuda", generator=g))[0] for _ in range(3)]
        x = torch.einsum("abc,ia,jb,kc->kji", core, U[0], U[1], U[2])      # (k, j, i): i fastest
        noise = torch.randn(x.shape, device="cuda", generator=g)
        x = x + 1e-3 * x.norm() / noise.norm() * noise
        pool[I] = x.contiguous().reshape(-1).cpu().pin_memory()
        del x, noise
        ii = torch.arange(r, device="cuda", dtype=torch.float32)
        decay = 0.9 ** (ii[:, None, None] + ii[None, :, None] + ii[None, None, :])
        xa = torch.einsum("abc,ia,jb,kc->kji", core * decay, U[0], U[1], U[2])
        noise = torch.randn(xa.shape, device="cuda", generator=g)
        xa = xa + 1e-4 * xa.norm() / noise.norm() * noise
        pool_acc[I] = xa.contiguous().reshape(-1).cpu().pin_memory()
        del xa, noise, core, U
    torch.cuda.empty_cache()

    def requests():
        out = []
        for i in range(n):
            I = int(sizes[i])
            if fixed_acc[i]:
                out.append(serving.Request(i, (I,) * 3, (int(ranks[i]),) * 3, float(arrivals[i]), x_host=pool_acc[I],
                                           seed=i, tol=1e-2, block=16, k_max=(min(I, 96),) * 3))
            else:
                out.append(serving.Request(i, (I,) * 3, (int(ranks[i]),) * 3, float(arrivals[i]), x_host=pool[I],
                                           p=10, q=1, seed=i))
        return out

    # warm-up: the whole stream once, untimed, so that kernel attributes, the
    # device and pinned-host caching allocators and the per-size workspaces are
    # settled before either timed run (otherwise the first run pays for them)
    serving.serve(requests(), slots=4, budget_bytes=150 * 10 ** 9)
    line = {"mode": "serve", "requests": n, "arrival_rate_per_s": rate,
            "sizes": "cubic, log-uniform in [64, 768], multiples of 64", "ranks": "uniform 8..64",
            "algo": "half R-STHOSVD p=10 q=1 (fixed rank), half fixed-accuracy R-STHOSVD eps=1e-2 "
                    "(blocked range finder, block 16, k_max 96)", "budget_gb": 150}
    for slots in (4, 1):
        res = serving.serve(requests(), slots=slots, budget_bytes=150 * 10 ** 9)
        line[f"slots{slots}"] = serving.latency_summary(res)
        acc = [r for r in res if fixed_acc[r.rid]]
        if acc:
            line[f"slots{slots}"]["fixed_accuracy"] = serving.latency_summary(acc)
            line[f"slots{slots}"]["fixed_accuracy"]["mean_rank"] = float(np.mean([r.ranks[0] for r in acc]))
        rk = [r for r in res if not fixed_acc[r.rid]]
        if rk:
            line[f"slots{slots}"]["fixed_rank"] = serving.latency_summary(rk)
    if not args.no_cpu_baseline:
        # the FP64 oracle on one fixed-rank request (rank 32, p = 10, q = 1) per size bucket
        # of the stream, one after another on the host cores
        from oracle import algorithms as A
        from oracle import philox
        per_size = {}
        for I in (64, 128, 256, 512, 768):
            if I not in pool:
                continue
            x = pool[I].numpy().astype(np.float64).reshape((I, I, I), order="F")
            rk3 = (min(32, I),) * 3
            t0 = time.perf_counter()
            om = [philox.omega(0, m, r, c).astype(np.float64)
                  for m, (r, c) in enumerate(A.omega_shapes("rsthosvd", (I,) * 3, rk3, 10))]
            A.rsthosvd(x, rk3, 1, om)
            per_size[str(I)] = time.perf_counter() - t0
            del x
        if per_size:
            line["cpu_baseline"] = {"value": len(per_size) / sum(per_size.values()), "unit": "requests/s",
                                    "cores": _CORES, "kind": "oracle",
                                    "sample": "one fixed-rank request (rank 32) per size bucket, serially",
                                    "seconds_per_request": per_size}
    print(json.dumps(line), flush=True)


def run_batch(args):
    """N small independent decompositions: per-tensor launch loop vs batched CUDA graphs."""
    import torch
    import paper_2001_07124_gb300 as pkg
    from paper_2001_07124_gb300 import rhosvd as R
    pkg.build()
    R.lib()
    n = args.batch
    rng = np.random.default_rng(1004)
    g = torch.Generator(device="cuda")
    g.manual_seed(1004)
    items = []
    for b in range(n):
        dims = tuple(int(v) for v in rng.integers(16, 97, size=3))
        ranks = tuple(int(min(r, d)) for r, d in zip(rng.integers(4, 17, size=3), dims))
        core = torch.randn(*ranks, device="cuda", generator=g)
        # the orthonormal factors come from a host QR (the device linear-algebra
        # library does not load under the profiler)
        U = [torch.linalg.qr(torch.randn(d, r, device="cuda", generator=g).cpu())[0].cuda()
             for d, r in zip(dims, ranks)]
        x = torch.einsum("abc,ia,jb,kc->kji", core, U[0], U[1], U[2])
        noise = torch.randn(x.shape, device="cuda", generator=g)
        x = x + 1e-3 * x.norm() / noise.norm() * noise
        items.append((x.contiguous().reshape(-1), dims, ranks))
    kw = dict(algo="rsthosvd", p=5, q=1, seed=0)
    # one persistent launch over the whole batch, its launch shape picked by the tuner
    persistent = R.BatchPersistent(items, **kw)
    tune_ms = persistent.tune()

    def run_persistent():
        persistent.run()

    # per-tensor launch loop (each tensor its own workspace and outputs, one stream)
    loop = []
    for X, dims, ranks in items:
        ws = R.Workspace(R.rhosvd_workspace_size(dims, ranks, "rsthosvd", 5, 1))
        out = (R.empty_colmajor(ranks), [R.empty_colmajor((d, r)) for d, r in zip(dims, ranks)])
        loop.append((X, dims, ranks, ws, out))

    def run_loop():
        for X, dims, ranks, ws, out in loop:
            R.rhosvd_decompose(X, dims, ranks, ws=ws, out=out, check=False, **kw)

    chunk = 512
    graphs = [R.BatchGraph(items[i:i + chunk], branches=16, **kw) for i in range(0, n, chunk)]

    def run_graphs():
        for gr in graphs:
            gr.replay()

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rates = {}
    for name, fn in (("persistent", run_persistent), ("per_tensor_loop", run_loop), ("batch_graph", run_graphs)):
        fn()
        torch.cuda.synchronize()
        reps = 3
        t0 = time.perf_counter()
        ev0.record()
        for _ in range(reps):
            fn()
        ev1.record()
        torch.cuda.synchronize()
        wall = (time.perf_counter() - t0) / reps
        rates[name] = {"decomps_per_s": n / (ev0.elapsed_time(ev1) / reps / 1e3), "wall_s_per_batch": wall}
    # the two forms compute the same decompositions
    same = True
    for gr, lo in zip(graphs, [loop[i:i + chunk] for i in range(0, n, chunk)]):
        for it_g, it_l in zip(gr.items, lo):
            (Gg, Ug), (Gl, Ul) = it_g[4], it_l[4]            # flat column-major output buffers
            same &= bool(torch.equal(Gg, Gl)) and all(bool(torch.equal(a, b)) for a, b in zip(Ug, Ul))
    status = max(max(gr.device_status() for gr in graphs), persistent.device_status())
    # accuracy of the persistent form against the graph form (same algorithm and
    # test matrices, different FP32 arithmetic): relative errors on every item

    def rel_err(X, dims, G, Us):
        Xh = torch.einsum("abc,ia,jb,kc->kji", G.double(), Us[0].double(), Us[1].double(), Us[2].double())
        x = X.reshape(dims[2], dims[1], dims[0]).double()
        return float((x - Xh).norm() / x.norm())

    e_graph, e_pers = [], []
    for gr in graphs:
        for (g, us), it in zip(gr.results(), gr.items):
            e_graph.append(rel_err(it[0], it[1], g, us))
    for (g, us), it in zip(persistent.results(), persistent.items):
        e_pers.append(rel_err(it[0], it[1], g, us))
    e_graph, e_pers = np.array(e_graph), np.array(e_pers)
    cpu = None
    if not args.no_cpu_baseline:
        # the FP64 oracle's R-STHOSVD (same test matrices) on the first 64 tensors, one after another
        from oracle import algorithms as A
        from oracle import philox
        ns = min(n, 64)
        hosts = [(X.double().cpu().numpy().reshape(dims, order="F"), dims, rk) for X, dims, rk in items[:ns]]
        t0 = time.perf_counter()
        for x, dims, rk in hosts:
            om = [philox.omega(0, m, r, c).astype(np.float64)
                  for m, (r, c) in enumerate(A.omega_shapes("rsthosvd", dims, rk, 5))]
            A.rsthosvd(x, rk, 1, om)
        cpu = {"value": ns / (time.perf_counter() - t0), "unit": "decomps/s", "cores": _CORES, "kind": "oracle",
               "sample": f"the first {ns} of the {n} tensors, one after another (FP64 NumPy)"}
    print(json.dumps({"mode": "batch", "tensors": n, "sizes": "each mode uniform in [16, 96]",
                      "ranks": "uniform in [4, 16], capped", "algo": "rsthosvd p=5 q=1",
                      "graph_chunk": chunk, "branches": 16, **rates,
                      "speedup": rates["batch_graph"]["decomps_per_s"] / rates["per_tensor_loop"]["decomps_per_s"],
                      "speedup_persistent_vs_graph": rates["persistent"]["decomps_per_s"]
                      / rates["batch_graph"]["decomps_per_s"],
                      "persistent_config": persistent.config, "tune_best_ms": tune_ms,
                      "identical_results": same,
                      "rel_error_graph_mean": float(e_graph.mean()),
                      "rel_error_persistent_mean": float(e_pers.mean()),
                      "rel_error_max_abs_diff": float(np.max(np.abs(e_pers - e_graph))),
                      "device_status": status, "cpu_baseline": cpu}), flush=True)


def run_primitive(args, w):
    """Time one primitive on one mode of the workload (device-drawn inputs):
    sketch (explicit Omega), power step, orthonormalisation of a J_n x K_n matrix,
    or the core TTM chain with widths K_n (S_n for a single-pass workload)."""
    import torch
    import paper_2001_07124_gb300 as pkg
    from paper_2001_07124_gb300 import rhosvd as R
    pkg.build()
    R.lib()
    dims = w.dims
    n = args.mode - 1
    if not 0 <= n < len(dims):
        raise SystemExit(f"--mode must be in 1..{len(dims)}")
    Kp, _, _ = R.rhosvd_plan(dims, w.ranks, w.algo, w.p, w.q, K=w.K, S=w.S)
    Kn, In = Kp[n], dims[n]
    Jn = int(np.prod(dims)) // In
    g = torch.Generator(device="cuda")
    g.manual_seed(w.seed)
    ws = R.Workspace(R.rhosvd_primitive_workspace_size(dims, max(Kp)))
    X = torch.randn(int(np.prod(dims)), device="cuda", generator=g)
    if args.primitive == "sketch":
        om = R.rhosvd_omega(w.omega_seed, n, Jn, Kn).t().contiguous().reshape(-1)
        Y = R.empty_colmajor((In, Kn))
        call = lambda: R.rhosvd_sketch(X, dims, n, Kn, Omega=om, Y=Y, ws=ws)
    elif args.primitive == "power":
        Q, _ = R.rhosvd_orth(torch.randn(In, Kn, device="cuda", generator=g), ws=ws)
        call = lambda: R.rhosvd_power(X, dims, n, Q.clone(), ws=ws)
    elif args.primitive == "orth":
        del X
        Z = torch.randn(Kn, Jn, device="cuda", generator=g).t()
        call = lambda: R.rhosvd_orth(Z, ws=ws)
    else:
        widths = list(w.S) if w.S else list(Kp)
        Qs = [R.rhosvd_orth(torch.randn(dims[m], widths[m], device="cuda", generator=g), ws=ws)[0]
              for m in range(len(dims))]
        t, mt = list(dims), 1
        for m in range(len(dims)):
            t[m] = widths[m]
            mt = max(mt, int(np.prod(t)))
        cws = R.Workspace(256 + 2 * (mt * 4 + 256))
        call = lambda: R.rhosvd_core(X, dims, Qs, ws=cws)
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        call()
    ev1.record()
    torch.cuda.synchronize()
    print(json.dumps({"primitive": args.primitive, "workload": w.name, "mode": args.mode, "K": Kn,
                      "ms_per_call": ev0.elapsed_time(ev1) / args.steps, "calls": args.steps}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="decay512_rsthosvd", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--primitive", choices=["sketch", "power", "orth", "core"], default=None)
    ap.add_argument("--mode", type=int, default=1, help="mode (1-based) of --primitive sketch/power/orth")
    ap.add_argument("--no-graph", action="store_true", help="launch the decomposition kernel by kernel")
    ap.add_argument("--serve", type=int, default=0, metavar="N", help="serving run with N requests")
    ap.add_argument("--serve-rate", type=float, default=200.0, metavar="R", help="Poisson arrival rate (req/s)")
    ap.add_argument("--batch", type=int, default=0, metavar="N", help="batched run with N small tensors")
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16", "e4m3"],
                    help="arithmetic of the sketch passes (reduced-precision copy of X)")
    ap.add_argument("--refine", type=int, default=0, help="RP-HOOI sweeps after the decomposition")
    ap.add_argument("--kron", action="store_true", help="R-PET with Kronecker-structured factor sketches")
    ap.add_argument("--concurrent", type=int, default=8, metavar="P",
                    help="independent decompositions in flight per step (each its own tensor)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    w = WORKLOADS[args.workload]

    if args.impl == "reference":
        return run_reference(args, w, rank)
    if args.primitive is not None:
        return run_primitive(args, w)
    if args.serve > 0:
        return run_serving(args)
    if args.batch > 0:
        return run_batch(args)

    import torch
    import paper_2001_07124_gb300 as pkg
    from paper_2001_07124_gb300 import rhosvd as R

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pkg.build()
    R.lib()

    # each replica decomposes its own tensor (data seed + rank)
    wr = replica_workload(w, rank)
    x = wr.tensor()
    x_host = torch.from_numpy(device_layout(x))
    x32 = None
    if rank == 0 and not args.no_cpu_baseline:
        x32 = np.asfortranarray(x.astype(np.float32).astype(np.float64))
    del x
    X = x_host.cuda()
    dims, ranks = w.dims, w.ranks
    P = max(1, int(args.concurrent))
    kw = dict(algo=w.algo, p=w.p, q=w.q, seed=w.omega_seed, K=w.K, S=w.S, dtype=args.dtype, refine=args.refine,
              kron=args.kron)
    need = R.rhosvd_workspace_size(dims, ranks, w.algo, w.p, w.q, K=w.K, S=w.S, dtype=args.dtype,
                                   refine=args.refine, kron=args.kron)
    stream = torch.cuda.current_stream()

    def new_outputs():
        return (R.empty_colmajor(ranks), [R.empty_colmajor((dims[n], ranks[n])) for n in range(len(dims))])

    # P independent decompositions per step, each on its own tensor (a copy of the
    # workload's), workspace and outputs; graph form: one graph, P parallel branches
    Xs = [X] + [X.clone() for _ in range(P - 1)]
    wss = [R.Workspace(need) for _ in range(P)]
    outs = [new_outputs() for _ in range(P)]
    side = [torch.cuda.Stream() for _ in range(P)]

    def eager_set(xs, wsl, outl):
        def run():
            for s_ in side:
                s_.wait_stream(stream)
            for b in range(P):
                R.rhosvd_decompose(xs[b], dims, ranks, ws=wsl[b], out=outl[b], check=False, stream=side[b], **kw)
            for s_ in side:
                stream.wait_stream(s_)
        return run

    def graph_set(xs, wsl, outl):
        g_ = R.BatchGraph([(xs[b], dims, ranks) for b in range(P)], branches=P, warmup=1, **kw)
        # the graph keeps its own workspaces and outputs; point the set's lists at them
        for b in range(P):
            wsl[b] = g_.items[b][3]
            outl[b] = g_.items[b][4]
        return g_.replay

    for _ in range(args.warmup):
        eager_set(Xs, wss, outs)()
    step = eager_set(Xs, wss, outs) if args.no_graph else graph_set(Xs, wss, outs)
    for _ in range(2):
        step()
    torch.cuda.synchronize()
    ws, out = wss[0], outs[0]
    G, Us = out
    for b in range(P):
        code, flags = R.rhosvd_device_status(wss[b])
        if code != 0:
            raise RuntimeError(f"device status {code} after warm-up")
    # code, flags, orth_fail, fallbacks, fallback_rows, eig_sweeps
    st_words = ws.buf[:24].view(torch.int32).cpu().tolist()

    def barrier():
        if dist is not None:
            dist.barrier()

    # ---------------------------------------------------------------- timed region (device)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    elapsed_ms = slowest_rank_ms(ev0.elapsed_time(ev1), dist, "cuda")
    clocks = clk.summary()
    for b in range(P):
        code, _ = R.rhosvd_device_status(wss[b])
        if code != 0:
            raise RuntimeError(f"device status {code} in timed region")
    value = job_rate(args.steps * P, world, elapsed_ms)

    # latency of one decomposition alone (one graph launch, nothing else in flight)
    single = R.DecomposeGraph(X, dims, ranks, ws=R.Workspace(need), out=new_outputs(), warmup=1, **kw)
    for _ in range(3):
        single.replay()
    torch.cuda.synchronize()
    lat_reps = max(5, min(args.steps, 100))
    ev0.record(stream)
    for _ in range(lat_reps):
        single.replay()
    ev1.record(stream)
    torch.cuda.synchronize()
    single_ms = ev0.elapsed_time(ev1) / lat_reps
    del single

    # ---------------------------------------------------------------- e2e through host buffers
    # Every step copies its P tensors from pinned host memory and reads their factors
    # and cores back.  Two device sets alternate: step i's host-to-device copies run on
    # a copy stream while step i-1 computes (the usual double buffering a caller does).
    xh = x_host.pin_memory()
    nbuf = 2
    sets = [(Xs, wss, outs, step)]
    for _ in range(nbuf - 1):
        xs2 = [torch.empty_like(X) for _ in range(P)]
        ws2 = [R.Workspace(need) for _ in range(P)]
        out2 = [new_outputs() for _ in range(P)]
        run2 = eager_set(xs2, ws2, out2) if args.no_graph else graph_set(xs2, ws2, out2)
        sets.append((xs2, ws2, out2, run2))
    host_out = [[(torch.empty(G.numel(), dtype=torch.float32).pin_memory(),
                  [torch.empty(u.numel(), dtype=torch.float32).pin_memory() for u in Us]) for _ in range(P)]
                for _ in range(nbuf)]
    copy_stream = torch.cuda.Stream()
    h2d_done = [torch.cuda.Event() for _ in range(nbuf)]
    buf_free = [torch.cuda.Event() for _ in range(nbuf)]
    for e in buf_free:
        e.record(stream)

    def e2e_step(i):
        bset = i % nbuf
        xs_b, _, outs_b, run_b = sets[bset]
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(buf_free[bset])       # step i - nbuf has finished with this set
            for xb in xs_b:
                xb.copy_(xh, non_blocking=True)
            h2d_done[bset].record(copy_stream)
        stream.wait_event(h2d_done[bset])
        run_b()
        for (gh, uh), (gd, ud) in zip(host_out[bset], outs_b):
            gh.copy_(gd, non_blocking=True)
            for a_, c_ in zip(uh, ud):
                a_.copy_(c_, non_blocking=True)
        buf_free[bset].record(stream)

    e2e_steps = max(3, min(args.steps, 50))
    for i in range(2 * nbuf):
        e2e_step(i)
    barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    for i in range(e2e_steps):
        e2e_step(i)
    stream.wait_stream(copy_stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = slowest_rank_ms(ev0.elapsed_time(ev1), dist, "cuda")
    e2e_value = job_rate(e2e_steps * P, world, e2e_ms)
    h2d = P * X.numel() * 4
    d2h = P * (G.numel() + sum(u.numel() for u in Us)) * 4

    # ---------------------------------------------------------------- dominant kernel: mode-1 sketch pass
    peaks, peak_src = _peaks()
    I0 = dims[0]
    J0 = int(np.prod(dims)) // I0
    Kp, _, _ = R.rhosvd_plan(dims, ranks, w.algo, w.p, w.q, K=w.K, S=w.S)
    K0 = Kp[0]
    om = R.rhosvd_omega(w.omega_seed, 0, J0, K0)
    om_buf = om.t().contiguous().reshape(-1)
    pws = R.Workspace(R.rhosvd_primitive_workspace_size(dims, K0))
    Y0 = R.empty_colmajor((I0, K0))
    reps = 50
    for _ in range(3):
        R.rhosvd_sketch(X, dims, 0, K0, Omega=om_buf, Y=Y0, ws=pws)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(reps):
        R.rhosvd_sketch(X, dims, 0, K0, Omega=om_buf, Y=Y0, ws=pws)
    ev1.record(stream)
    torch.cuda.synchronize()
    sk_ms = ev0.elapsed_time(ev1) / reps
    sk_bytes = (X.numel() + J0 * K0 + I0 * K0) * 4      # X once, Omega_1 once, Y once
    sk_gbs = sk_bytes / (sk_ms * 1e-3) / 1e9
    hbm_peak = float(peaks["hbm_gbs"])
    roofline = {"bound": "hbm",
                "kernel": "tc_sketch_kernel<48,1> + reduce_partials (mode-1 sketch Y = X_(1) Omega_1, rhosvd_sketch)",
                "achieved": round(sk_gbs, 1), "peak": hbm_peak, "unit": "GB/s", "frac": round(sk_gbs / hbm_peak, 4),
                "peak_source": peak_src, "algorithmic_bytes_per_launch": sk_bytes, "ms_per_launch": sk_ms,
                "traffic": _traffic_for(os.path.join(ROOT, "paper_2001_07124_gb300", "csrc", "tc_sketch.cu"),
                                        f"tc_sketch_mode1:{w.name}")}

    # ---------------------------------------------------------------- CPU oracle and error gate
    cpu = None
    accuracy = None
    if rank == 0 and x32 is not None:
        t_or, g_or, u_or = oracle_decompose(w, x32, args.dtype, args.refine, args.kron)
        g_gpu = R.fortran_view(G, ranks).cpu().numpy().astype(np.float64)
        u_gpu = [R.matrix(u, dims[n], ranks[n]).cpu().numpy().astype(np.float64) for n, u in enumerate(Us)]
        if args.dtype == "f32" and args.refine == 0:
            accuracy = accuracy_report(x32, g_gpu, u_gpu, g_or, u_or)
        elif args.dtype == "f32":
            # after a randomized refinement sweep the subspaces are fixed by the data only to
            # about the spread between test-matrix draws, so the gate is the reconstruction
            accuracy = accuracy_report(x32, g_gpu, u_gpu, g_or, u_or, max_sine=1.0)
            accuracy["tolerance"] = "FP32 path after refinement: |dE| <= 1e-5 (sines reported, not gated)"
        else:
            # reduced-precision tolerance: |dE| <= 2% of E_oracle and <= 1e-3 (subspaces not gated)
            accuracy = accuracy_report(x32, g_gpu, u_gpu, g_or, u_or, tol=1.0, max_sine=1.0)
            d = abs(accuracy["E_gpu"] - accuracy["E_oracle"])
            accuracy["pass"] = bool(d <= 0.02 * accuracy["E_oracle"] and d <= 1e-3)
            accuracy["tolerance"] = "reduced precision: |dE| <= 2% E_oracle and <= 1e-3"
        cpu = {"value": 1.0 / t_or, "unit": UNIT, "cores": _CORES, "kind": "oracle",
               "sample": f"one full decomposition of the {w.name} workload in FP64 NumPy (seeded Philox test matrices)"}

    launches = P * R.rhosvd_launch_count(dims, ranks, w.algo, w.p, w.q, K=w.K, S=w.S, dtype=args.dtype,
                                         refine=args.refine, kron=args.kron)
    if rank == 0:
        line = {
            "metric": metric_name(w, args.dtype, args.refine, args.kron), "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.dtype,
            "data": "synthetic (seeded low-rank tensor, device-drawn Philox test matrices)",
            "config": {"workload": w.name, "dims": list(dims), "ranks": list(ranks), "algo": w.algo, "p": w.p,
                       "q": w.q, "parallelism": f"replicas{world}", "l2_flush": _l2_note(w),
                       "launch": "eager" if args.no_graph else "cuda_graph",
                       "concurrent_decompositions": P,
                       "step": f"{P} independent decompositions, each on its own copy of the tensor, "
                               f"on parallel graph branches"},
            "single_decomposition_ms": single_ms,
            "clocks": clocks,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps, "overlap": "double-buffered: step i's H2D copies run during step i-1"},
            "gpu_launches": launches * args.steps,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "accuracy": accuracy,
            "householder_fallbacks_per_step": st_words[3],
            "max_jacobi_sweeps": st_words[5],
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
