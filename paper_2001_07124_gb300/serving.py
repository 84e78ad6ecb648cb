"""Continuous-batching decomposition server over the C ABI.

Requests (a tensor in pinned host memory, its dims, target ranks and the
algorithm options) arrive over time.  The scheduler admits them in arrival
order whenever a slot (a CUDA stream with its own workspace) is free and the
device-memory budget covers the request's tensor, workspace and outputs (the
library's own workspace query sizes it exactly). An admitted request copies
its tensor to the device, runs rhosvd_decompose on its slot's stream and
copies the core and factors back; completion is observed through a CUDA event.
Requests that are on the device at the same time overlap there: one request's
single-CTA factorisations leave most SMs free for another's bandwidth-bound
passes.  Every kernel of the library is deterministic and each request has its
own buffers, so a request's result does not depend on what else is running.

The scheduler itself (admission order, budget and slot accounting) is separate
from the executor that touches the GPU, so it can be exercised with a fake
executor on the CPU.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Callable, List, Optional, Sequence

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    dims: tuple
    ranks: tuple
    arrival: float                      # seconds from the start of the run
    x_host: object = None               # flat column-major FP32 tensor (torch, pinned) for the GPU executor
    algo: str = "rsthosvd"
    p: int = 10
    q: int = 1
    seed: int = 0


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    G: Optional[np.ndarray] = None
    Us: Optional[List[np.ndarray]] = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class Scheduler:
    """FIFO admission under a slot count and a device-memory budget.

    executor.bytes_needed(req) -> int, executor.start(req, slot) -> handle,
    executor.done(handle) -> bool, executor.finish(handle) -> (G, Us) are the
    only operations it uses; clock() returns seconds since the run started."""

    def __init__(self, executor, slots: int, budget_bytes: int, clock: Callable[[], float]):
        if slots < 1 or budget_bytes <= 0:
            raise ValueError("need at least one slot and a positive budget")
        self.ex, self.slots, self.budget, self.clock = executor, slots, int(budget_bytes), clock

    def run(self, requests: Sequence[Request], idle: Callable[[], None] = lambda: None) -> List[Result]:
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        for r in pending:
            if self.ex.bytes_needed(r) > self.budget:
                raise ValueError(f"request {r.rid} needs more device memory than the whole budget")
        free_slots = list(range(self.slots))
        used = 0
        active = []                                   # (req, slot, handle, bytes, admitted)
        results: List[Result] = []
        head = 0
        while head < len(pending) or active:
            now = self.clock()
            still = []
            for req, slot, h, nb, adm in active:       # retire finished requests
                if self.ex.done(h):
                    G, Us = self.ex.finish(h)
                    results.append(Result(req.rid, req.arrival, adm, self.clock(), G, Us))
                    free_slots.append(slot)
                    used -= nb
                else:
                    still.append((req, slot, h, nb, adm))
            active = still
            # admit in arrival order; the head of the queue waits until it fits
            while head < len(pending) and pending[head].arrival <= now and free_slots:
                req = pending[head]
                nb = self.ex.bytes_needed(req)
                if used + nb > self.budget:
                    break
                slot = free_slots.pop(0)
                h = self.ex.start(req, slot)
                active.append((req, slot, h, nb, self.clock()))
                used += nb
                head += 1
            idle()
        return results


class GpuExecutor:
    """Runs requests on CUDA streams through the library (one workspace per slot)."""

    def __init__(self, slots: int):
        import torch
        from . import rhosvd as R
        self.torch, self.R = torch, R
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.ws = [None] * slots

    def bytes_needed(self, req: Request) -> int:
        R = self.R
        n = int(np.prod(req.dims))
        need = R.rhosvd_workspace_size(req.dims, req.ranks, req.algo, req.p, req.q)
        out = int(np.prod(req.ranks)) + sum(int(d) * int(r) for d, r in zip(req.dims, req.ranks))
        return 4 * (n + out) + int(need)

    def start(self, req: Request, slot: int):
        torch, R = self.torch, self.R
        s = self.streams[slot]
        need = R.rhosvd_workspace_size(req.dims, req.ranks, req.algo, req.p, req.q)
        with torch.cuda.stream(s):
            if self.ws[slot] is None or self.ws[slot].nbytes < need:
                self.ws[slot] = R.Workspace(need)
            X = torch.empty(int(np.prod(req.dims)), dtype=torch.float32, device="cuda")
            X.copy_(req.x_host, non_blocking=True)
            G = R.empty_colmajor(req.ranks)                               # flat column-major buffers
            Us = [R.empty_colmajor((d, r)) for d, r in zip(req.dims, req.ranks)]
            R.rhosvd_decompose(X, req.dims, req.ranks, algo=req.algo, p=req.p, q=req.q, seed=req.seed,
                               ws=self.ws[slot], out=(G, Us), stream=s, check=False)
            gh = torch.empty(G.numel(), dtype=torch.float32).pin_memory()
            uh = [torch.empty(u.numel(), dtype=torch.float32).pin_memory() for u in Us]
            gh.copy_(G, non_blocking=True)
            for a, b in zip(uh, Us):
                a.copy_(b, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        return (req, slot, X, G, Us, gh, uh, ev)

    def done(self, h) -> bool:
        return h[-1].query()

    def finish(self, h):
        req, slot, X, G, Us, gh, uh, ev = h
        ev.synchronize()
        code, _ = self.R.rhosvd_device_status(self.ws[slot], self.streams[slot])
        if code != 0:
            raise RuntimeError(f"request {req.rid}: device status {code}")
        return gh.numpy().copy(), [u.numpy().copy() for u in uh]


def serve(requests: Sequence[Request], slots: int = 4, budget_bytes: int = 150 * 10 ** 9) -> List[Result]:
    """Run the requests against the GPU with the arrival times they carry."""
    ex = GpuExecutor(slots)
    t0 = time.perf_counter()
    return Scheduler(ex, slots, budget_bytes, lambda: time.perf_counter() - t0).run(requests)


def latency_summary(results: Sequence[Result]) -> dict:
    lat = np.array([r.latency for r in results]) * 1e3
    span = max(r.finished for r in results) - min(r.arrival for r in results)
    return {"requests": len(results), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "decomps_per_s": len(results) / span if span > 0 else float("inf")}
