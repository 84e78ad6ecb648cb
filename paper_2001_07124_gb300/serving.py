"""Continuous-batching decomposition server over the C ABI.

Requests (a tensor in pinned host memory, its dims, target ranks and the
algorithm options) arrive over time.  The scheduler admits them in arrival
order whenever a slot (a CUDA stream with its own workspace) is free and the
device-memory budget covers what the slots hold: each slot keeps one device
arena (workspace, tensor and outputs, sized by the library's own workspace
query) and one pinned host buffer between requests, so steady-state requests
allocate nothing. An admitted request copies
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
    ranks: tuple                        # fixed rank (ignored by fixed-accuracy requests)
    arrival: float                      # seconds from the start of the run
    x_host: object = None               # flat column-major FP32 tensor (torch, pinned) for the GPU executor
    algo: str = "rsthosvd"
    p: int = 10
    q: int = 1
    seed: int = 0
    tol: float = 0.0                    # > 0: fixed-accuracy request, ||X - X_hat|| <= tol ||X||, ranks found
    block: int = 16                     # range-finder block of a fixed-accuracy request
    k_max: Optional[tuple] = None       # largest rank per mode of a fixed-accuracy request (default min(I_n, 128))


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    G: Optional[np.ndarray] = None
    Us: Optional[List[np.ndarray]] = None
    ranks: Optional[tuple] = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class Scheduler:
    """FIFO admission under a slot count and a device-memory budget.

    A slot keeps its device buffers between requests (so that a request does
    not pay for an allocation), which makes the memory a slot holds, not the
    memory its current request needs, the quantity the budget has to cover.
    The scheduler therefore charges every slot what it holds: admitting a
    request of ``bytes_needed`` b on a slot that holds h raises the slot's
    holding to max(h, b), and idle slots hold their buffers until the head of
    the queue needs the room, at which point the largest idle holdings are
    released first.  The sum of all holdings never exceeds the budget.

    executor.bytes_needed(req) -> int, executor.start(req, slot) -> handle,
    executor.done(handle) -> bool, executor.finish(handle) -> (G, Us) and
    executor.release(slot) are the only operations it uses; clock() returns
    seconds since the run started."""

    def __init__(self, executor, slots: int, budget_bytes: int, clock: Callable[[], float]):
        if slots < 1 or budget_bytes <= 0:
            raise ValueError("need at least one slot and a positive budget")
        self.ex, self.slots, self.budget, self.clock = executor, slots, int(budget_bytes), clock
        self.held = [0] * slots                       # bytes each slot holds (grows, or drops on release)
        self.peak_held = 0

    def _fit(self, need: int, free_slots: List[int]) -> Optional[int]:
        """A free slot for a request of `need` bytes, releasing idle holdings
        if the budget requires it; None when the request has to wait."""
        # best fit: the smallest idle holding that already covers the request, else the largest one
        covering = [s for s in free_slots if self.held[s] >= need]
        slot = min(covering, key=lambda s: self.held[s]) if covering else max(free_slots, key=lambda s: self.held[s])
        total = sum(self.held) - self.held[slot] + max(self.held[slot], need)
        if total > self.budget:
            for other in sorted((s for s in free_slots if s != slot and self.held[s] > 0),
                                key=lambda s: -self.held[s]):
                self.ex.release(other)
                total -= self.held[other]
                self.held[other] = 0
                if total <= self.budget:
                    break
        if total > self.budget:
            return None
        self.held[slot] = max(self.held[slot], need)
        self.peak_held = max(self.peak_held, sum(self.held))
        return slot

    def run(self, requests: Sequence[Request], idle: Callable[[], None] = lambda: None) -> List[Result]:
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        for r in pending:
            if self.ex.bytes_needed(r) > self.budget:
                raise ValueError(f"request {r.rid} needs more device memory than the whole budget")
        free_slots = list(range(self.slots))
        active = []                                   # (req, slot, handle, admitted)
        results: List[Result] = []
        head = 0
        while head < len(pending) or active:
            now = self.clock()
            still = []
            for req, slot, h, adm in active:           # retire finished requests
                if self.ex.done(h):
                    out = self.ex.finish(h)
                    G, Us = out[0], out[1]
                    ranks = out[2] if len(out) > 2 else tuple(req.ranks)
                    results.append(Result(req.rid, req.arrival, adm, self.clock(), G, Us, ranks))
                    free_slots.append(slot)
                else:
                    still.append((req, slot, h, adm))
            active = still
            # admit in arrival order; the head of the queue waits until it fits
            while head < len(pending) and pending[head].arrival <= now and free_slots:
                req = pending[head]
                slot = self._fit(self.ex.bytes_needed(req), free_slots)
                if slot is None:
                    break
                free_slots.remove(slot)
                h = self.ex.start(req, slot)
                active.append((req, slot, h, self.clock()))
                head += 1
            idle()
        return results


def _align(n: int, a: int = 256) -> int:
    return (int(n) + a - 1) // a * a


class GpuExecutor:
    """Runs requests on CUDA streams through the library.

    Each slot owns one device arena, carved per request into the workspace,
    the tensor and the outputs, and one pinned host buffer for the outputs.
    Both are reused by the slot's next request and only grow (or are dropped
    by ``release``), so a request in steady state allocates nothing.
    Fixed-rank requests are enqueued on the slot's stream and observed through
    an event.  A fixed-accuracy request (rhosvd_decompose_tol) reads its error
    indicator on the host after every block, so it runs in a worker thread on
    its slot's stream; the other slots keep going meanwhile."""

    def __init__(self, slots: int):
        import concurrent.futures as cf
        import torch
        from . import rhosvd as R
        self.torch, self.R = torch, R
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.arena = [None] * slots                  # device uint8 buffers
        self.host = [None] * slots                   # pinned float32 output buffers
        self.pool = cf.ThreadPoolExecutor(max_workers=slots)

    @staticmethod
    def _kmax(req: Request):
        return tuple(req.k_max) if req.k_max is not None else tuple(min(int(d), 128) for d in req.dims)

    def _layout(self, req: Request):
        """Byte offsets (ws, X, G, U_1..U_N) of a request inside its slot's arena and the total."""
        R = self.R
        if req.tol > 0:
            km = self._kmax(req)
            ws = _align(R.rhosvd_workspace_size_tol(req.dims, req.block, km))
            out_ranks = km
        else:
            ws = _align(R.rhosvd_workspace_size(req.dims, req.ranks, req.algo, req.p, req.q))
            out_ranks = req.ranks
        sizes = [4 * int(np.prod(req.dims)), 4 * int(np.prod(out_ranks))] + \
                [4 * int(d) * int(r) for d, r in zip(req.dims, out_ranks)]
        offs, off = [0], ws
        for sz in sizes:
            offs.append(off)
            off += _align(sz)
        return offs, sizes, off

    def bytes_needed(self, req: Request) -> int:
        return self._layout(req)[2]

    def release(self, slot: int):
        self.arena[slot] = None

    def start(self, req: Request, slot: int):
        torch, R = self.torch, self.R
        s = self.streams[slot]
        offs, sizes, total = self._layout(req)
        if self.arena[slot] is None or self.arena[slot].numel() < total:
            self.arena[slot] = None
            self.arena[slot] = torch.empty(total, dtype=torch.uint8, device="cuda")
        nout = sum(sizes[1:]) // 4
        if self.host[slot] is None or self.host[slot].numel() < nout:
            self.host[slot] = torch.empty(nout, dtype=torch.float32).pin_memory()
        a = self.arena[slot]
        ws = R.Workspace.wrap(a[:offs[1]])
        views = [a[o:o + sz].view(torch.float32) for o, sz in zip(offs[1:], sizes)]
        X, G, Us = views[0], views[1], views[2:]
        hv, off = [], 0
        for sz in sizes[1:]:
            hv.append(self.host[slot][off:off + sz // 4])
            off += sz // 4
        if req.tol > 0:
            def work():
                with torch.cuda.stream(s):
                    X.copy_(req.x_host, non_blocking=True)
                    _, _, ranks = R.rhosvd_decompose_tol(X, req.dims, req.tol, block=req.block,
                                                         k_max=self._kmax(req), seed=req.seed, ws=ws,
                                                         out=(G, Us), stream=s, check=False)
                    ng = int(np.prod(ranks))
                    hv[0][:ng].copy_(G[:ng], non_blocking=True)
                    for n, (d, r) in enumerate(zip(req.dims, ranks)):
                        hv[1 + n][:d * r].copy_(Us[n][:d * r], non_blocking=True)
                    s.synchronize()
                return tuple(ranks)
            return ("tol", req, slot, ws, hv, self.pool.submit(work))
        with torch.cuda.stream(s):
            X.copy_(req.x_host, non_blocking=True)
            R.rhosvd_decompose(X, req.dims, req.ranks, algo=req.algo, p=req.p, q=req.q, seed=req.seed,
                               ws=ws, out=(G, Us), stream=s, check=False)
            for hbuf, dbuf in zip(hv, [G] + Us):
                hbuf.copy_(dbuf, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        return ("rank", req, slot, ws, hv, ev)

    def done(self, h) -> bool:
        return h[-1].done() if h[0] == "tol" else h[-1].query()

    def finish(self, h):
        kind, req, slot, ws, hv, waitable = h
        if kind == "tol":
            ranks = waitable.result()
        else:
            waitable.synchronize()
            ranks = tuple(req.ranks)
        code, _ = self.R.rhosvd_device_status(ws, self.streams[slot])
        if code != 0:
            raise RuntimeError(f"request {req.rid}: device status {code}")
        ng = int(np.prod(ranks))
        G = hv[0][:ng].numpy().copy()
        Us = [hv[1 + n][:d * r].numpy().copy() for n, (d, r) in enumerate(zip(req.dims, ranks))]
        return G, Us, ranks


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
