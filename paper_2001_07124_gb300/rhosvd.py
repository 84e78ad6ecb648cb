"""Python binding of librhosvd (argument marshalling only).

Every step of the decomposition runs in the CUDA library; this module turns
torch tensors into device pointers, sizes and the caller's CUDA stream, and
checks status codes.  PyTorch provides device memory and streams only.

Layout: a tensor of sizes (I_1..I_N) is column-major, i_1 fastest.  The
functions accept a float32 CUDA tensor that is either contiguous (any shape
with the right number of elements; a (I_N, ..., I_1) tensor is the natural
one) or a Fortran-strided view of shape (I_1..I_N).  Matrices returned to the
caller (factors U_n, sketches Y_n) are column-major I x K blocks exposed as
(I, K) views; the core G is exposed as an (R_1..R_N) view of its column-major
buffer.
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

import numpy as np

from . import _build

MAX_MODES = 8
MAX_K = 128
ALGOS = {"rhosvd": 0, "rsthosvd": 1, "rpet": 2}
DTYPES = {"f32": 0, "bf16": 1, "e4m3": 2}
STATUS = {0: "RHOSVD_OK", 1: "RHOSVD_EINVAL", 2: "RHOSVD_ENOMEM", 3: "RHOSVD_ECUDA", 4: "RHOSVD_ENONFINITE",
          5: "RHOSVD_EBREAKDOWN", 6: "RHOSVD_ETIMEOUT", 7: "RHOSVD_EUNSUPPORTED"}
FLAG_FALLBACK = 1
OPT_KRONECKER = 1


class RhosvdError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = int(code)
        msg = lib().rhosvd_status_string(self.code).decode() if _LIB is not None else STATUS.get(code, "?")
        super().__init__(f"{where}: {STATUS.get(self.code, self.code)} ({msg})")


class Shape(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("dims", ctypes.c_int64 * MAX_MODES)]


class Opts(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int32), ("p", ctypes.c_int32), ("q", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("K", ctypes.c_int32 * MAX_MODES), ("S", ctypes.c_int32 * MAX_MODES),
                ("dtype", ctypes.c_int32), ("refine_iters", ctypes.c_int32)]


class BatchItem(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("G", ctypes.c_void_p), ("U", ctypes.c_void_p * MAX_MODES),
                ("dims", ctypes.c_int64 * MAX_MODES), ("ranks", ctypes.c_int32 * MAX_MODES), ("N", ctypes.c_int32)]


class BatchPlan(ctypes.Structure):
    _fields_ = [("n_items", ctypes.c_int32), ("q", ctypes.c_int32), ("p", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("jc", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("imax", ctypes.c_int32), ("kmax", ctypes.c_int32), ("sms", ctypes.c_int32),
                ("max_ctas", ctypes.c_int32), ("seed", ctypes.c_uint64), ("zb_floats", ctypes.c_int64),
                ("s_floats", ctypes.c_int64), ("ws_bytes", ctypes.c_size_t)]


_LIB = None
_P = ctypes.c_void_p
_PP = ctypes.POINTER(ctypes.c_void_p)
_I32P = ctypes.POINTER(ctypes.c_int32)
_I64P = ctypes.POINTER(ctypes.c_int64)


def library_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Load librhosvd.so; raise if it has not been built (there is no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"librhosvd.so is not built ({path}); call paper_2001_07124_gb300.build() first")
    L = ctypes.CDLL(path)
    st = ctypes.c_int
    sig = {
        "rhosvd_plan": (st, [ctypes.POINTER(Shape), _I32P, ctypes.POINTER(Opts), _I32P, _I32P, _I64P]),
        "rhosvd_workspace_size": (ctypes.c_size_t, [ctypes.POINTER(Shape), _I32P, ctypes.POINTER(Opts)]),
        "rhosvd_primitive_workspace_size": (ctypes.c_size_t, [ctypes.POINTER(Shape), ctypes.c_int32]),
        "rhosvd_launch_count": (ctypes.c_int64, [ctypes.POINTER(Shape), _I32P, ctypes.POINTER(Opts)]),
        "rhosvd_omega": (st, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, ctypes.c_int32, _P,
                              ctypes.c_int64, _P]),
        "rhosvd_sketch": (st, [_P, ctypes.POINTER(Shape), ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, _P,
                               _P, _P, ctypes.c_size_t, _P]),
        "rhosvd_sketch_noalloc": (st, [_P, ctypes.POINTER(Shape), ctypes.c_int32, ctypes.c_int32, _P, _P, _P]),
        "rhosvd_sketch_all": (st, [_P, ctypes.POINTER(Shape), _I32P, _I32P, ctypes.c_uint64, _PP, _PP, _PP,
                                   _P, _P, ctypes.c_size_t, _P]),
        "rhosvd_power": (st, [_P, ctypes.POINTER(Shape), ctypes.c_int32, ctypes.c_int32, _P, _P,
                              ctypes.c_size_t, _P]),
        "rhosvd_orth": (st, [_P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, _I32P, _P, ctypes.c_size_t,
                             _P]),
        "rhosvd_core": (st, [_P, ctypes.POINTER(Shape), _PP, _I32P, _P, _P, ctypes.c_size_t, _P]),
        "rhosvd_decompose": (st, [_P, ctypes.POINTER(Shape), _I32P, ctypes.POINTER(Opts), _PP, _PP, _PP, _P,
                                  _P, ctypes.c_size_t, _P]),
        "rhosvd_device_status": (st, [_P, ctypes.c_size_t, _P, _I32P]),
        "rhosvd_workspace_size_tol": (ctypes.c_size_t, [ctypes.POINTER(Shape), ctypes.c_int32, _I32P]),
        "rhosvd_decompose_tol": (st, [_P, ctypes.POINTER(Shape), ctypes.c_double, ctypes.c_int32, _I32P,
                                      ctypes.c_uint64, _I32P, _PP, _P, _P, ctypes.c_size_t, _P]),
        "rhosvd_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "rhosvd_batch_plan_create": (st, [ctypes.POINTER(BatchItem), ctypes.c_int32, ctypes.POINTER(Opts),
                                          ctypes.POINTER(BatchPlan)]),
        "rhosvd_batch_upload": (st, [ctypes.POINTER(BatchPlan), ctypes.POINTER(BatchItem), _P, ctypes.c_size_t,
                                     _P]),
        "rhosvd_batch_run": (st, [ctypes.POINTER(BatchPlan), _P, ctypes.c_size_t, _P]),
        "rhosvd_batch_tune": (st, [ctypes.POINTER(BatchPlan), _P, ctypes.c_size_t, _P,
                                   ctypes.POINTER(ctypes.c_float)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = L
    return L


def declared_symbols() -> list[str]:
    """Entry points declared in include/rhosvd.h, parsed from the header text."""
    import re
    hdr = os.path.join(_build.INCLUDE, "rhosvd.h")
    text = open(hdr).read()
    return sorted(set(re.findall(r"\b(rhosvd_[a-z_]+)\s*\(", text)))


# ------------------------------------------------------------------ marshalling helpers

def make_shape(dims: Sequence[int]) -> Shape:
    dims = [int(d) for d in dims]
    if not 1 <= len(dims) <= MAX_MODES:
        raise ValueError("between 1 and 8 modes")
    sh = Shape()
    sh.N = len(dims)
    for n, d in enumerate(dims):
        sh.dims[n] = d
    return sh


def make_opts(algo: str = "rsthosvd", p: int = 10, q: int = 1, seed: int = 0,
              K: Sequence[int] | None = None, S: Sequence[int] | None = None,
              dtype: str = "f32", refine: int = 0, kron: bool = False) -> Opts:
    o = Opts()
    o.dtype = DTYPES[dtype]
    o.refine_iters = int(refine)
    o.algo = ALGOS[algo]
    o.p, o.q, o.flags, o.seed = int(p), int(q), OPT_KRONECKER if kron else 0, int(seed) & 0xFFFFFFFFFFFFFFFF
    for n in range(MAX_MODES):
        o.K[n] = int(K[n]) if K is not None and n < len(K) else 0
        o.S[n] = int(S[n]) if S is not None and n < len(S) else 0
    return o


def _i32(vals: Sequence[int]):
    arr = (ctypes.c_int32 * max(1, len(vals)))(*[int(v) for v in vals])
    return arr


def _ptrs(tensors):
    if tensors is None:
        return None
    arr = (ctypes.c_void_p * MAX_MODES)()
    for n, t in enumerate(tensors):
        arr[n] = None if t is None else _dptr(t)
    return arr


def _dptr(t) -> int:
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    return t.data_ptr()


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _check(code: int, where: str):
    if code != 0:
        raise RhosvdError(code, where)


def colmajor(x, dims: Sequence[int]):
    """Validate that x holds a column-major FP32 CUDA tensor of sizes dims."""
    import torch
    n = int(np.prod(dims))
    if x.dtype != torch.float32 or not x.is_cuda or x.numel() != n:
        raise ValueError(f"expected a float32 CUDA tensor with {n} elements")
    if x.is_contiguous():
        return x
    if tuple(x.shape) == tuple(dims) and x.permute(*reversed(range(x.dim()))).is_contiguous():
        return x
    raise ValueError("tensor is neither contiguous nor a Fortran-ordered view of dims")


def fortran_view(buf, dims: Sequence[int]):
    """(I_1..I_N) view of a column-major buffer."""
    return buf.reshape(tuple(reversed([int(d) for d in dims]))).permute(*reversed(range(len(dims))))


def empty_colmajor(dims: Sequence[int], device=None):
    import torch
    return torch.empty(int(np.prod(dims)), dtype=torch.float32, device=device or "cuda")


def matrix(buf, rows: int, cols: int):
    """(rows, cols) view of a column-major rows x cols buffer."""
    return buf.reshape(int(cols), int(rows)).t()


class Workspace:
    """Caller-owned device workspace (the library itself never allocates).

    ``ensure`` replaces the buffer when a call needs more bytes than it holds.
    The old buffer goes back to torch's allocator for the current stream, so a
    workspace must not grow while work that uses it is still in flight on
    another stream (size it with the workspace query first)."""

    def __init__(self, nbytes: int, device=None):
        import torch
        self.nbytes = int(max(nbytes, 256))
        self.buf = torch.empty(self.nbytes, dtype=torch.uint8, device=device or "cuda")

    @classmethod
    def wrap(cls, buf):
        """A workspace over an existing uint8 CUDA buffer (256-byte aligned), for
        callers that carve it from memory they manage themselves."""
        import torch
        if buf.dtype != torch.uint8 or not buf.is_cuda or buf.data_ptr() % 256 != 0:
            raise ValueError("expected a 256-byte aligned uint8 CUDA buffer")
        ws = cls.__new__(cls)
        ws.nbytes, ws.buf = int(buf.numel()), buf
        return ws

    @property
    def ptr(self) -> int:
        return self.buf.data_ptr()

    def ensure(self, nbytes: int):
        if nbytes > self.nbytes:
            self.__init__(nbytes, self.buf.device)
        return self


# ------------------------------------------------------------------ entry points

def rhosvd_plan(dims, ranks, algo="rsthosvd", p=10, q=1, K=None, S=None, dtype="f32", refine=0, kron=False):
    """(K_n, S_n, J_n) lists a decomposition uses."""
    N = len(dims)
    Ko, So, Jo = (ctypes.c_int32 * N)(), (ctypes.c_int32 * N)(), (ctypes.c_int64 * N)()
    _check(lib().rhosvd_plan(ctypes.byref(make_shape(dims)), _i32(ranks),
                             ctypes.byref(make_opts(algo, p, q, 0, K, S, dtype, refine, kron)), Ko, So, Jo), "rhosvd_plan")
    return list(Ko), list(So), list(Jo)


def rhosvd_workspace_size(dims, ranks, algo="rsthosvd", p=10, q=1, K=None, S=None, dtype="f32", refine=0,
                          kron=False) -> int:
    return int(lib().rhosvd_workspace_size(ctypes.byref(make_shape(dims)), _i32(ranks),
                                           ctypes.byref(make_opts(algo, p, q, 0, K, S, dtype, refine, kron))))


def rhosvd_launch_count(dims, ranks, algo="rsthosvd", p=10, q=1, K=None, S=None, dtype="f32", refine=0,
                        kron=False) -> int:
    return int(lib().rhosvd_launch_count(ctypes.byref(make_shape(dims)), _i32(ranks),
                                         ctypes.byref(make_opts(algo, p, q, 0, K, S, dtype, refine, kron))))


def rhosvd_primitive_workspace_size(dims, Kmax) -> int:
    return int(lib().rhosvd_primitive_workspace_size(ctypes.byref(make_shape(dims)), int(Kmax)))


def rhosvd_omega(seed: int, stream_id: int, rows: int, cols: int, out=None, stream=None):
    """rows x cols Gaussian test matrix; returns the (rows, cols) column-major view."""
    import torch
    own = out is None
    if own:
        out = torch.empty(int(rows) * int(cols), dtype=torch.float32, device="cuda")
    _check(lib().rhosvd_omega(int(seed), int(stream_id), int(rows), int(cols), _dptr(out), int(rows),
                              _stream(stream)), "rhosvd_omega")
    _hold(stream, out if own else None)
    return matrix(out, rows, cols)


def _ws_for(ws, nbytes):
    if ws is None:
        return Workspace(nbytes)
    return ws.ensure(nbytes)


def _hold(stream, *tensors, current=None):
    """Keep buffers this binding allocated alive for work on another stream.

    The buffers come from torch's caching allocator on the current stream. When
    the library's work goes to a different ``stream``, freeing them at return
    would let a later allocation on the current stream reuse the memory while
    the kernels still use it; ``record_stream`` defers the reuse until the work
    enqueued on ``stream`` so far has finished. ``None`` entries are skipped."""
    if stream is None:
        return
    if current is None:
        import torch
        current = torch.cuda.current_stream()
    if stream == current:
        return
    for t in tensors:
        if t is not None:
            t.record_stream(stream)


def rhosvd_sketch(X, dims, mode: int, K: int, seed: int = 0, Omega=None, Y=None, ws=None, stream=None):
    """Y = X_(mode) Omega (I_mode x K)."""
    X = colmajor(X, dims)
    I = int(dims[mode])
    own_y, own_ws = Y is None, ws is None
    Y = empty_colmajor((I, K)) if Y is None else Y
    ws = _ws_for(ws, rhosvd_primitive_workspace_size(dims, K))
    om = None if Omega is None else _dptr(Omega)
    _check(lib().rhosvd_sketch(_dptr(X), ctypes.byref(make_shape(dims)), int(mode), int(K), int(seed), om,
                               _dptr(Y), ws.ptr, ws.nbytes, _stream(stream)), "rhosvd_sketch")
    _hold(stream, Y if own_y else None, ws.buf if own_ws else None)
    return matrix(Y, I, K)


def rhosvd_sketch_noalloc(X, dims, mode: int, K: int, Omega, Y=None, stream=None):
    """Y = X_(mode) Omega without a workspace, for callers that cannot allocate
    device memory at the call site (the partial sums live in a fixed 4 MiB
    device array owned by the library; Y may be passed in preallocated).
    Calls that overlap on the GPU share that array and race; order them."""
    X = colmajor(X, dims)
    I = int(dims[mode])
    own_y = Y is None
    Y = empty_colmajor((I, K)) if Y is None else Y
    _check(lib().rhosvd_sketch_noalloc(_dptr(X), ctypes.byref(make_shape(dims)), int(mode), int(K), _dptr(Omega),
                                       _dptr(Y), _stream(stream)), "rhosvd_sketch_noalloc")
    _hold(stream, Y if own_y else None)
    return matrix(Y, I, K)


def rhosvd_sketch_all(X, dims, K, S=None, seed: int = 0, Omega=None, Omega_tilde=None, want_H=True,
                      ws=None, stream=None):
    """All mode sketches Y_n and (optionally) the core sketch H of R-PET."""
    X = colmajor(X, dims)
    N = len(dims)
    Ys = [empty_colmajor((dims[n], K[n])) for n in range(N)]
    H = empty_colmajor(S) if (want_H and S is not None) else None
    need = rhosvd_primitive_workspace_size(dims, max(K))
    if H is not None:
        t = list(dims)
        mt = 1
        om = 0
        for n in range(N):
            t[n] = S[n]
            mt = max(mt, int(np.prod(t)))
            om += S[n] * dims[n] * 4 + 256
        need += 2 * (mt * 4 + 256) + om
    own_ws = ws is None
    ws = _ws_for(ws, need)
    _check(lib().rhosvd_sketch_all(_dptr(X), ctypes.byref(make_shape(dims)), _i32(K),
                                   _i32(S) if S is not None else None, int(seed), _ptrs(Omega),
                                   _ptrs(Omega_tilde), _ptrs(Ys), None if H is None else _dptr(H), ws.ptr,
                                   ws.nbytes, _stream(stream)), "rhosvd_sketch_all")
    _hold(stream, H, ws.buf if own_ws else None, *Ys)
    Ys = [matrix(Ys[n], dims[n], K[n]) for n in range(N)]
    return Ys, (None if H is None else fortran_view(H, S))


def rhosvd_power(X, dims, mode: int, Q, ws=None, stream=None):
    """One stable power step: returns X_(n) orth(X_(n)^T Q) (I x K)."""
    X = colmajor(X, dims)
    I, K = int(Q.shape[0]), int(Q.shape[1])
    buf = Q.t().contiguous().reshape(-1).clone()
    own_ws = ws is None
    ws = _ws_for(ws, rhosvd_primitive_workspace_size(dims, K))
    _check(lib().rhosvd_power(_dptr(X), ctypes.byref(make_shape(dims)), int(mode), K, _dptr(buf), ws.ptr,
                              ws.nbytes, _stream(stream)), "rhosvd_power")
    _hold(stream, buf, ws.buf if own_ws else None)
    return matrix(buf, I, K)


def rhosvd_orth(Y, ws=None, stream=None, report_fallback=False):
    """Orthonormalise the columns of Y (m x K, given as an (m, K) tensor); returns (Q, fallback)."""
    m, K = int(Y.shape[0]), int(Y.shape[1])
    buf = Y.t().contiguous().reshape(-1).clone()
    own_ws = ws is None
    ws = _ws_for(ws, rhosvd_primitive_workspace_size((m, K), K))
    fb = ctypes.c_int32(0)
    _check(lib().rhosvd_orth(_dptr(buf), m, K, m, ctypes.byref(fb) if report_fallback else None, ws.ptr,
                             ws.nbytes, _stream(stream)), "rhosvd_orth")
    _hold(stream, buf, ws.buf if own_ws else None)
    return matrix(buf, m, K), (bool(fb.value) if report_fallback else None)


def rhosvd_core(X, dims, Qs, ws=None, stream=None):
    """G = X x_1 Q_1^T ... x_N Q_N^T; Qs[n] is (I_n, K_n) or None to skip the mode."""
    X = colmajor(X, dims)
    N = len(dims)
    K = [int(dims[n]) if Qs[n] is None else int(Qs[n].shape[1]) for n in range(N)]
    qbufs = [None if q is None else q.t().contiguous().reshape(-1) for q in Qs]
    G = empty_colmajor(K)
    t = list(dims)
    mt = 1
    for n in range(N):
        t[n] = K[n]
        mt = max(mt, int(np.prod(t)))
    own_ws = ws is None
    ws = _ws_for(ws, 256 + 2 * (mt * 4 + 256))
    _check(lib().rhosvd_core(_dptr(X), ctypes.byref(make_shape(dims)), _ptrs(qbufs), _i32(K), _dptr(G),
                             ws.ptr, ws.nbytes, _stream(stream)), "rhosvd_core")
    _hold(stream, G, ws.buf if own_ws else None, *qbufs)
    return fortran_view(G, K)


def rhosvd_decompose(X, dims, ranks, algo="rsthosvd", p=10, q=1, seed=0, Omega=None, Omega_tilde=None,
                     K=None, S=None, ws=None, out=None, stream=None, check=True, dtype="f32", refine=0,
                     kron=False):
    """Randomized Tucker decomposition; returns (G as an (R_1..R_N) view, [U_n as (I_n, R_n) views]).

    Omega / Omega_tilde: optional lists of explicit test matrices as column-major
    buffers (rows x cols) with the sizes rhosvd_plan reports.  ``out``: optional
    (G_buf, [U_bufs]) preallocated buffers.  ``check``: synchronise and raise on
    a device-detected error.  ``dtype``: "f32", "bf16" or "e4m3", the
    arithmetic of the sketch passes; ``refine``: RP-HOOI sweeps afterwards;
    ``kron``: R-PET with Kronecker-structured factor sketches (Omega[p] then
    supplies Phi_p, I_p x k)."""
    X = colmajor(X, dims)
    N = len(dims)
    shape, opts = make_shape(dims), make_opts(algo, p, q, seed, K, S, dtype, refine, kron)
    r = _i32(ranks)
    if out is None:
        G = empty_colmajor(ranks)
        Us = [empty_colmajor((dims[n], ranks[n])) for n in range(N)]
    else:
        G, Us = out
    need = int(lib().rhosvd_workspace_size(ctypes.byref(shape), r, ctypes.byref(opts)))
    if need == 0:
        _check(1, "rhosvd_workspace_size")
    own_ws = ws is None
    ws = _ws_for(ws, need)
    code = lib().rhosvd_decompose(_dptr(X), ctypes.byref(shape), r, ctypes.byref(opts), _ptrs(Omega),
                                  _ptrs(Omega_tilde), _ptrs(Us), _dptr(G), ws.ptr, ws.nbytes, _stream(stream))
    _check(code, "rhosvd_decompose")
    if out is None:
        _hold(stream, G, *Us)
    if own_ws:
        _hold(stream, ws.buf)
    if check:
        dev, _ = rhosvd_device_status(ws, stream)
        _check(dev, "rhosvd_decompose (device)")
    return fortran_view(G, ranks), [matrix(Us[n], dims[n], ranks[n]) for n in range(N)]


class DecomposeGraph:
    """One rhosvd_decompose call captured into a CUDA graph.

    The call is recorded with fixed X, shape, ranks, options, workspace and
    output buffers; ``replay()`` re-runs every kernel of the decomposition with
    one graph launch (no per-kernel host launch cost, no gaps between launches).
    New input is given by copying it into the same X buffer before replaying.
    The library allocates nothing and synchronises nothing inside the call, so
    the capture records exactly the eager sequence; results are bitwise equal
    to an eager call on the same input."""

    def __init__(self, X, dims, ranks, ws=None, out=None, warmup=2, **kw):
        import torch
        X = colmajor(X, dims)
        N = len(dims)
        if out is None:
            out = (empty_colmajor(ranks), [empty_colmajor((dims[n], ranks[n])) for n in range(N)])
        shape, opts = make_shape(dims), make_opts(kw.get("algo", "rsthosvd"), kw.get("p", 10), kw.get("q", 1),
                                                 kw.get("seed", 0), kw.get("K"), kw.get("S"),
                                                 kw.get("dtype", "f32"), kw.get("refine", 0), kw.get("kron", False))
        need = int(lib().rhosvd_workspace_size(ctypes.byref(shape), _i32(ranks), ctypes.byref(opts)))
        if need == 0:
            _check(1, "rhosvd_workspace_size")
        ws = _ws_for(ws, need)
        self.X, self.dims, self.ranks, self.ws, self.out = X, tuple(dims), tuple(ranks), ws, out
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(warmup):        # per-kernel attributes and tensor-map encoders settle before capture
                rhosvd_decompose(X, dims, ranks, ws=ws, out=out, check=False, **kw)
        torch.cuda.current_stream().wait_stream(side)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            rhosvd_decompose(X, dims, ranks, ws=ws, out=out, check=False, **kw)

    def replay(self):
        self.graph.replay()

    def result(self):
        G, Us = self.out
        return fortran_view(G, self.ranks), [matrix(Us[n], self.dims[n], self.ranks[n])
                                             for n in range(len(self.dims))]


class BatchGraph:
    """Many independent decompositions in one CUDA graph.

    items: list of (X, dims, ranks) with X a column-major device tensor; each
    item gets its own workspace and output buffers.  The items are spread over
    ``branches`` parallel branches of the graph (item i on branch i % branches),
    so the GPU overlaps independent decompositions; ``replay()`` runs the whole
    batch with one launch.  ``results()`` returns (G, [U_n]) views per item."""

    def __init__(self, items, branches=16, warmup=1, **kw):
        import torch
        self.items = []
        for X, dims, ranks in items:
            X = colmajor(X, dims)
            N = len(dims)
            out = (empty_colmajor(ranks), [empty_colmajor((dims[n], ranks[n])) for n in range(N)])
            shape, opts = make_shape(dims), make_opts(kw.get("algo", "rsthosvd"), kw.get("p", 10),
                                                     kw.get("q", 1), kw.get("seed", 0), kw.get("K"), kw.get("S"),
                                                     kw.get("dtype", "f32"), kw.get("refine", 0), kw.get("kron", False))
            need = int(lib().rhosvd_workspace_size(ctypes.byref(shape), _i32(ranks), ctypes.byref(opts)))
            if need == 0:
                _check(1, "rhosvd_workspace_size")
            self.items.append((X, tuple(dims), tuple(ranks), Workspace(need), out))
        self.kw = kw
        nb = max(1, min(int(branches), len(self.items)))
        self.streams = [torch.cuda.Stream() for _ in range(nb)]
        cur = torch.cuda.current_stream()
        for s in self.streams:
            s.wait_stream(cur)
        for _ in range(warmup):
            self._enqueue()
        for s in self.streams:
            cur.wait_stream(s)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            cap = torch.cuda.current_stream()
            fork = torch.cuda.Event()
            fork.record(cap)
            for s in self.streams:
                s.wait_event(fork)
            self._enqueue()
            for s in self.streams:
                done = torch.cuda.Event()
                done.record(s)
                cap.wait_event(done)

    def _enqueue(self):
        for i, (X, dims, ranks, ws, out) in enumerate(self.items):
            rhosvd_decompose(X, dims, ranks, ws=ws, out=out, check=False, stream=self.streams[i % len(self.streams)],
                             **self.kw)

    def replay(self):
        self.graph.replay()

    def results(self):
        res = []
        for X, dims, ranks, ws, (G, Us) in self.items:
            res.append((fortran_view(G, ranks), [matrix(Us[n], dims[n], ranks[n]) for n in range(len(dims))]))
        return res

    def device_status(self):
        """Worst device status over the items (synchronises)."""
        worst = 0
        for X, dims, ranks, ws, out in self.items:
            code, _ = rhosvd_device_status(ws)
            worst = worst or code
        return worst


class BatchPersistent:
    """Many small R-STHOSVDs in one persistent launch (rhosvd_batch_*).

    items: list of (X, dims, ranks) with X a column-major device tensor.  Each
    item gets its own outputs; the batch shares one workspace (the item table,
    the work queue and per-CTA scratch).  ``tune()`` times the launchable
    configurations on this batch and keeps the fastest; ``run()`` enqueues the
    batch on a stream (a memset and one kernel, capturable); ``results()``
    returns (G, [U_n]) views per item."""

    def __init__(self, items, algo="rsthosvd", p=5, q=1, seed=0, stream=None):
        if algo != "rsthosvd":
            raise ValueError("the persistent batch runs R-STHOSVD")
        self.items = []
        n = len(items)
        self._table = (BatchItem * max(1, n))()
        for t, (X, dims, ranks) in enumerate(items):
            X = colmajor(X, dims)
            N = len(dims)
            out = (empty_colmajor(ranks), [empty_colmajor((dims[k], ranks[k])) for k in range(N)])
            self.items.append((X, tuple(dims), tuple(ranks), out))
            it = self._table[t]
            it.X, it.G, it.N = _dptr(X), _dptr(out[0]), N
            for k in range(N):
                it.U[k] = _dptr(out[1][k])
                it.dims[k] = int(dims[k])
                it.ranks[k] = int(ranks[k])
        self.plan = BatchPlan()
        opts = make_opts(algo, p, q, seed)
        _check(lib().rhosvd_batch_plan_create(self._table, n, ctypes.byref(opts), ctypes.byref(self.plan)),
               "rhosvd_batch_plan_create")
        self.ws = Workspace(int(self.plan.ws_bytes))
        _check(lib().rhosvd_batch_upload(ctypes.byref(self.plan), self._table, _P(self.ws.ptr), self.ws.nbytes,
                                         _stream(stream)), "rhosvd_batch_upload")

    @property
    def config(self):
        return {"threads": int(self.plan.threads), "tile_columns": int(self.plan.jc),
                "ctas_per_sm": int(self.plan.ctas_per_sm)}

    def tune(self, stream=None) -> float:
        ms = ctypes.c_float(0.0)
        _check(lib().rhosvd_batch_tune(ctypes.byref(self.plan), _P(self.ws.ptr), self.ws.nbytes, _stream(stream),
                                       ctypes.byref(ms)), "rhosvd_batch_tune")
        return float(ms.value)

    def run(self, stream=None):
        _check(lib().rhosvd_batch_run(ctypes.byref(self.plan), _P(self.ws.ptr), self.ws.nbytes, _stream(stream)),
               "rhosvd_batch_run")

    def results(self):
        return [(fortran_view(G, ranks), [matrix(Us[k], dims[k], ranks[k]) for k in range(len(dims))])
                for X, dims, ranks, (G, Us) in self.items]

    def device_status(self):
        code, _ = rhosvd_device_status(self.ws)
        return code


def rhosvd_workspace_size_tol(dims, block, k_max) -> int:
    return int(lib().rhosvd_workspace_size_tol(ctypes.byref(make_shape(dims)), int(block), _i32(k_max)))


def rhosvd_decompose_tol(X, dims, eps, block=8, k_max=None, seed=0, ws=None, out=None, stream=None, check=True):
    """Fixed-accuracy R-STHOSVD: returns (G as an (R_1..R_N) view, [U_n as (I_n, R_n) views], ranks).
    Synchronises the stream after every block of the range finder."""
    X = colmajor(X, dims)
    N = len(dims)
    k_max = [min(int(d), MAX_K) for d in dims] if k_max is None else [int(k) for k in k_max]
    if out is None:
        G = empty_colmajor(k_max)
        Us = [empty_colmajor((dims[n], k_max[n])) for n in range(N)]
    else:
        G, Us = out
    need = rhosvd_workspace_size_tol(dims, block, k_max)
    if need == 0:
        _check(1, "rhosvd_workspace_size_tol")
    own_ws = ws is None
    ws = _ws_for(ws, need)
    ranks = (ctypes.c_int32 * N)()
    _check(lib().rhosvd_decompose_tol(_dptr(X), ctypes.byref(make_shape(dims)), float(eps), int(block),
                                      _i32(k_max), int(seed) & 0xFFFFFFFFFFFFFFFF, ranks, _ptrs(Us), _dptr(G),
                                      ws.ptr, ws.nbytes, _stream(stream)), "rhosvd_decompose_tol")
    r = [int(v) for v in ranks]
    if own_ws:
        _hold(stream, ws.buf)
    if check:
        dev, _ = rhosvd_device_status(ws, stream)
        _check(dev, "rhosvd_decompose_tol (device)")
    ng = int(np.prod(r))
    return fortran_view(G[:ng], r), [matrix(Us[n][:dims[n] * r[n]], dims[n], r[n]) for n in range(N)], r


def rhosvd_device_status(ws, stream=None):
    flags = ctypes.c_int32(0)
    code = lib().rhosvd_device_status(ws.ptr, ws.nbytes, _stream(stream), ctypes.byref(flags))
    return int(code), int(flags.value)
