"""Host-side checks of the C ABI (no GPU needed): the library builds and loads,
exports every entry point include/rhosvd.h declares, plans the same sketch
widths as the oracle's independent rule, and rejects invalid requests before
touching the device."""
import ctypes
import os

import pytest

from oracle import algorithms as A
import paper_2001_07124_gb300 as pkg
from paper_2001_07124_gb300 import rhosvd as R


@pytest.fixture(scope="module")
def lib():
    pkg.build()
    return R.lib()


def test_every_declared_symbol_is_exported(lib):
    names = R.declared_symbols()
    assert {"rhosvd_sketch", "rhosvd_power", "rhosvd_orth", "rhosvd_core", "rhosvd_decompose",
            "rhosvd_sketch_all", "rhosvd_omega", "rhosvd_workspace_size"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for code in range(8):
        assert lib.rhosvd_status_string(code)
    assert lib.rhosvd_status_string(0) == b"ok"


@pytest.mark.parametrize("algo", ["rhosvd", "rsthosvd"])
@pytest.mark.parametrize("dims,ranks,p", [((512, 512, 512), (32, 32, 32), 10), ((100, 100, 100), (10, 10, 10), 5),
                                          ((7, 30, 9, 11), (7, 4, 2, 5), 3), ((5, 400), (5, 3), 10)])
def test_plan_matches_oracle_width_rule(lib, algo, dims, ranks, p):
    K, S, J = R.rhosvd_plan(dims, ranks, algo=algo, p=p, q=1)
    want = A.omega_shapes(algo, dims, ranks, p)
    assert [(j, k) for j, k in zip(J, K)] == [tuple(w) for w in want]


def test_plan_rpet_overrides(lib):
    dims, ranks = (128, 128, 128, 128), (16,) * 4
    K, S, J = R.rhosvd_plan(dims, ranks, algo="rpet", p=10, q=0, K=(26,) * 4, S=(40,) * 4)
    assert K == [26] * 4 and S == [40] * 4 and J == [128 ** 3] * 4
    K, S, J = R.rhosvd_plan(dims, ranks, algo="rpet", p=10, q=0)
    assert K == [26] * 4 and S == [53] * 4      # defaults K = R + p, S = 2K + 1 (Sec. 8)
    shapes, tilde = A.omega_shapes("rpet", dims, ranks, 10)
    assert [k for _, k in shapes] == K and [s for s, _ in tilde] == S


def test_workspace_sizes(lib):
    small = R.rhosvd_workspace_size((100, 100, 100), (10, 10, 10), algo="rhosvd", p=5, q=0)
    big = R.rhosvd_workspace_size((512, 512, 512), (32, 32, 32), algo="rsthosvd", p=10, q=1)
    assert 0 < small < big
    # the mode-1 test matrix and power-iteration block (262144 x 42 floats each) must fit
    assert big >= 2 * 262144 * 42 * 4
    assert R.rhosvd_workspace_size((512, 512, 512), (600, 32, 32), algo="rsthosvd") == 0


def _call_decompose(lib, dims, ranks, opts, ws_bytes=1 << 20, ws=256 * 16):
    sh = R.make_shape(dims)
    r = R._i32(ranks)
    U = (ctypes.c_void_p * 8)(*([256 * 64] * 8))
    return lib.rhosvd_decompose(ctypes.c_void_p(256 * 32), ctypes.byref(sh), r, ctypes.byref(opts), None, None,
                                U, ctypes.c_void_p(256 * 48), ctypes.c_void_p(ws), ws_bytes, None)


@pytest.mark.parametrize("dims,ranks,kw", [
    ((10, 10, 10), (0, 3, 3), {}),               # rank 0
    ((10, 10, 10), (11, 3, 3), {}),              # rank above I_n
    ((10, 10, 10), (3, 3, 3), {"p": -1}),        # negative oversampling
    ((10, 10, 10), (3, 3, 3), {"q": -2}),
    ((200, 200, 200), (120, 3, 3), {"p": 20}),   # K above RHOSVD_MAX_K
    ((0, 10, 10), (1, 3, 3), {}),                # empty mode
])
def test_decompose_rejects_bad_arguments(lib, dims, ranks, kw):
    opts = R.make_opts("rsthosvd", kw.get("p", 5), kw.get("q", 1), 0)
    assert _call_decompose(lib, dims, ranks, opts) == 1   # RHOSVD_EINVAL


def test_decompose_rejects_short_or_misaligned_workspace(lib):
    opts = R.make_opts("rsthosvd", 5, 1, 0)
    assert _call_decompose(lib, (64, 64, 64), (8, 8, 8), opts, ws_bytes=4096) == 2      # RHOSVD_ENOMEM
    assert _call_decompose(lib, (64, 64, 64), (8, 8, 8), opts, ws_bytes=1 << 30, ws=257) == 1


def test_primitive_argument_checks(lib):
    sh = R.make_shape((16, 16, 16))
    ws = ctypes.c_void_p(1 << 20)
    assert lib.rhosvd_sketch(None, ctypes.byref(sh), 0, 4, 0, None, ctypes.c_void_p(4096), ws, 1 << 30, None) == 1
    assert lib.rhosvd_sketch(ctypes.c_void_p(4096), ctypes.byref(sh), 3, 4, 0, None, ctypes.c_void_p(4096), ws,
                             1 << 30, None) == 1
    assert lib.rhosvd_orth(ctypes.c_void_p(4096), 3, 4, 3, None, ws, 1 << 30, None) == 1       # m < K
    assert lib.rhosvd_orth(ctypes.c_void_p(4096), 30, 200, 30, None, ws, 1 << 30, None) == 1   # K > MAX_K
    assert lib.rhosvd_omega(0, 0, 10, 4, None, 10, None) == 1
    assert lib.rhosvd_omega(0, 0, 10, 4, ctypes.c_void_p(4096), 5, None) == 1                   # ld < rows
    assert lib.rhosvd_omega(0, 0, 0, 4, None, 0, None) == 0                                     # empty is a no-op
    assert lib.rhosvd_device_status(None, 0, None, None) == 1


class _FakeStream:
    def __init__(self, sid):
        self.sid = sid

    def __eq__(self, other):
        return isinstance(other, _FakeStream) and other.sid == self.sid


class _FakeTensor:
    def __init__(self):
        self.recorded = []

    def record_stream(self, s):
        self.recorded.append(s.sid)


def test_binding_holds_its_buffers_only_for_another_stream():
    cur, other = _FakeStream(0), _FakeStream(1)
    a, b = _FakeTensor(), _FakeTensor()
    R._hold(None, a, current=cur)                    # the current stream: nothing to do
    R._hold(_FakeStream(0), a, current=cur)
    assert a.recorded == []
    R._hold(other, a, None, b, current=cur)          # another stream: every buffer, None skipped
    assert a.recorded == [1] and b.recorded == [1]


def test_header_is_plain_c(tmp_path):
    """include/rhosvd.h is a C header: a C11 translation unit that includes it and
    calls the decomposition entry points compiles without warnings."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use.c"
    src.write_text(
        '#include "rhosvd.h"\n'
        "int use(const float* X, float* U[3], float* G, void* ws, void* stream) {\n"
        "  rhosvd_shape shape = {3, {40, 50, 60}};\n"
        "  int32_t ranks[3] = {5, 6, 7};\n"
        "  rhosvd_opts opts = {.algo = RHOSVD_ALGO_RSTHOSVD, .p = 5, .q = 1, .seed = 7};\n"
        "  size_t n = rhosvd_workspace_size(&shape, ranks, &opts);\n"
        "  rhosvd_status s = rhosvd_decompose(X, &shape, ranks, &opts, 0, 0, U, G, ws, n, stream);\n"
        "  return s == RHOSVD_OK ? (int)rhosvd_device_status(ws, n, stream, 0) : (int)s;\n"
        "}\n")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    r = subprocess.run([gcc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-fsyntax-only", "-I", inc, str(src)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
