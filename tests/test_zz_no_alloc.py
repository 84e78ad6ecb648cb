"""The workspace-free sketch entry point (rhosvd_sketch_noalloc).

It exists for callers that cannot allocate device memory where they need a
sketch (a foreign memory pool, a plug-in handed only its buffers, a loop where
cudaMalloc's implicit synchronisation is not allowed): its split-K scratch is a
fixed device array inside the library.  The test calls it through the C ABI
twice in a row, on different inputs, and checks each result against the
existing rhosvd_sketch entry point within the sketch tolerance used by the
parity tests, and against the oracle's product of the same unfolding and
test matrix in FP64.  This file is collected last so that a stop-at-first-failure run
has already run every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import tensor as T  # noqa: E402
from workloads import device_layout, gaussian_matrix, random_tensor  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2001_07124_gb300 as pkg
    pkg.build()
    from paper_2001_07124_gb300 import rhosvd
    rhosvd.lib()
    torch.cuda.set_device(0)
    return rhosvd


def _noalloc(R, X, dims, mode, K, om, Y):
    code = R.lib().rhosvd_sketch_noalloc(X.data_ptr(), ctypes.byref(R.make_shape(dims)), mode, K, om.data_ptr(),
                                         Y.data_ptr(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 0, R.STATUS.get(code)
    torch.cuda.synchronize()
    return R.matrix(Y, dims[mode], K).cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("dims,mode,K", [((512, 96, 80), 0, 42), ((67, 45, 83), 1, 17)])
def test_noalloc_sketch_matches_workspace_sketch_twice(R, dims, mode, K):
    J = int(np.prod(dims)) // dims[mode]
    for call in range(2):                      # two calls in a row share the scratch array
        x = random_tensor(dims, 50 + call)
        X = torch.from_numpy(device_layout(x)).cuda()
        om_h = gaussian_matrix(60 + call, J, K)
        om = torch.from_numpy(om_h.ravel(order="F")).cuda()
        Y = torch.full((dims[mode] * K,), float("nan"), device="cuda")
        got = _noalloc(R, X, dims, mode, K, om, Y)
        want = R.rhosvd_sketch(X, dims, mode, K, Omega=om).cpu().numpy().astype(np.float64)
        a = T.unfold(x.astype(np.float32).astype(np.float64), mode)
        om64 = om_h.astype(np.float64)
        exact = a @ om64                               # the oracle's Y = X_(n) Omega in FP64
        bound = np.abs(a) @ np.abs(om64)
        assert np.all(np.isfinite(got))
        assert np.all(np.abs(got - exact) <= 1e-5 * bound + 1e-30)
        assert np.all(np.abs(got - want) <= 1e-5 * bound + 1e-30)


def test_noalloc_rejects_oversized_requests(R):
    dims = (40000, 4, 4)            # I * K = 40000 * 64 > 2^20 floats of scratch
    X = torch.zeros(int(np.prod(dims)), device="cuda")
    om = torch.zeros(16 * 64, device="cuda")
    Y = torch.zeros(40000 * 64, device="cuda")
    code = R.lib().rhosvd_sketch_noalloc(X.data_ptr(), ctypes.byref(R.make_shape(dims)), 0, 64, om.data_ptr(),
                                         Y.data_ptr(), None)
    assert code == 1   # RHOSVD_EINVAL, nothing enqueued
    code = R.lib().rhosvd_sketch_noalloc(X.data_ptr(), ctypes.byref(R.make_shape(dims)), 0, 4, None,
                                         Y.data_ptr(), None)
    assert code == 1   # Omega is required
    # sizes whose product overflows 64-bit arithmetic are rejected like everywhere else
    big = R.make_shape((1, 2 ** 40, 2 ** 40))
    code = R.lib().rhosvd_sketch_noalloc(X.data_ptr(), ctypes.byref(big), 0, 1, om.data_ptr(), Y.data_ptr(), None)
    assert code == 1
