"""R-PET with Kronecker-structured factor sketches (the memory-efficient test
matrices of Sec. 5.1), two reads of X, through the C ABI.

The factor sketch of mode n is X_(n) (Phi_N x ... x Phi_1 without Phi_n); the
oracle's R-PET receives that Kronecker product as an explicit test matrix
(oracle.algorithms.kronecker_test_matrix), the GPU the small Phi_p, and the two
must agree within the FP32-path tolerances (principal-angle sines <= 1e-4 per
mode, |E_gpu - E_oracle| <= 1e-5).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import algorithms as A  # noqa: E402
from oracle import metrics as M  # noqa: E402
from oracle import philox  # noqa: E402
from workloads import device_layout, gaussian_matrix, lowrank_tensor  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2001_07124_gb300 as pkg
    pkg.build()
    pkg.rhosvd.lib()
    torch.cuda.set_device(0)


def R():
    from paper_2001_07124_gb300 import rhosvd
    return rhosvd


def dev(x):
    return torch.from_numpy(device_layout(np.asarray(x))).cuda()


def dev_mat(m):
    return torch.from_numpy(np.asfortranarray(m, dtype=np.float32).ravel(order="F")).cuda()


def f32(x):
    return np.asfortranarray(np.asarray(x).astype(np.float32).astype(np.float64))


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("dims,ranks,K", [((64, 48, 40, 32), (4, 4, 4, 3), 10), ((60, 50, 70), (5, 4, 6), 12),
                                          ((40, 36), (4, 4), 9), ((128, 96, 64), (8, 8, 8), 20)])
def test_kronecker_rpet_matches_oracle(dims, ranks, K):
    N = len(dims)
    x32 = f32(lowrank_tensor(dims, ranks, seed=76, noise=1e-3))
    Kp, Sp, _ = R().rhosvd_plan(dims, ranks, "rpet", 0, 0, K=[K] * N, kron=True)
    k = int(round(Kp[0] ** (1.0 / (N - 1))))
    assert k ** (N - 1) == Kp[0] >= K and (k - 1) ** (N - 1) < K
    phis = [gaussian_matrix(110 + p, dims[p], k) for p in range(N)]
    ot = [gaussian_matrix(120 + n, Sp[n], dims[n]) for n in range(N)]
    G, U = R().rhosvd_decompose(dev(x32), dims, ranks, algo="rpet", K=[K] * N, kron=True,
                                Omega=[dev_mat(f) for f in phis], Omega_tilde=[dev_mat(o) for o in ot])
    g, u = host(G), [host(v) for v in U]
    om = [A.kronecker_test_matrix([f.astype(np.float64) for f in phis], n) for n in range(N)]
    g_or, u_or, _ = A.rpet(x32, ranks, om, [o.astype(np.float64) for o in ot])
    e_gpu, e_or = M.rel_error(x32, g, u), M.rel_error(x32, g_or, u_or)
    sines = [M.max_principal_sine(a, b) for a, b in zip(u, u_or)]
    print(f"{dims} k={k}: E_gpu {e_gpu:.6e} E_oracle {e_or:.6e} max sine {max(sines):.2e}")
    assert abs(e_gpu - e_or) <= 1e-5 and max(sines) <= 1e-4
    assert max(M.orthonormality(v) for v in u) <= 1e-5


def test_kronecker_rpet_seeded_matches_oracle_generator():
    """Phi_p drawn on stream_id 10N + p and Omega~_n on N + n, on both sides."""
    dims, ranks, K = (64, 48, 40, 32), (4, 4, 4, 3), 10
    N, seed = 4, 3
    x32 = f32(lowrank_tensor(dims, ranks, seed=77, noise=1e-3))
    Kp, Sp, _ = R().rhosvd_plan(dims, ranks, "rpet", 0, 0, K=[K] * N, kron=True)
    k = int(round(Kp[0] ** (1.0 / (N - 1))))
    G, U = R().rhosvd_decompose(dev(x32), dims, ranks, algo="rpet", K=[K] * N, kron=True, seed=seed)
    g, u = host(G), [host(v) for v in U]
    phis = [philox.omega(seed, 10 * N + p, dims[p], k).astype(np.float64) for p in range(N)]
    ot = [philox.omega(seed, N + n, Sp[n], dims[n]).astype(np.float64) for n in range(N)]
    om = [A.kronecker_test_matrix(phis, n) for n in range(N)]
    g_or, u_or, _ = A.rpet(x32, ranks, om, ot)
    assert abs(M.rel_error(x32, g, u) - M.rel_error(x32, g_or, u_or)) <= 1e-5
    assert max(M.max_principal_sine(a, b) for a, b in zip(u, u_or)) <= 1e-4


def test_kronecker_option_is_validated():
    with pytest.raises(Exception):                      # only R-PET takes the option
        R().rhosvd_plan((32, 32, 32), (4, 4, 4), "rsthosvd", 5, 1, kron=True)
    with pytest.raises(Exception):                      # k^(N-1) columns must fit the modes
        R().rhosvd_plan((8, 8, 8), (4, 4, 4), "rpet", 0, 0, K=[60] * 3, kron=True)
