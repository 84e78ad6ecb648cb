"""Fixed-accuracy R-STHOSVD on the GPU (rhosvd_decompose_tol) against the
oracle's rsthosvd_fixed_accuracy with the same seeded test blocks (block i of
mode n on stream_id 4096 + 256 n + i).

Checks: the GPU meets the guarantee ||X - X_hat||_F <= eps ||X||_F, chooses the
oracle's ranks, and its E agrees with the oracle's within the FP32-path
tolerance (1e-5); on a tensor of exact multilinear rank with a tolerance far
above the noise it recovers that rank.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import algorithms as A  # noqa: E402
from oracle import metrics as M  # noqa: E402
from oracle import philox  # noqa: E402
from workloads import device_layout, lowrank_tensor  # noqa: E402

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


def f32(x):
    return np.asfortranarray(np.asarray(x).astype(np.float32).astype(np.float64))


def _blocks(seed):
    def f(n, i, j, b):
        return philox.omega(seed, 4096 + 256 * n + i, j, b).astype(np.float64)
    return f


@pytest.mark.parametrize("dims,ranks,decay,noise,eps,block", [
    ((96, 80, 64), (20, 20, 20), 0.9, 1e-4, 1e-2, 8), ((96, 80, 64), (20, 20, 20), 0.8, 1e-4, 0.1, 8),
    ((128, 64, 48), (16, 12, 10), 0.85, 1e-3, 3e-2, 6),
    ((40, 30, 20, 12), (6, 5, 4, 3), None, 1e-3, 1e-2, 4)])
def test_fixed_accuracy_matches_oracle(dims, ranks, decay, noise, eps, block):
    seed = 11
    x32 = f32(lowrank_tensor(dims, ranks, seed=78, noise=noise, decay=decay))
    k_max = [min(d, 64) for d in dims]
    X = torch.from_numpy(device_layout(x32)).cuda()
    G, U, r = R().rhosvd_decompose_tol(X, dims, eps, block=block, k_max=k_max, seed=seed)
    g = G.detach().cpu().numpy().astype(np.float64)
    u = [v.detach().cpu().numpy().astype(np.float64) for v in U]
    g_or, u_or, r_or = A.rsthosvd_fixed_accuracy(x32, eps, block, k_max, _blocks(seed))
    e_gpu, e_or = M.rel_error(x32, g, u), M.rel_error(x32, g_or, u_or)
    print(f"{dims} eps={eps}: ranks gpu {r} oracle {r_or}, E_gpu {e_gpu:.6e} E_oracle {e_or:.6e}")
    assert e_gpu <= eps
    assert list(r) == list(r_or)
    assert abs(e_gpu - e_or) <= 1e-5
    assert max(M.orthonormality(v) for v in u) <= 1e-5


def test_fixed_accuracy_recovers_exact_rank():
    dims, ranks = (64, 56, 48), (7, 5, 6)
    x32 = f32(lowrank_tensor(dims, ranks, seed=79, noise=1e-6))
    X = torch.from_numpy(device_layout(x32)).cuda()
    G, U, r = R().rhosvd_decompose_tol(X, dims, 1e-3, block=4, k_max=[32, 32, 32], seed=2)
    assert list(r) == list(ranks)
    e = M.rel_error(x32, G.detach().cpu().numpy().astype(np.float64),
                    [v.detach().cpu().numpy().astype(np.float64) for v in U])
    assert e <= 1e-5


def test_fixed_accuracy_rejects_bad_arguments():
    dims = (16, 16, 16)
    X = torch.zeros(16 ** 3, device="cuda")
    for eps, block, k_max in [(0.0, 4, [8] * 3), (1.5, 4, [8] * 3), (0.1, 0, [8] * 3), (0.1, 4, [17, 8, 8])]:
        with pytest.raises(Exception):
            R().rhosvd_decompose_tol(X, dims, eps, block=block, k_max=k_max)
