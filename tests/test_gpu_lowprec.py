"""Reduced-precision sketch passes and the RP-HOOI refinement, through the C ABI.

* The BF16 / e4m3 single pass of R-PET computes, apart from FP32 accumulation,
  the R-PET of the quantized tensor X_q (BF16, or e4m3 with one power-of-two
  scale per frontal slice of the last mode) with test matrices rounded to the
  format.  The oracle runs exactly that in FP64 (oracle.precision makes X_q and
  the rounded test matrices from their definitions), and the GPU result meets
  the FP32-path tolerances against it: largest principal-angle sine <= 1e-4
  per mode and |E_gpu - E_oracle| <= 1e-5, E measured against the FP32 X.
* One RP-HOOI sweep (Alg. 7) after the decomposition, on the FP32 X, with the
  sweep's test matrices seeded on stream_id 2N + n: against the oracle's sweep
  from the oracle's own decomposition, same tolerances.
* Against the FP64 oracle on the unquantized tensor (the reduced-precision
  tolerance): with one refinement sweep, E within 2% of the oracle's refined E
  and within 1e-3 absolute.
* The mode-1 power products of R-STHOSVD on the BF16 copy: the same
  reduced-precision tolerance against the FP64 oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import algorithms as A  # noqa: E402
from oracle import metrics as M  # noqa: E402
from oracle import philox  # noqa: E402
from oracle import precision as P  # noqa: E402
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


def _gpu_rpet(x, dims, ranks, K, S, om, ot, dtype, refine=0, p=10, seed=0):
    G, U = R().rhosvd_decompose(dev(x), dims, ranks, algo="rpet", p=p, K=K, S=S, seed=seed,
                                Omega=[dev_mat(o) for o in om], Omega_tilde=[dev_mat(o) for o in ot],
                                dtype=dtype, refine=refine)
    return host(G), [host(u) for u in U]


def _refine_omegas(seed, dims, ranks, p, sweep=0):
    n_modes = len(dims)
    return [philox.omega(seed, 2 * n_modes + sweep * n_modes + n, j, k).astype(np.float64)
            for n, (j, k) in enumerate(A.rp_hooi_omega_shapes(dims, ranks, p))]


def _compare(x32, g, u, g_or, u_or, tol=1e-5, sine=1e-4):
    e_gpu, e_or = M.rel_error(x32, g, u), M.rel_error(x32, g_or, u_or)
    sines = [M.max_principal_sine(a, b) for a, b in zip(u, u_or)]
    assert abs(e_gpu - e_or) <= tol, (e_gpu, e_or)
    assert max(sines) <= sine, sines
    assert max(M.orthonormality(v) for v in u) <= 1e-5
    return e_gpu, e_or


# every mode in a layout the reduced-precision kernels take (rows 8 / 16 elements
# aligned, fibre lengths multiples of 32, slices of whole stages); the first has
# only short modes (one 128-row tile per CTA), the second a 256-row mode too
CASES = [((64, 48, 40, 32), (4, 4, 4, 3)), ((256, 128, 48), (6, 5, 4))]


@pytest.mark.parametrize("dtype", ["bf16", "e4m3"])
@pytest.mark.parametrize("dims,ranks", CASES)
def test_reduced_precision_single_pass_is_rpet_of_the_quantized_tensor(dims, ranks, dtype):
    x32 = f32(lowrank_tensor(dims, ranks, seed=70, noise=1e-2))
    K = [r + 6 for r in ranks]
    S = [2 * k + 1 for k in K]
    shapes, tilde = A.omega_shapes("rpet", dims, ranks, 0, K=K, S=S)
    om = [P.round_to(gaussian_matrix(80 + n, r, c), dtype) for n, (r, c) in enumerate(shapes)]
    ot = [P.round_to(gaussian_matrix(90 + n, r, c), dtype) for n, (r, c) in enumerate(tilde)]
    g, u = _gpu_rpet(x32, dims, ranks, K, S, om, ot, dtype)
    xq, _ = P.quantize(x32, dtype)
    g_or, u_or, _ = A.rpet(np.asfortranarray(xq), ranks, om, ot)
    e_gpu, e_or = _compare(x32, g, u, g_or, u_or)
    print(f"{dtype} {dims}: E_gpu {e_gpu:.6e} E_oracle(X_q) {e_or:.6e}")


@pytest.mark.parametrize("dtype", ["f32", "bf16", "e4m3"])
def test_refinement_sweep_matches_the_oracle_sweep(dtype):
    """Noise 1e-3: there one randomized sweep fixes the subspaces to a few 1e-5
    (two test-matrix draws give results 4e-5 apart), so the FP32-path sine bar
    applies; at noise 1e-2 the draws already differ by 3e-4."""
    dims, ranks = (64, 48, 40, 32), (4, 4, 4, 3)
    p, seed = 10, 5
    x32 = f32(lowrank_tensor(dims, ranks, seed=71, noise=1e-3))
    K = [r + 6 for r in ranks]
    S = [2 * k + 1 for k in K]
    shapes, tilde = A.omega_shapes("rpet", dims, ranks, 0, K=K, S=S)
    om = [P.round_to(gaussian_matrix(81 + n, r, c), dtype) for n, (r, c) in enumerate(shapes)]
    ot = [P.round_to(gaussian_matrix(91 + n, r, c), dtype) for n, (r, c) in enumerate(tilde)]
    g, u = _gpu_rpet(x32, dims, ranks, K, S, om, ot, dtype, refine=1, p=p, seed=seed)
    xq, _ = P.quantize(x32, dtype)
    _, u0, _ = A.rpet(np.asfortranarray(xq), ranks, om, ot)
    g_or, u_or = A.rp_hooi_sweep(x32, u0, ranks, _refine_omegas(seed, dims, ranks, p))
    e_gpu, e_or = _compare(x32, g, u, g_or, u_or)
    # the refinement reaches (near) the HOOI error whatever the single pass's precision
    g_h, u_h = A.hooi(x32, ranks, sweeps=5)
    assert e_gpu <= 1.02 * M.rel_error(x32, g_h, u_h)
    print(f"{dtype} + 1 sweep: E_gpu {e_gpu:.6e} E_oracle {e_or:.6e}")


@pytest.mark.parametrize("dtype", ["bf16", "e4m3"])
def test_refined_reduced_precision_meets_the_reduced_precision_tolerance(dtype):
    """Against the FP64 oracle on the unquantized tensor: R-PET with the same
    (rounded) test matrices plus one RP-HOOI sweep, |dE| <= 2% E and <= 1e-3."""
    dims, ranks = (64, 48, 40, 32), (4, 4, 4, 3)
    p, seed = 10, 6
    x32 = f32(lowrank_tensor(dims, ranks, seed=72, noise=1e-3))
    K = [r + 6 for r in ranks]
    S = [2 * k + 1 for k in K]
    shapes, tilde = A.omega_shapes("rpet", dims, ranks, 0, K=K, S=S)
    om = [P.round_to(gaussian_matrix(82 + n, r, c), dtype) for n, (r, c) in enumerate(shapes)]
    ot = [P.round_to(gaussian_matrix(92 + n, r, c), dtype) for n, (r, c) in enumerate(tilde)]
    g, u = _gpu_rpet(x32, dims, ranks, K, S, om, ot, dtype, refine=1, p=p, seed=seed)
    _, u0, _ = A.rpet(x32, ranks, om, ot)
    g_or, u_or = A.rp_hooi_sweep(x32, u0, ranks, _refine_omegas(seed, dims, ranks, p))
    e_gpu, e_or = M.rel_error(x32, g, u), M.rel_error(x32, g_or, u_or)
    print(f"{dtype} refined: E_gpu {e_gpu:.6e} E_oracle(FP64, unquantized) {e_or:.6e}")
    assert abs(e_gpu - e_or) <= 0.02 * e_or and abs(e_gpu - e_or) <= 1e-3


@pytest.mark.parametrize("dtype", ["bf16", "e4m3"])
def test_mixed_layouts_with_refinement(dtype):
    """A tensor where some modes fall outside the reduced-precision kernels'
    layouts (those passes run in FP32): with one refinement sweep the result
    still meets the reduced-precision tolerance against the FP64 oracle."""
    dims, ranks = (40, 30, 20), (4, 3, 2)
    p, seed = 10, 7
    x32 = f32(lowrank_tensor(dims, ranks, seed=75, noise=1e-3))
    K = [r + 6 for r in ranks]
    S = [2 * k + 1 for k in K]
    shapes, tilde = A.omega_shapes("rpet", dims, ranks, 0, K=K, S=S)
    om = [P.round_to(gaussian_matrix(84 + n, r, c), dtype) for n, (r, c) in enumerate(shapes)]
    ot = [P.round_to(gaussian_matrix(94 + n, r, c), dtype) for n, (r, c) in enumerate(tilde)]
    g, u = _gpu_rpet(x32, dims, ranks, K, S, om, ot, dtype, refine=1, p=p, seed=seed)
    _, u0, _ = A.rpet(x32, ranks, om, ot)
    g_or, u_or = A.rp_hooi_sweep(x32, u0, ranks, _refine_omegas(seed, dims, ranks, p))
    e_gpu, e_or = M.rel_error(x32, g, u), M.rel_error(x32, g_or, u_or)
    assert abs(e_gpu - e_or) <= 0.02 * e_or and abs(e_gpu - e_or) <= 1e-3, (e_gpu, e_or)


def test_bf16_power_products_of_rsthosvd():
    dims, ranks, p, q = (256, 96, 80), (12, 10, 8), 8, 1
    x32 = f32(lowrank_tensor(dims, ranks, seed=73, noise=1e-3))
    shapes = A.omega_shapes("rsthosvd", dims, ranks, p)
    om = [gaussian_matrix(83 + n, r, c) for n, (r, c) in enumerate(shapes)]
    G, U = R().rhosvd_decompose(dev(x32), dims, ranks, algo="rsthosvd", p=p, q=q,
                                Omega=[dev_mat(o) for o in om], dtype="bf16")
    g, u = host(G), [host(v) for v in U]
    g_or, u_or = A.rsthosvd(x32, ranks, q, [o.astype(np.float64) for o in om])
    e_gpu, e_or = M.rel_error(x32, g, u), M.rel_error(x32, g_or, u_or)
    print(f"R-STHOSVD bf16 power: E_gpu {e_gpu:.6e} E_oracle {e_or:.6e}")
    assert abs(e_gpu - e_or) <= 0.02 * e_or and abs(e_gpu - e_or) <= 1e-3
    assert max(M.orthonormality(v) for v in u) <= 1e-5


def test_seeded_reduced_precision_run_and_launch_count():
    """Seed-drawn (rounded) test matrices: the decomposition runs, reports a clean
    device status, and enqueues the number of kernels rhosvd_launch_count gives
    (compared with the FP32 run it adds the quantisation and rounding kernels)."""
    dims, ranks = (64, 48, 40, 32), (4, 4, 4, 3)
    K = [r + 6 for r in ranks]
    S = [2 * k + 1 for k in K]
    x32 = f32(lowrank_tensor(dims, ranks, seed=74, noise=1e-2))
    ws = R().Workspace(R().rhosvd_workspace_size(dims, ranks, "rpet", 10, 0, K=K, S=S, dtype="e4m3", refine=1))
    G, U = R().rhosvd_decompose(dev(x32), dims, ranks, algo="rpet", K=K, S=S, dtype="e4m3", refine=1, ws=ws)
    assert R().rhosvd_device_status(ws)[0] == 0
    e = M.rel_error(x32, host(G), [host(v) for v in U])
    assert e < 2e-2
    n32 = R().rhosvd_launch_count(dims, ranks, "rpet", 10, 0, K=K, S=S)
    n8 = R().rhosvd_launch_count(dims, ranks, "rpet", 10, 0, K=K, S=S, dtype="e4m3")
    assert n8 > n32 > 0
