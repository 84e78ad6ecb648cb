"""The persistent batched R-STHOSVD (rhosvd_batch_*, one launch for many small
tensors) against the FP64 oracle, through the C ABI.

Every item is compared with the oracle's R-STHOSVD (Alg. 8) on the same
seeded test matrices (the oracle draws them from its own Philox
implementation, mode n on stream_id n) within the FP32-path tolerances: largest
principal-angle sine <= 1e-4 per mode, |E_gpu - E_oracle| <= 1e-5,
orthonormality <= 1e-5.  Also: the autotuner keeps a launchable configuration
and the result still matches; a captured CUDA graph of the launch replays to
bitwise the eager result; modes with R_n = I_n are skipped; a zero tensor gives
finite outputs; invalid requests are rejected on the host.
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


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def _oracle(x32, dims, ranks, p, q, seed):
    shapes = A.omega_shapes("rsthosvd", dims, ranks, p)
    om = [philox.omega(seed, n, r, c).astype(np.float64) for n, (r, c) in enumerate(shapes)]
    return A.rsthosvd(x32, ranks, q, om)


def _check_item(x32, g, us, dims, ranks, p, q, seed):
    g_or, u_or = _oracle(x32, dims, ranks, p, q, seed)
    e_gpu, e_or = M.rel_error(x32, g, us), M.rel_error(x32, g_or, u_or)
    sines = [M.max_principal_sine(a, b) for a, b in zip(us, u_or)]
    assert max(sines) <= 1e-4, (dims, ranks, sines)
    assert abs(e_gpu - e_or) <= 1e-5, (dims, ranks, e_gpu, e_or)
    assert max(M.orthonormality(u) for u in us) <= 1e-5
    return e_gpu, e_or


def _uneven_batch(n, seed0, lo=16, hi=97, rlo=4, rhi=16):
    # ranks stay below every mode size: a mode with R_n = I_n is skipped by the
    # device (identity factor) but rotated by the oracle, which changes the test
    # matrices the later modes effectively see (covered separately, last mode)
    rng = np.random.default_rng(seed0)
    items, xs = [], []
    for b in range(n):
        dims = tuple(int(v) for v in rng.integers(lo, hi, size=3))
        ranks = tuple(int(min(r, d)) for r, d in zip(rng.integers(rlo, rhi, size=3), dims))
        x = lowrank_tensor(dims, ranks, seed0 + 1 + b, noise=1e-3)
        xs.append(f32(x))
        items.append((torch.from_numpy(device_layout(x)).cuda(), dims, ranks))
    return items, xs


def test_persistent_batch_of_small_uneven_tensors_matches_oracle():
    """Modes uniform in [16, 96], ranks uniform in [4, 15], p = 5, q = 1, low
    rank plus 1e-3 noise: every item agrees with the oracle."""
    items, xs = _uneven_batch(32, 3000)
    batch = R().BatchPersistent(items, p=5, q=1, seed=9)
    batch.run()
    torch.cuda.synchronize()
    assert batch.device_status() == 0
    for (g, us), (X, dims, ranks), x32 in zip(batch.results(), items, xs):
        _check_item(x32, host(g), [host(u) for u in us], dims, ranks, 5, 1, 9)


@pytest.mark.parametrize("dims,ranks,p,q", [
    ((20, 24, 18, 16), (4, 5, 3, 16), 4, 1),      # 4-way, last mode skipped (R = I)
    ((40, 30, 16), (6, 5, 16), 5, 2),             # last mode skipped, two power steps
    ((200, 24), (7, 7), 6, 0),                    # 2-way, a 200-row mode, no power step
    ((33, 17, 65), (5, 4, 6), 3, 1),              # odd sizes, ragged tiles
    ((256, 24, 10), (6, 5, 4), 5, 1),             # the largest mode size (shared-memory bound)
    ((256, 256), (20, 20), 6, 1),                 # 2-way, both modes at the limit, K = 26
])
def test_persistent_batch_shapes(dims, ranks, p, q):
    x = lowrank_tensor(dims, ranks, 77, noise=1e-3)
    items = [(torch.from_numpy(device_layout(x)).cuda(), dims, ranks)]
    batch = R().BatchPersistent(items, p=p, q=q, seed=5)
    batch.run()
    torch.cuda.synchronize()
    assert batch.device_status() == 0
    (g, us), = batch.results()
    _check_item(f32(x), host(g), [host(u) for u in us], dims, ranks, p, q, 5)


def test_tuner_keeps_a_valid_configuration_and_the_result():
    items, xs = _uneven_batch(64, 4000)
    batch = R().BatchPersistent(items, p=5, q=1, seed=3)
    ms = batch.tune()
    cfg = batch.config
    assert ms > 0.0
    assert cfg["threads"] in (128, 256, 512) and cfg["tile_columns"] in (32, 64) and 1 <= cfg["ctas_per_sm"] <= 4
    batch.run()
    torch.cuda.synchronize()
    for (g, us), (X, dims, ranks), x32 in list(zip(batch.results(), items, xs))[:16]:
        _check_item(x32, host(g), [host(u) for u in us], dims, ranks, 5, 1, 3)


def test_graph_replay_is_bitwise_the_eager_result():
    items, _ = _uneven_batch(40, 5000)
    batch = R().BatchPersistent(items, p=5, q=1, seed=11)
    batch.run()
    torch.cuda.synchronize()
    eager = [(host(g), [host(u) for u in us]) for g, us in batch.results()]
    for g, us in batch.results():
        g.zero_()
        for u in us:
            u.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batch.run()
    graph.replay()
    torch.cuda.synchronize()
    for (g0, u0), (g, us) in zip(eager, batch.results()):
        np.testing.assert_array_equal(g0, host(g))
        for a, b in zip(u0, us):
            np.testing.assert_array_equal(a, host(b))


def test_zero_tensor_gives_finite_outputs():
    dims, ranks = (24, 20, 18), (3, 4, 2)
    X = torch.zeros(int(np.prod(dims)), device="cuda")
    batch = R().BatchPersistent([(X, dims, ranks)], p=4, q=1, seed=1)
    batch.run()
    torch.cuda.synchronize()
    (g, us), = batch.results()
    assert np.all(host(g) == 0.0)
    for u, r in zip(us, ranks):
        uh = host(u)
        assert np.all(np.isfinite(uh))
        assert M.orthonormality(uh) <= 1e-5


def test_invalid_requests_are_rejected():
    rh = R()
    x = torch.zeros(300 * 20 * 4, device="cuda")
    with pytest.raises(rh.RhosvdError):                          # a mode above 256
        rh.BatchPersistent([(x, (300, 20, 4), (4, 4, 2))], p=5, q=1)
    y = torch.zeros(40 * 40 * 40, device="cuda")
    with pytest.raises(rh.RhosvdError):                          # sketch width above 32
        rh.BatchPersistent([(y, (40, 40, 40), (30, 4, 4))], p=5, q=1)
    with pytest.raises(ValueError):
        rh.BatchPersistent([(y, (40, 40, 40), (4, 4, 4))], algo="rpet")
