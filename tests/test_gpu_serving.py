"""Served decompositions (several requests on the device at once, on their own
streams) give bitwise the results of the same decompositions run alone."""
import numpy as np
import pytest

from workloads import device_layout, lowrank_tensor

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2001_07124_gb300 as pkg
    pkg.build()
    pkg.rhosvd.lib()


def test_served_results_equal_results_alone():
    from paper_2001_07124_gb300 import rhosvd as R
    from paper_2001_07124_gb300.serving import Request, latency_summary, serve
    shapes = [((96, 80, 64), (8, 7, 6)), ((128, 128, 128), (16, 16, 16)), ((64, 72, 40), (5, 9, 4)),
              ((160, 96, 112), (12, 10, 14)), ((48, 48, 48, 20), (4, 4, 4, 3)), ((200, 150, 100), (20, 15, 10))]
    reqs = []
    for i, (dims, ranks) in enumerate(shapes):
        x = lowrank_tensor(dims, ranks, 500 + i, noise=1e-3)
        xh = torch.from_numpy(device_layout(x)).pin_memory()
        reqs.append(Request(i, dims, ranks, arrival=0.0, x_host=xh, p=5, q=1, seed=7 + i))
    res = serve(reqs, slots=3, budget_bytes=2 * 10 ** 9)
    assert sorted(r.rid for r in res) == list(range(len(reqs)))
    s = latency_summary(res)
    assert s["requests"] == len(reqs) and s["p99_ms"] >= s["p50_ms"] > 0
    for r in res:
        q = reqs[r.rid]
        G, Us = R.empty_colmajor(q.ranks), [R.empty_colmajor((d, k)) for d, k in zip(q.dims, q.ranks)]
        R.rhosvd_decompose(q.x_host.cuda(), q.dims, q.ranks, p=q.p, q=q.q, seed=q.seed, out=(G, Us))
        np.testing.assert_array_equal(r.G, G.cpu().numpy())
        for a, b in zip(r.Us, Us):
            np.testing.assert_array_equal(a, b.cpu().numpy())


def test_fixed_accuracy_requests_in_the_mix_equal_alone():
    """Fixed-accuracy requests (ranks found on the device by the blocked range
    finder) served next to fixed-rank ones: each one's ranks, core and factors
    are bitwise those of the same call made alone, and meet the tolerance."""
    from oracle import metrics as M
    from paper_2001_07124_gb300 import rhosvd as R
    from paper_2001_07124_gb300.serving import Request, serve
    reqs = []
    specs = [((96, 80, 64), (16, 16, 16), 0.9, 1e-2), ((128, 96, 72), (10, 9, 8), None, 0.0),
             ((64, 64, 64), (20, 20, 20), 0.85, 5e-2), ((80, 72, 40), (8, 7, 6), None, 0.0),
             ((48, 40, 32, 16), (6, 5, 4, 3), None, 1e-2)]
    xs = []
    for i, (dims, ranks, decay, tol) in enumerate(specs):
        x = lowrank_tensor(dims, ranks, 600 + i, noise=1e-4 if decay else 1e-3, decay=decay)
        xs.append(np.asfortranarray(x.astype(np.float32).astype(np.float64)))
        xh = torch.from_numpy(device_layout(x)).pin_memory()
        reqs.append(Request(i, dims, ranks, arrival=0.0, x_host=xh, p=5, q=1, seed=30 + i, tol=tol, block=8,
                            k_max=tuple(min(d, 48) for d in dims) if tol > 0 else None))
    res = serve(reqs, slots=3, budget_bytes=4 * 10 ** 9)
    assert sorted(r.rid for r in res) == list(range(len(reqs)))
    for r in res:
        q = reqs[r.rid]
        if q.tol <= 0:
            continue
        G, U, ranks = R.rhosvd_decompose_tol(q.x_host.cuda(), q.dims, q.tol, block=q.block, k_max=q.k_max,
                                             seed=q.seed)
        assert tuple(ranks) == tuple(r.ranks)
        np.testing.assert_array_equal(r.G, G.contiguous().cpu().numpy().ravel(order="F"))
        for a, b in zip(r.Us, U):
            np.testing.assert_array_equal(a, b.cpu().numpy().ravel(order="F"))
        g = r.G.reshape(r.ranks, order="F").astype(np.float64)
        us = [u.reshape(d, k, order="F").astype(np.float64) for u, d, k in zip(r.Us, q.dims, r.ranks)]
        assert M.rel_error(xs[r.rid], g, us) <= q.tol
