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
