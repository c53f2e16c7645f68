"""The serving form: requests submitted while others run are admitted as
memory frees up, and each result is the same as partitioning the graph
alone (sbp_partition).  Needs a GPU."""
import threading
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2305_18663_gb300 as P  # noqa: E402
from synth.dcsbm import batch_specs, dcsbm  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.load()


def _graphs(count, n_hi, seed):
    specs = batch_specs(count, seed=seed, n_lo=300, n_hi=n_hi)
    return [P.Graph(s["n"], *(lambda g: (g.src, g.dst))(dcsbm(**s))) for s in specs]


@pytest.mark.parametrize("opts", [dict(), dict(workers=2, mem_fraction=1e-9)])
def test_served_results_equal_alone(opts):
    graphs = _graphs(8, 6000, seed=21)
    params = P.Params.default(seed=6)
    alone = [g.partition(params) for g in graphs]
    srv = P.Server(params, P.BatchOptions.default(**opts))
    rids = {}

    def feed():
        # staggered arrivals: later requests come in while earlier ones run
        for i, g in enumerate(graphs):
            rids[i] = srv.submit(g)
            time.sleep(0.003 * (i % 3))

    t = threading.Thread(target=feed)
    t.start()
    t.join()
    outs = [srv.wait(rids[i]) for i in range(len(graphs))]
    st = srv.stats()
    srv.close()
    for (b, B, dl, ns, ts, ta, td), (pb, pB, pdl, pns) in zip(outs, alone):
        assert B == pB and dl == pdl and ns == pns
        assert np.array_equal(b, pb)
        assert ts <= ta <= td
    assert st.phases_batched + st.phases_per_graph > 0


def test_server_poll_and_order():
    graphs = _graphs(3, 2000, seed=5)
    srv = P.Server(P.Params.default(seed=1), P.BatchOptions.default(workers=1, mem_fraction=1e-9))
    rids = [srv.submit(g) for g in graphs]
    res = [srv.wait(r) for r in rids]
    assert all(srv.done(r) for r in rids)
    # one at a time: admissions follow submission order
    assert res[0][5] <= res[1][5] <= res[2][5]
    srv.close()
    s2 = P.sbp_server_create()
    with pytest.raises(P.SbpError):
        P.sbp_server_poll(s2, 99)
    P.sbp_server_destroy(s2)
