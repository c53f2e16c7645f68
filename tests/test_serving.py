"""The serving form: requests submitted while others run are admitted as
memory frees up, and each result is the same as partitioning the graph
alone (sbp_partition) and as the oracle's full run (Section II-B):
assignment, B and sweep count identical, DL within 1e-12 relative of the
oracle's FP64 value.  Needs a GPU."""
import os
import threading
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
import paper_2305_18663_gb300 as P  # noqa: E402
from synth.dcsbm import batch_specs, dcsbm  # noqa: E402

NT = max(1, min(16, os.cpu_count() or 1))
_ORACLE = {}

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.load()


def _graphs(count, n_hi, seed, with_host=False):
    specs = batch_specs(count, seed=seed, n_lo=300, n_hi=n_hi)
    hg = [dcsbm(**s) for s in specs]
    pg = [P.Graph(g.n, g.src, g.dst) for g in hg]
    return (pg, hg) if with_host else pg


@pytest.mark.parametrize("opts", [dict(), dict(workers=2, mem_fraction=1e-9)])
def test_served_results_equal_alone(opts):
    graphs, host = _graphs(8, 6000, seed=21, with_host=True)
    params = P.Params.default(seed=6)
    alone = [g.partition(params) for g in graphs]
    if "oracle" not in _ORACLE:
        _ORACLE["oracle"] = [O.partition(O.Graph(g.n, g.src, g.dst), O.Params(seed=6), nthreads=NT) for g in host]
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
    for (b, B, dl, ns, ts, ta, td), (pb, pB, pdl, pns), (ob, oB, odl, ons) in zip(outs, alone, _ORACLE["oracle"]):
        assert B == oB and ns == ons and np.array_equal(b, ob)
        assert dl == pytest.approx(odl, rel=1e-12)
        assert B == pB and dl == pdl and ns == pns
        assert np.array_equal(b, pb)
        assert ts <= ta <= td
    assert st.phases_batched + st.phases_per_graph > 0
    if not opts:
        # with the default limits every request's search goes to the
        # persistent kernel once it is down to B <= 1024, merges included
        assert st.merges_batched > 0


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
