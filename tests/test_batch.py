"""The batching form: every graph of a batch ends with exactly the result of
the oracle's full run (Section II-B: merge phases, MCMC phases, golden-ratio
search) and of its own sbp_partition run (assignment, B, sweep count
identical; DL within 1e-12 relative of the oracle's FP64 value, identical to
sbp_partition's), whatever the batch's schedule (workers, batch limit,
admission waves).  Needs a GPU."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
import paper_2305_18663_gb300 as P  # noqa: E402
from synth.dcsbm import batch_specs, dcsbm  # noqa: E402

NT = max(1, min(16, os.cpu_count() or 1))
_ORACLE = {}


def oracle_runs(key, gs, seed):
    """O.partition of every graph (cached per graph set and seed)."""
    if (key, seed) not in _ORACLE:
        _ORACLE[(key, seed)] = [O.partition(O.Graph(g.n, g.src, g.dst), O.Params(seed=seed), nthreads=NT) for g in gs]
    return _ORACLE[(key, seed)]


def assert_matches_oracle(res, ref):
    b, B, dl, ns = res
    ob, oB, odl, ons = ref
    assert B == oB and ns == ons
    assert dl == pytest.approx(odl, rel=1e-12)
    assert np.array_equal(b, ob)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.load()


def _graphs(count, n_hi, seed=3):
    specs = batch_specs(count, seed=seed, n_lo=300, n_hi=n_hi)
    gs = [dcsbm(**s) for s in specs]
    return gs, [P.Graph(g.n, g.src, g.dst) for g in gs]


def _plain(pg, params):
    return pg.partition(params)


@pytest.mark.parametrize("opts", [
    dict(),                                            # defaults
    dict(workers=3, max_B=64, dense_max_B=128),        # more per-graph phases, sparse rows above 128
    dict(workers=2, max_B=1024, mem_fraction=1e-9),    # one graph admitted at a time
    dict(movers_per_warp=1, max_n=100000),             # a warp per mover, every graph batched
    dict(movers_per_warp=4, max_B=256, ctas_per_sm=3), # 8 lanes per mover
])
def test_batch_equals_plain(opts):
    gs, pgs = _graphs(10, 4000)
    params = P.Params.default(seed=4, dense_max_B=opts.get("dense_max_B", 1024))
    out = P.partition_batch(pgs, params, P.BatchOptions.default(**opts))
    ref = oracle_runs("n4000", gs, 4)
    for g, pg, (b, B, dl, ns, ta, td), o in zip(gs, pgs, out, ref):
        assert_matches_oracle((b, B, dl, ns), o)
        pb, pB, pdl, pns = _plain(pg, params)
        assert B == pB and ns == pns
        assert dl == pdl
        assert np.array_equal(b, pb)
        assert 0.0 <= ta <= td


def test_whole_phases_in_the_launch_match_the_oracle():
    # graphs of at most 1024 vertices: every phase of the search, from the
    # first merge at B = N on, runs whole in the persistent launch (start
    # state, merge rounds, sweeps, compaction), including the phases that
    # start from a bracket state the model no longer holds
    gs, pgs = _graphs(12, 1000, seed=21)
    params = P.Params.default(seed=6)
    st = P.BatchStats()
    out = P.partition_batch(pgs, params, P.BatchOptions.default(max_B=1024, max_n=1024), st)
    ref = oracle_runs("n1000", gs, 6)
    for pg, (b, B, dl, ns, ta, td), o in zip(pgs, out, ref):
        assert_matches_oracle((b, B, dl, ns), o)
        pb, pB, pdl, pns = _plain(pg, params)
        assert B == pB and dl == pdl and ns == pns and np.array_equal(b, pb)
    assert st.phases_per_graph == 0
    assert st.merges_batched == st.phases_batched > 0
    assert st.starts_batched > 0


def test_batch_dense_switch_does_not_change_results():
    # the batch's dense/sparse switch is a schedule choice: the same graph
    # partitioned with dense rows up to 4096 or sparse rows above 64 agrees
    gs, pgs = _graphs(4, 2500, seed=9)
    a = P.partition_batch(pgs, P.Params.default(seed=1), P.BatchOptions.default(dense_max_B=4096))
    b = P.partition_batch(pgs, P.Params.default(seed=1), P.BatchOptions.default(max_B=64, dense_max_B=64))
    for x, y in zip(a, b):
        assert x[1] == y[1] and x[2] == y[2] and x[3] == y[3] and np.array_equal(x[0], y[0])


def test_batch_bad_options_raise():
    gs, pgs = _graphs(1, 600)
    with pytest.raises(P.SbpError):
        P.partition_batch(pgs, None, P.BatchOptions.default(max_B=5000))
    with pytest.raises(P.SbpError):
        P.partition_batch(pgs, None, P.BatchOptions.default(workers=0))
    with pytest.raises(P.SbpError):
        P.partition_batch(pgs, None, P.BatchOptions.default(movers_per_warp=3))
    assert P.partition_batch([], None, None) == []


def test_autotuner_returns_valid_options_with_unchanged_results():
    gs, pgs = _graphs(8, 3000, seed=13)
    params = P.Params.default(seed=2)
    best, rate, trials = P.autotune_batch(pgs, params, sample=4)
    assert rate > 0.0 and trials >= 2 + 5  # warm-up, baseline and one run per knob at least
    assert best.movers_per_warp in (1, 2, 4) and 1 <= best.ctas_per_sm <= 4
    assert best.max_B in (128, 256, 512, 1024) and best.dense_max_B >= best.max_B
    out = P.partition_batch(pgs, params, best)
    for pg, (b, B, dl, ns, ta, td) in zip(pgs, out):
        pb, pB, pdl, pns = _plain(pg, params)
        assert B == pB and dl == pdl and ns == pns and np.array_equal(b, pb)
