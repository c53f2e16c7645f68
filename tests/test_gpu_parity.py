"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bar: assignments, proposals and M bit-exact; Delta DL within
1e-9 * max(|Delta DL|, 1) (FP64 on both sides, different summation order);
DL within 1e-12 relative.  A proposal whose log acceptance ratio lies
within 1e-9 * max(|logA|, 1) of ln(u) is a margin case: it is not counted as
a mismatch, and the oracle adopts the GPU's decision for it.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
import paper_2305_18663_gb300 as P  # noqa: E402
from synth.dcsbm import dcsbm, make_config, perturb, random_labels  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-9
NT = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.load()


def close(a, b, tol=TOL):
    return np.abs(a - b) <= tol * np.maximum(np.abs(b), 1.0)


def gpu_decide(model, n, sweep_id, lo=0, hi=None):
    dev = torch.device("cuda")
    s = torch.full((n,), -7, dtype=torch.int32, device=dev)
    flags = torch.full((n,), -7, dtype=torch.int32, device=dev)
    dH = torch.zeros(n, dtype=torch.float64, device=dev)
    logA = torch.zeros(n, dtype=torch.float64, device=dev)
    P.sbp_nodal_decide(model.h, sweep_id, lo, n if hi is None else hi, s=s, flags=flags, dH=dH, logA=logA)
    torch.cuda.synchronize()
    return s.cpu().numpy(), flags.cpu().numpy(), dH.cpu().numpy(), logA.cpu().numpy()


def compare_decisions(od, gd, b, idx):
    """Compare oracle decisions od with GPU trace gd on vertices idx.
    Returns the boolean margin mask over idx."""
    s, flags, dH, logA = (x[idx] for x in gd)
    assert np.array_equal(s, od.s[idx]), "proposals differ"
    assert np.array_equal(flags & 1, od.flags[idx] & 1), "proposed flags differ"
    moved = (s != b[idx]) & ((flags & 1) != 0)
    assert np.all(close(dH[moved], od.dH[idx][moved])), np.max(np.abs(dH[moved] - od.dH[idx][moved]))
    assert np.all(close(logA[moved], od.logA[idx][moved]))
    o_margin = np.abs(od.lnu[idx] - od.logA[idx]) <= TOL * np.maximum(np.abs(od.logA[idx]), 1.0)
    margin = moved & (o_margin | ((flags & 4) != 0))
    agree = (flags & 2) == (od.flags[idx] & 2)
    assert np.all(agree | margin), "accept decisions differ outside the margin band"
    return margin


def check_blockmodel(pm, om):
    assert pm.B == om.B
    keys, cnt = pm.coo()
    okeys, ocnt = om.coo()
    assert np.array_equal(keys, okeys) and np.array_equal(cnt.astype(np.int64), ocnt)
    dout, din = pm.degrees()
    odout, odin = om.degrees()
    assert np.array_equal(dout, odout) and np.array_equal(din, odin)
    assert pm.dl() == pytest.approx(om.dl(), rel=1e-12)


def run_sweeps(g, B, b, sweeps, seed=7, first_sweep=0, dense_max_B=4096):
    G = O.Graph(g.n, g.src, g.dst)
    om = O.Model(G, B, b)
    pg = P.Graph(g.n, g.src, g.dst)
    pm = P.Model(pg, B, b, P.Params.default(seed=seed, dense_max_B=dense_max_B))
    check_blockmodel(pm, om)
    total_margin = 0
    for sw in range(first_sweep, first_sweep + sweeps):
        bcur = om.assignment()
        gd = gpu_decide(pm, g.n, sw)
        od = om.nodal_decide(seed, sw, 3.0, nthreads=NT)
        margin = compare_decisions(od, gd, bcur, np.arange(g.n))
        total_margin += int(margin.sum())
        st = P.sbp_commit(pm.h)
        bg = pm.assignment()
        want = od.b_new.copy()
        want[margin] = bg[margin]
        assert np.array_equal(bg, want)
        assert st.n_accepted == int(((gd[1] & 2) != 0).sum())
        assert st.n_proposed == int(((gd[1] & 1) != 0).sum())
        om.set_b(B, bg)
        check_blockmodel(pm, om)
    return pm, om, total_margin


# ---------------------------------------------------------------------------

def test_philox_device_matches_oracle():
    rng = np.random.default_rng(3)
    for _ in range(20):
        ctr = rng.integers(0, 2**62, 4, dtype=np.uint64)
        key = rng.integers(0, 2**62, 2, dtype=np.uint64)
        got = P.sbp_philox_check(ctr, key, 64)
        for i in range(64):
            c = ctr.copy()
            c[0] = np.uint64(int(c[0]) + i)
            assert np.array_equal(got[i], O.philox4x64(c, key))


def test_fp32_term_within_its_bound():
    # the FP32 x ln x term against f(x+k) - f(x) in extended precision, over
    # small and large counts, k of both signs, the branch boundaries, and
    # counts beyond 2^24
    rng = np.random.default_rng(17)
    xs, ks = [], []
    for hi in (8, 100, 5000, 1 << 20, 1 << 26, (1 << 31) - 2):
        x = rng.integers(0, hi, 20000)
        k = np.where(rng.random(x.size) < 0.5, -rng.integers(0, x + 1), rng.integers(1, 2000, x.size))
        k = np.minimum(k, (1 << 31) - 1 - x)
        xs.append(x)
        ks.append(k)
    e = np.array([0, 1, 2, 3, 4, 10, 100, 1000], np.int64)
    for x0 in e:
        for k0 in (-x0, -(x0 // 2), -(x0 // 2) - 1, 1, 2, x0 // 2, x0):
            if x0 + k0 >= 0 and k0 != 0:
                xs.append(np.array([x0]))
                ks.append(np.array([k0]))
    x = np.concatenate(xs).astype(np.int64)
    k = np.concatenate(ks).astype(np.int64)
    keep = (x + k >= 0) & (k != 0)
    x, k = x[keep], k[keep]
    val, am = P.sbp_dxlogx32_check(x, k)
    xl, yl = x.astype(np.longdouble), (x + k).astype(np.longdouble)
    f = lambda z: np.where(z > 0, z * np.log(np.maximum(z, 1)), 0)  # noqa: E731
    exact = (f(yl) - f(xl)).astype(np.float64)
    err = np.abs(val.astype(np.float64) - exact)
    bound = 28 * 2.0 ** -24 * am.astype(np.float64) * 1.0001 + 1e-30
    assert np.all(err <= bound), (x[err > bound][:5], k[err > bound][:5], (err / bound).max())


@pytest.mark.parametrize("B,dmax", [(1, 4096), (8, 4096), (64, 4096), (1000, 4096), (8, 4), (64, 16), (1000, 16)])
def test_blockmodel_rebuild_matches_oracle(B, dmax):
    g = make_config("plain_1k")
    b = random_labels(g.n, B, seed=B) if B < g.n else np.arange(g.n, dtype=np.int32)
    G = O.Graph(g.n, g.src, g.dst)
    om = O.Model(G, B, b)
    pg = P.Graph(g.n, g.src, g.dst)
    pm = P.Model(pg, B, b, P.Params.default(dense_max_B=dmax))
    check_blockmodel(pm, om)
    assert pm.coo()[1].sum() == g.m


@pytest.mark.parametrize("B", [2, 300, 20000, 70000])
def test_sparse_rebuild_many_chunks_matches_oracle(B):
    # 150k vertices, 3M edges.  B = 2 and 300: counting sort over the B^2
    # cells; B = 20000: radix sort of 32-bit keys (4 passes, every chunk
    # spans several rounds); B = 70000: 64-bit keys (B^2 > 2^32)
    g = make_config("dcsbm_1m", seed=0, scale=0.15)
    b = random_labels(g.n, B, seed=5)
    G = O.Graph(g.n, g.src, g.dst)
    om = O.Model(G, B, b)
    pg = P.Graph(g.n, g.src, g.dst)
    pm = P.Model(pg, B, b, P.Params.default(dense_max_B=1))
    check_blockmodel(pm, om)


@pytest.mark.parametrize("B", [8, 64])
def test_nodal_sweeps_plain_1k(B):
    g = make_config("plain_1k")
    run_sweeps(g, B, random_labels(g.n, B, seed=B), sweeps=10)


@pytest.mark.parametrize("B", [8, 64, 500])
def test_nodal_sweeps_sparse_blockmodel(B):
    # dense_max_B below B: per-row hashed sparse rows and CSR/CSC searches
    g = make_config("plain_1k")
    run_sweeps(g, B, random_labels(g.n, B, seed=B + 1), sweeps=6, dense_max_B=4)


def test_nodal_sweeps_sparse_scaled_dcsbm():
    g = make_config("plain_200k", scale=0.1)
    b = perturb(g.planted, 100, 0.3, seed=0)
    run_sweeps(g, 100, b, sweeps=2, dense_max_B=32)


def test_nodal_sweeps_self_loops_duplicates_isolated():
    rng = np.random.default_rng(11)
    n = 300
    src = rng.integers(0, n - 20, 3000).astype(np.int32)  # last 20 vertices isolated
    dst = rng.integers(0, n - 20, 3000).astype(np.int32)
    src[:200] = dst[:200]  # self-loops
    src[200:400] = src[400:600]  # duplicates
    dst[200:400] = dst[400:600]
    hub = 5  # one high-degree vertex (CTA path) with self-loops
    src = np.concatenate([src, np.full(400, hub, np.int32), np.full(3, hub, np.int32)])
    dst = np.concatenate([dst, rng.integers(0, n - 20, 400).astype(np.int32), np.full(3, hub, np.int32)])

    class Gr:
        pass

    g = Gr()
    g.n, g.src, g.dst, g.m = n, src, dst, src.size
    run_sweeps(g, 12, random_labels(n, 12, seed=1), sweeps=8)


class _G:
    def __init__(self, n, src, dst):
        self.n, self.src, self.dst, self.m = n, src.astype(np.int32), dst.astype(np.int32), src.size


def test_nodal_sweeps_large_B_hubs_cta_path():
    # B = 3000 and hubs above 2048 edges: per-vertex tables beyond 4096
    # slots take the CTA-per-vertex kernel
    rng = np.random.default_rng(21)
    n = 6000
    src = rng.integers(0, n, 40000)
    dst = rng.integers(0, n, 40000)
    for hub, deg in [(7, 2600), (8, 3100), (9, 5000)]:
        src = np.concatenate([src, np.full(deg, hub), rng.integers(0, n, deg // 2), [hub, hub]])
        dst = np.concatenate([dst, rng.integers(0, n, deg), np.full(deg // 2, hub), [hub, hub]])
    g = _G(n, src, dst)
    run_sweeps(g, 3000, random_labels(n, 3000, seed=2), sweeps=3)


def test_nodal_sweeps_hub_table_beyond_shared_memory():
    # B = 9500 and a hub with 18,000 edges: its neighbour table needs 16,384
    # slots (256 KB), more than shared memory holds, so the CTA kernel keeps
    # it in global memory
    rng = np.random.default_rng(23)
    n = 30000
    src = rng.integers(0, n, 60000)
    dst = rng.integers(0, n, 60000)
    hub = 11
    src = np.concatenate([src, np.full(9000, hub), rng.integers(0, n, 9000)])
    dst = np.concatenate([dst, rng.integers(0, n, 9000), np.full(9000, hub)])
    g = _G(n, src, dst)
    run_sweeps(g, 9500, random_labels(n, 9500, seed=4), sweeps=2)


def test_nodal_sweeps_degree_above_65535():
    # a hub with 70,000 edges: 16-bit packed counts no longer fit
    rng = np.random.default_rng(22)
    n = 80000
    src = np.concatenate([np.zeros(70000, np.int64), rng.integers(1, n, 100000)])
    dst = np.concatenate([rng.integers(1, n, 70000), rng.integers(1, n, 100000)])
    g = _G(n, src, dst)
    run_sweeps(g, 16, random_labels(n, 16, seed=3), sweeps=2)


def test_nodal_sweeps_scaled_dcsbm():
    # 50k vertices, 1M edges, 316 planted blocks, 30% reassigned: spans
    # every degree group (one lane per edge, warp, CTA) and ragged tails
    g = make_config("dcsbm_1m", scale=0.05)
    b = perturb(g.planted, 316, 0.3, seed=0)
    _, _, margin = run_sweeps(g, 316, b, sweeps=2)
    assert margin <= 5


def _hub_graph():
    rng = np.random.default_rng(21)
    n = 6000
    src = rng.integers(0, n, 40000)
    dst = rng.integers(0, n, 40000)
    for hub, deg in [(7, 2600), (8, 3100), (9, 5000)]:
        src = np.concatenate([src, np.full(deg, hub), rng.integers(0, n, deg // 2), [hub, hub]])
        dst = np.concatenate([dst, rng.integers(0, n, deg), np.full(deg // 2, hub), [hub, hub]])
    return _G(n, src, dst)


@pytest.mark.parametrize("case", ["dcsbm_dense", "dcsbm_sparse", "hubs_B3000", "hubs_B64"])
def test_fp32_delta_dl_decides_as_exact(case):
    # the precision form (FP32 x ln x terms, exact recheck inside the error
    # band) must take exactly the decisions of the exact evaluation, with no
    # per-vertex trace (a trace forces the exact path)
    if case.startswith("dcsbm"):
        g = make_config("dcsbm_1m", scale=0.05)
        B, b = 316, perturb(g.planted, 316, 0.3, seed=0)
        dmax = 4096 if case.endswith("dense") else 1
    else:
        g = _hub_graph()
        B = 3000 if case == "hubs_B3000" else 64
        b, dmax = random_labels(g.n, B, seed=2), 4096
    pg = P.Graph(g.n, g.src, g.dst)
    fast = P.Model(pg, B, b, P.Params.default(seed=11, dense_max_B=dmax, dl_fp32=1))
    exact = P.Model(pg, B, b, P.Params.default(seed=11, dense_max_B=dmax, dl_fp32=0))
    rechecks = moves = 0
    for sw in range(5):
        sf = fast.sweep(sw)
        se = exact.sweep(sw)
        assert sf.n_accepted == se.n_accepted and sf.n_moves == se.n_moves
        assert np.array_equal(fast.assignment(), exact.assignment())
        assert fast.dl() == exact.dl()
        rechecks += sf.n_recheck
        moves += sf.n_moves
    assert rechecks < moves


@pytest.mark.parametrize("case", ["plain_1k_B8", "hubs_B64", "dcsbm_B316"])
def test_hybrid_sweeps_match_oracle(case):
    # hybrid pass: the h highest-degree vertices one after another against the
    # current state (one CTA, M updated in place), the rest by asynchronous
    # Gibbs against the result; compared vertex by vertex with the oracle
    if case == "plain_1k_B8":
        g, B, h = make_config("plain_1k"), 8, 40
        b = random_labels(g.n, B, seed=3)
    elif case == "hubs_B64":
        g, B, h = _hub_graph(), 64, 30
        b = random_labels(g.n, B, seed=4)
    else:
        g, B, h = make_config("dcsbm_1m", scale=0.02), 316, 200
        b = perturb(g.planted, 316, 0.3, seed=0)
    G = O.Graph(g.n, g.src, g.dst)
    om = O.Model(G, B, b)
    pg = P.Graph(g.n, g.src, g.dst)
    pm = P.Model(pg, B, b, P.Params.default(seed=7, hybrid_h=h))
    for sw in range(4):
        bcur = om.assignment()
        gd = gpu_decide(pm, g.n, sw)
        od = om.hybrid_decide(7, sw, 3.0, h, nthreads=NT)
        margin = compare_decisions(od, gd, bcur, np.arange(g.n))
        assert margin.sum() == 0
        P.sbp_commit(pm.h)
        assert np.array_equal(pm.assignment(), od.b_new)
        om.set_b(B, od.b_new)
        check_blockmodel(pm, om)


def test_shards_then_commit_equal_one_sweep():
    g = make_config("plain_1k")
    b = random_labels(g.n, 16, seed=4)
    pg = P.Graph(g.n, g.src, g.dst)
    full = P.Model(pg, 16, b)
    full.sweep(3)
    shard = P.Model(pg, 16, b)
    for lo, hi in [(0, 100), (100, 777), (777, g.n)]:
        P.sbp_nodal_decide(shard.h, 3, lo, hi)
    P.sbp_commit(shard.h)
    assert np.array_equal(full.assignment(), shard.assignment())
    assert np.array_equal(full.dense(), shard.dense())


@pytest.mark.parametrize("dmax", [4096, 1])
def test_repeated_and_discarded_decisions_before_commit(dmax):
    # a range decided twice (the accepted-move list no longer holds every
    # change once: the apply step scans the assignment instead), and
    # decisions dropped by a rebuild before the next pass
    g = make_config("dcsbm_1m", scale=0.02)
    B = 316
    b = perturb(g.planted, B, 0.3, seed=9)  # few accepted moves: the incremental apply step
    pg = P.Graph(g.n, g.src, g.dst)
    prm = P.Params.default(seed=5, dense_max_B=dmax)
    full = P.Model(pg, B, b, prm)
    full.sweep(2)
    twice = P.Model(pg, B, b, prm)
    P.sbp_nodal_decide(twice.h, 2, 0, g.n)
    P.sbp_nodal_decide(twice.h, 2, 1000, 3000)
    P.sbp_commit(twice.h)
    assert np.array_equal(full.assignment(), twice.assignment())
    assert np.array_equal(full.coo()[0], twice.coo()[0]) and np.array_equal(full.coo()[1], twice.coo()[1])
    dropped = P.Model(pg, B, b, prm)
    P.sbp_nodal_decide(dropped.h, 7, 0, g.n)  # discarded by the rebuild below
    P.sbp_set_assignment(dropped.h, B, b)
    P.sbp_nodal_decide(dropped.h, 2, 0, g.n)
    P.sbp_commit(dropped.h)
    assert np.array_equal(full.assignment(), dropped.assignment())
    assert np.array_equal(full.coo()[1], dropped.coo()[1])
    G = O.Graph(g.n, g.src, g.dst)
    check_blockmodel(dropped, O.Model(G, B, dropped.assignment()))
    for m in (full, twice, dropped):
        m.close()


def test_single_block_and_no_edges():
    g = make_config("plain_1k")
    pg = P.Graph(g.n, g.src, g.dst)
    pm = P.Model(pg, 1, np.zeros(g.n, np.int32))
    st = pm.sweep(0)
    assert st.n_accepted == 0 and st.n_moves == 0 and st.n_proposed == g.n
    G = O.Graph(g.n, g.src, g.dst)
    assert pm.dl() == pytest.approx(O.Model(G, 1, np.zeros(g.n, np.int32)).dl(), rel=1e-13)
    e = np.zeros(0, np.int32)
    pg0 = P.Graph(5, e, e)
    pm0 = P.Model(pg0, 3, np.array([0, 1, 2, 0, 1], np.int32))
    st = pm0.sweep(0)
    assert st.n_proposed == 0 and st.n_accepted == 0
    assert pm0.dl() == pytest.approx(O.Model(O.Graph(5, e, e), 3, np.array([0, 1, 2, 0, 1], np.int32)).dl(), rel=1e-14)


def test_bad_arguments_raise():
    g = make_config("plain_1k")
    pg = P.Graph(g.n, g.src, g.dst)
    with pytest.raises(P.SbpError) as e:
        P.Model(pg, 4, np.full(g.n, 4, np.int32))
    assert e.value.code == -1
    pm = P.Model(pg, 4, np.zeros(g.n, np.int32))
    with pytest.raises(P.SbpError):
        P.sbp_nodal_sweep(pm.h, 0, 10, 5)
    with pytest.raises(P.SbpError):
        P.sbp_merge_blocks(pm.h, 0, 4)
    with pytest.raises(P.SbpError):
        P.Graph(3, np.array([0, 3], np.int32), np.array([1, 2], np.int32))


def test_device_pointers_accepted():
    g = make_config("plain_1k")
    src = torch.from_numpy(g.src).cuda()
    dst = torch.from_numpy(g.dst).cuda()
    pg = P.Graph(g.n, src, dst)
    b = random_labels(g.n, 8, seed=2)
    pm = P.Model(pg, 8, torch.from_numpy(b).cuda())
    out = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    P.sbp_get_assignment(pm.h, out)
    assert np.array_equal(out.cpu().numpy(), b)
    G = O.Graph(g.n, g.src, g.dst)
    check_blockmodel(pm, O.Model(G, 8, b))


# ---------------------------------------------------------------------------
# merge phase

@pytest.mark.parametrize("B,dmax", [(40, 4096), (1000, 4096), (40, 8), (1000, 8)])
def test_merge_proposals_match_oracle(B, dmax):
    g = make_config("plain_1k")
    b = random_labels(g.n, B, seed=5) if B < g.n else np.arange(g.n, dtype=np.int32)
    G = O.Graph(g.n, g.src, g.dst)
    om = O.Model(G, B, b)
    pg = P.Graph(g.n, g.src, g.dst)
    pm = P.Model(pg, B, b, P.Params.default(seed=9, dense_max_B=dmax))
    bs = np.zeros(B, np.int32)
    bd = np.zeros(B, np.float64)
    P.sbp_merge_proposals(pm.h, 4, bs, bd)
    obs, obd = om.merge_proposals(9, 4, 10, nthreads=NT)
    assert np.all(close(bd, obd))
    diff = np.flatnonzero(bs != obs)
    for r in diff:  # only ties on the score grid may differ, and both must be proposals
        props = [om.merge_propose(9, 4, int(r), i) for i in range(10)]
        assert bs[r] in props
        assert O.merge_key(om.merge_delta(int(r), int(bs[r]))) == O.merge_key(obd[r])
    assert diff.size <= max(2, B // 200)


@pytest.mark.parametrize("dmax", [4096, 16])
def test_merge_blocks_matches_oracle_application(dmax):
    g = make_config("plain_1k")
    B = 200
    b = random_labels(g.n, B, seed=6)
    pg = P.Graph(g.n, g.src, g.dst)
    pm = P.Model(pg, B, b, P.Params.default(seed=2, dense_max_B=dmax))
    bs = np.zeros(B, np.int32)
    bd = np.zeros(B, np.float64)
    P.sbp_merge_proposals(pm.h, 8, bs, bd)
    n_merges = 60
    done, mp, Bn = O.merge_apply(B, bs, bd, n_merges)
    assert done == n_merges
    Bg, rounds = P.sbp_merge_blocks(pm.h, 8, n_merges)
    assert rounds == 1 and Bg == Bn == B - n_merges
    assert np.array_equal(pm.assignment(), mp[b])
    G = O.Graph(g.n, g.src, g.dst)
    check_blockmodel(pm, O.Model(G, Bn, mp[b]))


@pytest.mark.parametrize("dmax", [4096, 2])
def test_merge_blocks_second_round_matches_oracle(dmax):
    # 6 blocks in 3 pairs with no edge between pairs: round 0 can make only
    # 3 links, so 4 merges need a second proposal round on the merged model
    from test_oracle_driver_pins import _paired_blocks_graph

    n, src, dst, b = _paired_blocks_graph()
    om = O.Model(O.Graph(n, src, dst), 6, b)
    oB, orounds = om.merge_phase(O.Params(seed=5), 20, 4)
    assert (oB, orounds) == (2, 2)
    pm = P.Model(P.Graph(n, src, dst), 6, b, P.Params.default(seed=5, dense_max_B=dmax))
    Bg, rounds = P.sbp_merge_blocks(pm.h, 20, 4)
    assert (Bg, rounds) == (oB, orounds)
    assert np.array_equal(pm.assignment(), om.assignment())
    check_blockmodel(pm, om)


def test_compact_drops_empty_blocks():
    g = make_config("plain_1k")
    b = (random_labels(g.n, 10, seed=1) * 3).astype(np.int32)  # labels 0,3,...,27 of 30
    pg = P.Graph(g.n, g.src, g.dst)
    pm = P.Model(pg, 30, b)
    assert P.sbp_compact(pm.h) == 10
    Bo, bo = O.compact(30, b)
    assert Bo == 10 and np.array_equal(pm.assignment(), bo)


@pytest.mark.parametrize("dmax", [4096, 64])
def test_partition_plain_1k_matches_oracle(dmax):
    # dmax = 64: the run starts sparse at B = N and turns dense below 64
    g = make_config("plain_1k")
    G = O.Graph(g.n, g.src, g.dst)
    ob, oB, odl, ons = O.partition(G, O.Params(), nthreads=NT)
    pg = P.Graph(g.n, g.src, g.dst)
    b, B, dl, ns = pg.partition(P.Params.default(dense_max_B=dmax))
    assert B == oB == 8
    assert dl == pytest.approx(odl, rel=1e-12)
    assert np.array_equal(b, ob)
    assert ns == ons


@pytest.mark.slow
def test_partition_sparse_start_dcsbm_5k_matches_oracle():
    # 5,000 vertices / 100,000 edges with the 2:1 weak structure: the run
    # starts sparse at B = N = 5000, crosses to dense at B <= 256
    g = make_config("plain_200k", scale=0.025)
    G = O.Graph(g.n, g.src, g.dst)
    ob, oB, odl, ons = O.partition(G, O.Params(), nthreads=NT)
    pg = P.Graph(g.n, g.src, g.dst)
    b, B, dl, ns = pg.partition(P.Params.default(dense_max_B=256))
    assert B == oB
    assert dl == pytest.approx(odl, rel=1e-12)
    assert np.array_equal(b, ob)
    assert ns == ons


@pytest.mark.slow
def test_partition_plain_200k_matches_oracle():
    # the full run (golden-ratio search from B = N = 200,000, sparse rows
    # above 4096 blocks) of the 200k-vertex / 4M-edge configuration: the
    # same B, assignment, sweep count and DL as the oracle's run
    g = make_config("plain_200k")
    G = O.Graph(g.n, g.src, g.dst)
    ob, oB, odl, ons = O.partition(G, O.Params(), nthreads=NT)
    pg = P.Graph(g.n, g.src, g.dst)
    b, B, dl, ns = pg.partition(P.Params.default())
    assert B == oB
    assert ns == ons
    assert dl == pytest.approx(odl, rel=1e-12)
    assert np.array_equal(b, ob)


@pytest.mark.parametrize("dmax", [4096, 1])
def test_incremental_commit_equals_full_rebuild(dmax):
    # the apply step updates the counts (dense M, or the cell counts of the
    # sparse rows' counting rebuild) from the moved vertices' rows when few
    # moved; recounting from all edges must give the same M and DL
    g = make_config("dcsbm_1m", scale=0.05)
    b = perturb(g.planted, 316, 0.3, seed=0)
    pg = P.Graph(g.n, g.src, g.dst)
    inc = P.Model(pg, 316, b, P.Params.default(seed=5, dense_max_B=dmax))
    full = P.Model(pg, 316, b, P.Params.default(seed=5, dense_max_B=dmax, full_rebuild=1))
    G = O.Graph(g.n, g.src, g.dst)
    om = O.Model(G, 316, b)
    for sw in range(8):
        si = inc.sweep(sw)
        sf = full.sweep(sw)
        assert si.n_accepted == sf.n_accepted
        assert np.array_equal(inc.assignment(), full.assignment())
        ki, ci = inc.coo()
        kf, cf = full.coo()
        assert np.array_equal(ki, kf) and np.array_equal(ci, cf)
        assert inc.dl() == full.dl()
    om.set_b(316, inc.assignment())
    check_blockmodel(inc, om)


# ---------------------------------------------------------------------------
# the full-size workload in the configuration the benchmark times: 1M
# vertices, 20M edges, B = 316, FP32 Delta DL terms with the exact recheck,
# three warm-up sweeps, then every vertex of one sweep against the oracle

@pytest.fixture(scope="module")
def full_size():
    g = make_config("dcsbm_1m", seed=0)
    b0 = perturb(g.planted, 316, 0.3, seed=0)
    return g, b0, P.Graph(g.n, g.src, g.dst), O.Graph(g.n, g.src, g.dst)


@pytest.mark.parametrize("m_form", ["sparse", "dense"])
def test_full_size_sweep_in_benchmark_configuration(full_size, m_form):
    g, b0, pg, G = full_size
    B, seed = 316, 0
    params = P.Params.default(seed=seed, dense_max_B=1 if m_form == "sparse" else 4096, dl_fp32=1)
    pm = P.Model(pg, B, b0, params, torch.cuda.current_stream())
    for k in range(3):
        P.sbp_nodal_decide(pm.h, k, 0, g.n)
        P.sbp_commit(pm.h, stats=False)
    bcur = pm.assignment()
    om = O.Model(G, B, bcur)
    check_blockmodel(pm, om)
    gd = gpu_decide(pm, g.n, 3)
    od = om.nodal_decide(seed, 3, 3.0, nthreads=NT)
    margin = compare_decisions(od, gd, bcur, np.arange(g.n))
    moved = int(((gd[0] != bcur) & ((gd[1] & 1) != 0)).sum())
    assert moved > 100_000  # the sweep exercises every degree group
    st = P.sbp_commit(pm.h)
    bg = pm.assignment()
    want = od.b_new.copy()
    want[margin] = bg[margin]
    assert np.array_equal(bg, want)
    assert st.n_accepted == int(((gd[1] & 2) != 0).sum())
    om.set_b(B, bg)
    check_blockmodel(pm, om)
    pm.close()


# ---------------------------------------------------------------------------
# the timed kernels themselves against the oracle: no per-vertex trace (a
# trace sends every mover to the exact evaluation), FP32 terms with the
# exact recheck, sweeps 0..4 from the perturbed start (the heavy-move sweeps
# first), b bit for bit after every commit, then M, degrees and DL

def untraced_sweeps_vs_oracle(g, B, b0, pg, G, m_form, sweeps, seed=0, min_moves=0):
    dmax = 1 if m_form == "sparse" else 4096
    params = P.Params.default(seed=seed, dense_max_B=dmax, dl_fp32=1)
    pm = P.Model(pg, B, b0, params, torch.cuda.current_stream())
    om = O.Model(G, B, b0)
    total_margin = 0
    moves = []
    for sw in range(sweeps):
        bcur = om.assignment()
        P.sbp_nodal_decide(pm.h, sw, 0, g.n)  # the launch sequence bench.py times
        st = P.sbp_commit(pm.h)
        od = om.nodal_decide(seed, sw, 3.0, nthreads=NT)
        # margin cases, by the oracle's own draw and log acceptance ratio
        mv = (od.s != bcur) & ((od.flags & 1) != 0)
        margin = mv & (np.abs(od.lnu - od.logA) <= TOL * np.maximum(np.abs(od.logA), 1.0))
        bg = pm.assignment()
        want = od.b_new.copy()
        want[margin] = bg[margin]
        bad = np.flatnonzero(bg != want)
        assert bad.size == 0, f"sweep {sw}: {bad.size} labels differ from the oracle, first {bad[:5]}"
        assert st.n_moves == int(mv.sum()), "movers differ"
        acc_g = int((bg != bcur).sum())
        assert acc_g == st.n_accepted
        assert abs(st.n_accepted - od.accepted) <= int(margin.sum())
        om.set_b(B, bg)
        check_blockmodel(pm, om)
        total_margin += int(margin.sum())
        moves.append(int(mv.sum()))
    pm.close()
    assert max(moves) >= min_moves
    return total_margin, moves


@pytest.mark.parametrize("m_form", ["sparse", "dense"])
def test_untraced_fp32_sweeps_full_size_match_oracle(full_size, m_form):
    # 1M vertices, 20M edges, B = 316: E >= 2^22, so the decision pass forks
    # its degree groups onto three streams, as in the timed run
    g, b0, pg, G = full_size
    margin, moves = untraced_sweeps_vs_oracle(g, 316, b0, pg, G, m_form, sweeps=5, min_moves=400_000)
    assert margin <= 10


@pytest.mark.parametrize("m_form", ["sparse", "dense"])
def test_untraced_fp32_sweeps_just_above_fork_size_match_oracle(m_form):
    # 220k vertices, about 4.4M edges: just above the 2^22-edge size at which
    # the degree groups run on three streams
    g = make_config("dcsbm_1m", seed=0, scale=0.22)
    assert g.m >= 1 << 22
    b0 = perturb(g.planted, 316, 0.3, seed=0)
    margin, _ = untraced_sweeps_vs_oracle(g, 316, b0, P.Graph(g.n, g.src, g.dst), O.Graph(g.n, g.src, g.dst),
                                          m_form, sweeps=4, min_moves=50_000)
    assert margin <= 5


@pytest.mark.parametrize("m_form", ["sparse", "dense"])
def test_untraced_fp32_sweeps_below_fork_size_match_oracle(m_form):
    # 50k vertices, 1M edges: one stream, every degree group and ragged tails
    g = make_config("dcsbm_1m", seed=0, scale=0.05)
    assert g.m < 1 << 22
    b0 = perturb(g.planted, 316, 0.3, seed=0)
    untraced_sweeps_vs_oracle(g, 316, b0, P.Graph(g.n, g.src, g.dst), O.Graph(g.n, g.src, g.dst), m_form,
                              sweeps=5, min_moves=10_000)


@pytest.mark.parametrize("dmax", [4096, 1])
def test_set_assignment_of_a_nearby_state_equals_a_rebuild(dmax):
    # labels set with the model's block count are applied like a pass's
    # moves (incremental counts for a few changes, a recount for many); the
    # result must be the model built from those labels from scratch, and the
    # block-labelled rows must follow (later sweeps agree)
    g = make_config("dcsbm_1m", seed=0, scale=0.05)
    B = 316
    b0 = perturb(g.planted, B, 0.3, seed=0)
    pg = P.Graph(g.n, g.src, g.dst)
    prm = P.Params.default(seed=5, dense_max_B=dmax)
    pm = P.Model(pg, B, b0, prm)
    for sw in range(2):
        pm.sweep(sw)
    rng = np.random.default_rng(1)
    cur = pm.assignment()
    G = O.Graph(g.n, g.src, g.dst)
    for step, frac in enumerate((0.001, 0.02, 0.6)):
        x = cur.copy()
        idx = rng.choice(g.n, int(frac * g.n), replace=False)
        x[idx] = rng.integers(0, B, idx.size).astype(np.int32)
        if step == 1:
            P.sbp_set_assignment(pm.h, B, torch.from_numpy(x).cuda())  # device input
        else:
            P.sbp_set_assignment(pm.h, B, x)
        fresh = P.Model(pg, B, x, prm)
        assert np.array_equal(pm.assignment(), x)
        k1, c1 = pm.coo()
        k2, c2 = fresh.coo()
        assert np.array_equal(k1, k2) and np.array_equal(c1, c2)
        assert np.array_equal(pm.degrees()[0], fresh.degrees()[0]) and np.array_equal(pm.degrees()[1], fresh.degrees()[1])
        assert pm.dl() == fresh.dl()
        if step == 0:
            check_blockmodel(pm, O.Model(G, B, x))
        for sw in (10 + 2 * step, 11 + 2 * step):
            pm.sweep(sw)
            fresh.sweep(sw)
            assert np.array_equal(pm.assignment(), fresh.assignment())
            assert np.array_equal(pm.coo()[1], fresh.coo()[1]) and pm.dl() == fresh.dl()
        fresh.close()
        cur = pm.assignment()
    # a label out of range is refused and leaves the model as it was
    bad = cur.copy()
    bad[7] = B
    dl = pm.dl()
    with pytest.raises(P.SbpError):
        P.sbp_set_assignment(pm.h, B, bad)
    assert np.array_equal(pm.assignment(), cur) and pm.dl() == dl
    check_blockmodel(pm, O.Model(G, B, cur))
    pm.close()


def _loops_dups_isolated_graph():
    # self-loops, duplicate edges, 20 isolated vertices and a hub of ~400
    # edges (the group above 128 edges), as in the traced test above
    rng = np.random.default_rng(11)
    n = 300
    src = rng.integers(0, n - 20, 3000).astype(np.int32)
    dst = rng.integers(0, n - 20, 3000).astype(np.int32)
    src[:200] = dst[:200]
    src[200:400] = src[400:600]
    dst[200:400] = dst[400:600]
    hub = 5
    src = np.concatenate([src, np.full(400, hub, np.int32), np.full(3, hub, np.int32)])
    dst = np.concatenate([dst, rng.integers(0, n - 20, 400).astype(np.int32), np.full(3, hub, np.int32)])
    return _G(n, src, dst)


@pytest.mark.parametrize("m_form", ["dense", "sparse"])
def test_untraced_sweeps_self_loops_duplicates_isolated(m_form):
    # the kernels that draw their own proposals (full-range pass, no trace)
    # on self-loops, duplicates, isolated vertices and a hub, against the
    # oracle sweep by sweep
    g = _loops_dups_isolated_graph()
    untraced_sweeps_vs_oracle(g, 12, random_labels(g.n, 12, seed=1), P.Graph(g.n, g.src, g.dst),
                              O.Graph(g.n, g.src, g.dst), m_form, sweeps=8, seed=3, min_moves=50)


@pytest.mark.parametrize("case", ["hubs_B3000", "hub_table_global_B9500"])
def test_untraced_sweeps_large_B_table_kernels(case):
    # B above the direct-mapped limit: k_propose hands the movers to the
    # hash-table kernels (k_eval_warp, and k_eval_cta for the hubs, its
    # table in global memory at B = 9500), FP32 terms without a trace,
    # against the oracle sweep by sweep
    if case == "hubs_B3000":
        g, B = _hub_graph(), 3000
    else:
        rng = np.random.default_rng(23)
        n = 30000
        src = rng.integers(0, n, 60000)
        dst = rng.integers(0, n, 60000)
        hub = 11
        src = np.concatenate([src, np.full(9000, hub), rng.integers(0, n, 9000)])
        dst = np.concatenate([dst, rng.integers(0, n, 9000), np.full(9000, hub)])
        g, B = _G(n, src, dst), 9500
    untraced_sweeps_vs_oracle(g, B, random_labels(g.n, B, seed=2), P.Graph(g.n, g.src, g.dst),
                              O.Graph(g.n, g.src, g.dst), "dense", sweeps=3, seed=4, min_moves=100)
