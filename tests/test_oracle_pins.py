"""Pins for the CPU oracle: each test checks the oracle against something
other than itself -- numpy's independent Philox, a hand-derived worked
example, closed forms, brute-force recomputation of Eq. 1-2 on tiny graphs,
exact enumeration of the proposal mechanism, chi-square tests of the
sampled proposals, networkx connected components and a unimodal search.
"""
import math
import os

import networkx as nx
import numpy as np
import pytest

import oracle as O
from synth.dcsbm import dcsbm, make_config, random_labels

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# brute force from the printed equations (Eq. 1 and Eq. 2), numpy only

def brute_M(src, dst, b, B):
    M = np.zeros((B, B), np.int64)
    np.add.at(M, (b[src], b[dst]), 1)
    return M


def brute_L(M):
    """Eq. 1 as printed: sum_ij M_ij log(M_ij / (dout_i din_j))."""
    dout, din = M.sum(1), M.sum(0)
    i, j = np.nonzero(M)
    return float(np.sum(M[i, j] * np.log(M[i, j] / (dout[i] * din[j].astype(np.float64)))))


def brute_DL(M, E, V):
    C = M.shape[0]
    x = C * C / E
    h = (1 + x) * math.log(1 + x) - x * math.log(x)
    return E * h + V * math.log(C) - brute_L(M)


def tiny_graph(rng, n, m, self_loops=True):
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    if not self_loops:
        keep = src != dst
        src, dst = src[keep], dst[keep]
    return src, dst


# --------------------------------------------------------------------------
# P2: Philox4x64-10 against numpy's implementation

def test_philox_matches_numpy():
    rng = np.random.default_rng(1)
    cases = [([0, 0, 0, 0], [0, 0]), ([1, 2, 3, 4], [5, 6])]
    for _ in range(200):
        cases.append((rng.integers(0, 2**63, 4, dtype=np.uint64).tolist(), rng.integers(0, 2**63, 2, dtype=np.uint64).tolist()))
    for ctr, key in cases:
        # numpy's Philox increments its 256-bit counter before each block
        c = sum(int(x) << (64 * i) for i, x in enumerate(ctr))
        c = (c - 1) % (1 << 256)
        prev = [(c >> (64 * i)) & (2**64 - 1) for i in range(4)]
        ref = np.random.Philox(counter=prev, key=key).random_raw(4)
        got = O.philox4x64(ctr, key)
        assert np.array_equal(ref, got), (ctr, key)


# --------------------------------------------------------------------------
# P1: worked example, closed forms, brute force

def _golden():
    d = {}
    with open(os.path.join(GOLDEN, "worked_example_4v.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(":", 1)
            d[k.strip()] = v.strip()
    return d


def _ev(expr):
    return eval(expr, {"__builtins__": {}}, {"log": math.log})


def test_worked_example():
    d = _golden()
    src, dst = zip(*[tuple(map(int, e.split(">"))) for e in d["edges"].split()])
    g = O.Graph(int(d["n"]), np.array(src), np.array(dst))
    B = int(d["B"])
    m = O.Model(g, B, np.array(d["b"].split(), np.int32))
    assert m.dense().ravel().tolist() == list(map(int, d["M"].split()))
    dout, din = m.degrees()
    assert dout.tolist() == list(map(int, d["dout"].split()))
    assert din.tolist() == list(map(int, d["din"].split()))
    assert m.L() == pytest.approx(_ev(d["L"]), rel=1e-14)
    assert m.dl() == pytest.approx(_ev(d["DL"]), rel=1e-14)
    dH, pf, pb = m.move_delta(int(d["move_v"]), int(d["move_s"]))
    assert dH == pytest.approx(_ev(d["dH"]), rel=1e-13)
    assert pf == pytest.approx(_ev(d["pf"]), rel=1e-14)
    assert pb == pytest.approx(_ev(d["pb"]), rel=1e-14)


def test_dl_null_closed_form():
    # Section V-C: DL_null is the description length with one community.
    # With C = 1: M_00 = E, dout = din = E, L = -E ln E,
    # DL_null = E h(1/E) + E ln E.
    g = make_config("plain_1k")
    G = O.Graph(g.n, g.src, g.dst)
    m = O.Model(G, 1, np.zeros(g.n, np.int32))
    E = g.m
    x = 1.0 / E
    h = (1 + x) * math.log1p(x) - x * math.log(x)
    assert m.L() == pytest.approx(-E * math.log(E), rel=1e-14)
    assert m.dl() == pytest.approx(E * h + E * math.log(E), rel=1e-14)


@pytest.mark.parametrize("seed", range(6))
def test_blockmodel_and_dl_brute(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 60))
    src, dst = tiny_graph(rng, n, int(rng.integers(n, 6 * n)))
    B = int(rng.integers(1, 9))
    b = rng.integers(0, B, n).astype(np.int32)
    g = O.Graph(n, src, dst)
    m = O.Model(g, B, b)
    M = brute_M(src, dst, b, B)
    assert np.array_equal(m.dense(), M)
    dout, din = m.degrees()
    assert np.array_equal(dout, M.sum(1)) and np.array_equal(din, M.sum(0))
    assert M.sum() == src.size
    assert m.L() == pytest.approx(brute_L(M), rel=1e-12, abs=1e-9)
    assert m.dl() == pytest.approx(brute_DL(M, src.size, n), rel=1e-12)


def test_labels_out_of_range_rejected():
    g = O.Graph(3, np.array([0, 1]), np.array([1, 2]))
    with pytest.raises(ValueError):
        O.Model(g, 2, np.array([0, 1, 2], np.int32))
    with pytest.raises(ValueError):
        O.Graph(3, np.array([0, 3]), np.array([1, 2]))


# --------------------------------------------------------------------------
# P4: incremental Delta DL of a nodal move against full recomputation

@pytest.mark.parametrize("seed", range(8))
def test_move_delta_brute(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(3, 13))
    src, dst = tiny_graph(rng, n, int(rng.integers(n, 4 * n)), self_loops=True)
    B = int(rng.integers(2, 6))
    b = rng.integers(0, B, n).astype(np.int32)
    g = O.Graph(n, src, dst)
    m = O.Model(g, B, b)
    E = src.size
    base = brute_DL(brute_M(src, dst, b, B), E, n)
    for v in range(n):
        for s in range(B):
            if s == b[v]:
                continue
            b2 = b.copy()
            b2[v] = s
            want = brute_DL(brute_M(src, dst, b2, B), E, n) - base
            dH, _, _ = m.move_delta(v, s)
            assert dH == pytest.approx(want, rel=1e-10, abs=1e-10), (v, s)


# --------------------------------------------------------------------------
# P3 + P5: the Hastings weights equal the exact proposal probabilities of
# the sampling mechanism, enumerated over every draw outcome.

def _walk(weights, t):
    return int(np.searchsorted(np.cumsum(weights), t, side="right"))


def proposal_probs(n, src, dst, b, B, v):
    M = brute_M(src, dst, b, B)
    dout, din = M.sum(1), M.sum(0)
    nbrs = sorted(dst[src == v].tolist()) + sorted(src[dst == v].tolist())
    P = np.zeros(B)
    for w in nbrs:
        u = b[w]
        du = int(dout[u] + din[u])
        for y in range(du + B):
            if y < B:
                s = y
            elif y - B < dout[u]:
                s = _walk(M[u, :], y - B)
            else:
                s = _walk(M[:, u], y - B - dout[u])
            P[s] += 1.0 / (len(nbrs) * (du + B))
    return P, len(nbrs)


@pytest.mark.parametrize("seed", range(6))
def test_hastings_equals_enumerated_proposal(seed):
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(3, 10))
    src, dst = tiny_graph(rng, n, int(rng.integers(n, 4 * n)), self_loops=True)
    B = int(rng.integers(2, 5))
    b = rng.integers(0, B, n).astype(np.int32)
    g = O.Graph(n, src, dst)
    m = O.Model(g, B, b)
    for v in range(n):
        P, k = proposal_probs(n, src, dst, b, B, v)
        if k == 0:
            continue
        assert P.sum() == pytest.approx(1.0, rel=1e-12)
        r = int(b[v])
        for s in range(B):
            if s == r:
                continue
            _, pf, pb = m.move_delta(v, s)
            assert pf / k == pytest.approx(P[s], rel=1e-12)
            b2 = b.copy()
            b2[v] = s
            P2, _ = proposal_probs(n, src, dst, b2, B, v)
            assert pb / k == pytest.approx(P2[r], rel=1e-12)


def _chi2_ok(counts, probs, min_expected=5.0):
    tot = counts.sum()
    exp = probs * tot
    keep = exp >= min_expected
    assert counts[~keep].sum() <= max(10, 0.01 * tot)
    stat = float(np.sum((counts[keep] - exp[keep]) ** 2 / exp[keep]))
    dof = int(keep.sum()) - 1
    # p < 1e-5 rejects: Wilson-Hilferty approximation of the chi-square tail
    z = ((stat / dof) ** (1 / 3) - (1 - 2 / (9 * dof))) / math.sqrt(2 / (9 * dof))
    return z < 4.3, (stat, dof, z)


def test_nodal_proposal_distribution_chi2():
    rng = np.random.default_rng(7)
    n, B = 10, 4
    src, dst = tiny_graph(rng, n, 35, self_loops=True)
    b = rng.integers(0, B, n).astype(np.int32)
    g = O.Graph(n, src, dst)
    m = O.Model(g, B, b)
    draws = 20000
    counts = np.zeros((n, B))
    for sw in range(draws):
        d = m.nodal_decide(seed=11, sweep_id=sw, beta=3.0)
        counts[np.arange(n), d.s] += 1
    for v in range(n):
        P, k = proposal_probs(n, src, dst, b, B, v)
        if k == 0:
            continue
        ok, info = _chi2_ok(counts[v], P)
        assert ok, (v, info)


# --------------------------------------------------------------------------
# P6: sweep semantics

def test_sweep_shard_and_thread_invariance():
    g = make_config("plain_1k")
    G = O.Graph(g.n, g.src, g.dst)
    b = random_labels(g.n, 16, seed=3)
    m = O.Model(G, 16, b)
    full = m.nodal_decide(5, 9, 3.0, nthreads=1)
    par = m.nodal_decide(5, 9, 3.0, nthreads=4)
    assert np.array_equal(full.b_new, par.b_new)
    bn = b.copy()
    for lo, hi in [(0, 137), (137, 600), (600, g.n)]:
        part = m.nodal_decide(5, 9, 3.0, lo, hi)
        bn[lo:hi] = part.b_new[lo:hi]
        assert np.array_equal(part.b_new[:lo], b[:lo]) and np.array_equal(part.b_new[hi:], b[hi:])
    assert np.array_equal(bn, full.b_new)
    # decisions and flags are consistent
    acc = (full.flags & 2) != 0
    assert np.array_equal(full.b_new[acc], full.s[acc])
    assert np.all(full.s[acc] != b[acc])
    assert full.accepted == int(acc.sum())
    # rebuild invariants
    m.set_b(16, full.b_new)
    M = m.dense()
    dout, din = m.degrees()
    assert M.sum() == g.m and np.array_equal(M.sum(1), dout) and np.array_equal(M.sum(0), din)
    assert np.array_equal(M, brute_M(g.src, g.dst, full.b_new, 16))


def test_greedy_single_vertex_step():
    # beta large and one eligible vertex: the sweep is one greedy
    # Metropolis step whose Delta DL matches full recomputation.
    rng = np.random.default_rng(5)
    n, B = 12, 3
    src, dst = tiny_graph(rng, n, 40, self_loops=False)
    b = rng.integers(0, B, n).astype(np.int32)
    g = O.Graph(n, src, dst)
    m = O.Model(g, B, b)
    base = brute_DL(brute_M(src, dst, b, B), src.size, n)
    seen = 0
    for sw in range(200):
        for v in range(n):
            d = m.nodal_decide(1, sw, 1e6, v, v + 1)
            if d.flags[v] & 1 and d.s[v] != b[v]:
                b2 = b.copy()
                b2[v] = d.s[v]
                want = brute_DL(brute_M(src, dst, b2, B), src.size, n) - base
                assert d.dH[v] == pytest.approx(want, rel=1e-10, abs=1e-10)
                assert bool(d.flags[v] & 2) == (want < 0 or d.logA[v] >= 0)
                seen += 1
    assert seen > 100


def test_isolated_vertex_never_proposes():
    g = O.Graph(4, np.array([0, 1]), np.array([1, 0]))
    m = O.Model(g, 2, np.array([0, 1, 0, 1], np.int32))
    for sw in range(50):
        d = m.nodal_decide(0, sw, 3.0)
        assert d.flags[2] == 0 and d.flags[3] == 0
        assert d.b_new[2] == 0 and d.b_new[3] == 1


# --------------------------------------------------------------------------
# P7: merge proposals and merge Delta DL

@pytest.mark.parametrize("seed", range(6))
def test_merge_delta_brute(seed):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(4, 14))
    src, dst = tiny_graph(rng, n, int(rng.integers(n, 5 * n)), self_loops=True)
    B = int(rng.integers(2, 7))
    b = rng.integers(0, B, n).astype(np.int32)
    g = O.Graph(n, src, dst)
    m = O.Model(g, B, b)
    L0 = brute_L(brute_M(src, dst, b, B))
    for r in range(B):
        for s in range(B):
            if r == s:
                continue
            b2 = np.where(b == r, s, b).astype(np.int32)
            want = -(brute_L(brute_M(src, dst, b2, B)) - L0)
            assert m.merge_delta(r, s) == pytest.approx(want, rel=1e-10, abs=1e-10), (r, s)


def merge_proposal_probs(src, dst, b, B, r):
    M = brute_M(src, dst, b, B)
    dout, din = M.sum(1), M.sum(0)
    P = np.zeros(B)
    dr = int(dout[r] + din[r])
    if dr == 0:
        P[:] = 1.0 / (B - 1)
        P[r] = 0
        return P
    for t in range(dr):
        u = _walk(M[r, :], t) if t < dout[r] else _walk(M[:, r], t - dout[r])
        rw = M[u, :].copy()
        rw[r] = 0
        cw = M[:, u].copy()
        cw[r] = 0
        W = (B - 1) + rw.sum() + cw.sum()
        for y in range(W):
            if y < B - 1:
                s = y + (y >= r)
            elif y - (B - 1) < rw.sum():
                s = _walk(rw, y - (B - 1))
            else:
                s = _walk(cw, y - (B - 1) - rw.sum())
            P[s] += 1.0 / (dr * W)
    return P


def test_merge_proposal_distribution():
    rng = np.random.default_rng(9)
    n, B = 14, 5
    src, dst = tiny_graph(rng, n, 40, self_loops=True)
    b = rng.integers(0, B, n).astype(np.int32)
    g = O.Graph(n, src, dst)
    m = O.Model(g, B, b)
    M = brute_M(src, dst, b, B)
    d = M.sum(1) + M.sum(0)
    for r in range(B):
        P = merge_proposal_probs(src, dst, b, B, r)
        assert P[r] == 0 and P.sum() == pytest.approx(1.0)
        # closed form: sum_u (M[r][u]+M[u][r])/d_r * (1+M[u][s]+M[s][u])/W_u
        if d[r] > 0:
            Q = np.zeros(B)
            for u in range(B):
                wu = (M[r, u] + M[u, r]) / d[r]
                if wu == 0:
                    continue
                W = (B - 1) + d[u] - M[u, r] - M[r, u]
                for s in range(B):
                    if s != r:
                        Q[s] += wu * (1 + M[u, s] + M[s, u]) / W
            assert np.allclose(P, Q, rtol=1e-12)
        counts = np.zeros(B)
        for rid in range(6000):
            counts[m.merge_propose(4, rid, r, rid % 10)] += 1
        ok, info = _chi2_ok(counts, P)
        assert ok, (r, info)


def test_merge_best_is_min_over_proposals():
    g = make_config("plain_1k")
    G = O.Graph(g.n, g.src, g.dst)
    b = random_labels(g.n, 40, seed=2)
    m = O.Model(G, 40, b)
    bs, bd = m.merge_proposals(3, 17, 10)
    for r in range(40):
        props = [m.merge_propose(3, 17, r, i) for i in range(10)]
        vals = [m.merge_delta(r, s) for s in props]
        keys = [O.merge_key(v) for v in vals]
        i = int(np.argmin(keys))  # first minimum
        assert bs[r] == props[i] and bd[r] == vals[i]


# --------------------------------------------------------------------------
# P8: merge application against connected components of a sorted prefix

@pytest.mark.parametrize("seed", range(10))
def test_merge_apply_components(seed):
    rng = np.random.default_rng(400 + seed)
    B = int(rng.integers(2, 40))
    best_s = np.array([rng.choice([s for s in range(B) if s != r]) for r in range(B)], np.int32)
    best_d = np.round(rng.normal(size=B), 1)  # ties on purpose
    n_merges = int(rng.integers(1, B))
    done, mp, Bn = O.merge_apply(B, best_s, best_d, n_merges)
    order = sorted(range(B), key=lambda r: (math.floor(best_d[r] * 2**20 + 0.5), r))
    # smallest prefix of the sorted list whose union makes n_merges links
    G = nx.Graph()
    G.add_nodes_from(range(B))
    comps = None
    for K in range(B + 1):
        if K > 0:
            r = order[K - 1]
            G.add_edge(r, int(best_s[r]))
        links = B - nx.number_connected_components(G)
        if links == n_merges or K == B:
            comps = [sorted(c) for c in nx.connected_components(G)]
            break
    assert done == B - len(comps) and Bn == B - done
    comps.sort(key=lambda c: c[0])
    for label, c in enumerate(comps):
        assert all(mp[x] == label for x in c)


def test_compact():
    Bn, b = O.compact(7, np.array([6, 2, 2, 6, 4], np.int32))
    assert Bn == 3 and b.tolist() == [2, 0, 0, 2, 1]


# --------------------------------------------------------------------------
# P9: golden-ratio bracket on a unimodal description-length curve

@pytest.mark.parametrize("bstar,N", [(37, 1000), (1, 64), (8, 1000), (500, 1000), (123, 777)])
def test_bracket_finds_minimum_of_unimodal_curve(bstar, N):
    def f(B):
        return 3.0 * (B - bstar) ** 2 + 0.5 * abs(B - bstar) + 10.0

    br = O.Bracket()
    br.insert(N, f(N))
    states = {N}
    for _ in range(200):
        more, Bs, dls, start, target = br.next(0.5)
        # invariants: hi > mid > lo by C, mid holds the smallest DL
        present = [i for i in range(3) if Bs[i] > 0]
        assert Bs[1] > 0
        if Bs[0]:
            assert Bs[0] > Bs[1] and dls[0] >= dls[1]
        if Bs[2]:
            assert Bs[2] < Bs[1] and dls[2] >= dls[1]
        if not more:
            break
        assert Bs[start] > target >= 1
        states.add(target)
        br.insert(target, f(target))
    assert not more
    assert Bs[1] == bstar


# --------------------------------------------------------------------------
# sanity of the full run (not a parity pin): strong 5:1 structure recovered

def test_partition_recovers_planted_blocks():
    g = make_config("plain_1k")
    G = O.Graph(g.n, g.src, g.dst)
    b, B, dl, sweeps = O.partition(G, O.Params())
    assert B == 8
    # identical partitions up to relabelling
    pairs = set(zip(b.tolist(), g.planted.tolist()))
    assert len(pairs) == 8
    b2, B2, dl2, _ = O.partition(G, O.Params())
    assert np.array_equal(b, b2) and dl == dl2


def test_dl_without_edges_is_the_limit():
    # E h(C^2/E) -> 0 as E -> 0 (h(x) ~ ln x + 1 for large x), so Eq. 2
    # reduces to V ln C when the graph has no edges.
    g = O.Graph(5, np.zeros(0, np.int32), np.zeros(0, np.int32))
    m = O.Model(g, 3, np.array([0, 1, 2, 0, 1], np.int32))
    assert m.dl() == pytest.approx(5 * math.log(3), rel=1e-15)
    prev = None
    for E in (1e-2, 1e-4, 1e-6, 1e-8):
        x = 9 / E
        term = E * ((1 + x) * math.log1p(x) - x * math.log(x))
        assert prev is None or term < prev
        prev = term
    assert prev < 1e-6


# --------------------------------------------------------------------------
# Hybrid pass: the h highest-degree vertices are decided one after another
# against the current state, the others against the state the sequential
# part left.  Pinned by brute-force Delta DL along that sequence.

@pytest.mark.parametrize("seed", range(4))
def test_hybrid_pass_sequential_then_frozen(seed):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(6, 13))
    src, dst = tiny_graph(rng, n, int(rng.integers(2 * n, 5 * n)), self_loops=True)
    B = int(rng.integers(2, 5))
    b = rng.integers(0, B, n).astype(np.int32)
    E = src.size
    deg = np.bincount(src, minlength=n) + np.bincount(dst, minlength=n)
    order = sorted(range(n), key=lambda v: (-deg[v], v))
    h = int(rng.integers(1, n))
    g = O.Graph(n, src, dst)
    m = O.Model(g, B, b)
    d = m.hybrid_decide(seed, 4, 0.5, h)
    state = b.copy()
    for v in order[:h]:  # sequential part: each against the current state
        if (d.flags[v] & 1) and d.s[v] != state[v]:
            b2 = state.copy()
            b2[v] = d.s[v]
            want = brute_DL(brute_M(src, dst, b2, B), E, n) - brute_DL(brute_M(src, dst, state, B), E, n)
            assert d.dH[v] == pytest.approx(want, rel=1e-10, abs=1e-10)
            if d.flags[v] & 2:
                state = b2
    assert np.array_equal(m.assignment(), state)  # the model keeps the sequential result
    base = brute_DL(brute_M(src, dst, state, B), E, n)
    want_new = state.copy()
    for v in order[h:]:  # the rest: against the frozen state
        if (d.flags[v] & 1) and d.s[v] != state[v]:
            b2 = state.copy()
            b2[v] = d.s[v]
            assert d.dH[v] == pytest.approx(brute_DL(brute_M(src, dst, b2, B), E, n) - base, rel=1e-10, abs=1e-10)
            if d.flags[v] & 2:
                want_new[v] = d.s[v]
    assert np.array_equal(d.b_new, want_new)


def test_hybrid_with_h0_is_the_async_pass():
    g = make_config("plain_1k")
    G = O.Graph(g.n, g.src, g.dst)
    b = random_labels(g.n, 8, seed=2)
    a = O.Model(G, 8, b).nodal_decide(5, 1, 3.0)
    h = O.Model(G, 8, b).hybrid_decide(5, 1, 3.0, 0)
    assert np.array_equal(a.b_new, h.b_new) and np.array_equal(a.dH, h.dH)
