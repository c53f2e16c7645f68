"""Pins for the oracle's random draws and its phase rules, against values
computed here without the oracle's code.

- The words of each nodal draw: the proposal (P3) and the acceptance
  uniform u of the Metropolis test (Alg. 2, "accept with probability ...")
  are re-derived from numpy's own Philox bit generator, with u = (w2 >> 11)
  2^-53, and the decision from the brute-force Delta DL and the enumerated
  Hastings sums.
- The empirical acceptance rate of many proposals against min(1, e^logA).
- The stop rule of an MCMC phase (Alg. 2, "until Delta DL < t DL or x
  times"): the DL after every sweep recomputed from scratch (Eq. 1-2 by
  numpy), and the phase must stop at the first sweep k >= 3 with
  |DL_{k-3} - DL_k| < t DL_k, for both thresholds and the sweep cap.
- The merge phase's extra proposal rounds (Alg. 1 merge loop): a graph whose
  first round cannot make the requested links, so that a second round runs.
- The full run's phase sequence replayed through the bracket rule alone.
"""
import math

import numpy as np
import pytest

import oracle as O
from synth.dcsbm import make_config, random_labels

from test_oracle_pins import brute_DL, brute_M, tiny_graph

MASK64 = (1 << 64) - 1


def numpy_philox(ctr, key):
    """Philox4x64-10 block for counter ctr from numpy's implementation
    (numpy increments its 256-bit counter before producing a block)."""
    c = sum(int(x) << (64 * i) for i, x in enumerate(ctr))
    c = (c - 1) % (1 << 256)
    prev = [(c >> (64 * i)) & MASK64 for i in range(4)]
    gen = np.random.Philox(counter=np.array(prev, np.uint64), key=np.array([int(k) for k in key], np.uint64))
    return [int(x) for x in gen.random_raw(4)]


def nbr_list(src, dst, v):
    """Out-neighbours ascending, then in-neighbours ascending (P3's order)."""
    out = sorted(int(d) for s, d in zip(src, dst) if s == v)
    inn = sorted(int(s) for s, d in zip(src, dst) if d == v)
    return out + inn


def proposal_from_words(w, src, dst, b, B, M, v):
    """P3 written out with Python integers: j-th incident edge from w0, then
    the block from w1 (uniform part, row u, column u)."""
    nb = nbr_list(src, dst, v)
    if not nb:
        return None
    j = (w[0] * len(nb)) >> 64
    u = int(b[nb[j]])
    dout_u, din_u = int(M[u].sum()), int(M[:, u].sum())
    y = (w[1] * (dout_u + din_u + B)) >> 64
    if y < B:
        return y
    t = y - B
    if t < dout_u:
        return int(np.searchsorted(np.cumsum(M[u]), t, side="right"))
    t -= dout_u
    return int(np.searchsorted(np.cumsum(M[:, u]), t, side="right"))


@pytest.mark.parametrize("seed", range(4))
def test_nodal_draws_follow_philox_words(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(8, 30))
    src, dst = tiny_graph(rng, n, int(rng.integers(2 * n, 5 * n)))
    B = int(rng.integers(2, 7))
    b = rng.integers(0, B, n).astype(np.int32)
    G = O.Graph(n, src, dst)
    m = O.Model(G, B, b)
    M = brute_M(src, dst, b, B)
    beta, key = 1.5, 77 + seed
    movers = 0
    for sweep in range(6):
        od = m.nodal_decide(key, sweep, beta)
        for v in range(n):
            w = numpy_philox([sweep, v, 0, 0], [key, 0])
            s = proposal_from_words(w, src, dst, b, B, M, v)
            if s is None:
                assert od.flags[v] == 0 and od.s[v] == b[v]
                continue
            assert od.s[v] == s and od.flags[v] & 1
            if s == b[v]:
                assert not od.flags[v] & 2
                continue
            movers += 1
            u = (w[2] >> 11) * 2.0 ** -53
            lnu = math.log(u) if u > 0 else -math.inf
            assert od.lnu[v] == lnu
            # logA from the brute-force-pinned Delta DL and Hastings sums
            dH, pf, pb = m.move_delta(v, s)
            logA = -beta * dH + math.log(pb) - math.log(pf)
            assert od.logA[v] == pytest.approx(logA, rel=1e-12, abs=1e-12)
            accept = logA >= 0 or lnu < logA
            assert bool(od.flags[v] & 2) == accept
            assert od.b_new[v] == (s if accept else b[v])
    assert movers > 20


def test_acceptance_rate_matches_metropolis_probability():
    # one frozen state, many sweep ids: every move is accepted with
    # probability min(1, e^logA), so the accepted count over moves grouped by
    # that probability matches its expectation
    g = make_config("plain_1k")
    B = 8
    b = random_labels(g.n, B, seed=4)
    m = O.Model(O.Graph(g.n, g.src, g.dst), B, b)
    ps, acc = [], []
    for sweep in range(60):
        od = m.nodal_decide(9, sweep, 0.05)
        mv = (od.flags & 1).astype(bool) & (od.s != b)
        ps.append(np.minimum(1.0, np.exp(od.logA[mv])))
        acc.append((od.flags[mv] & 2) != 0)
    p = np.concatenate(ps)
    a = np.concatenate(acc)
    edges = [0.0, 0.1, 0.3, 0.5, 0.7, 0.9, 0.999999, 1.0 + 1e-9]
    checked = 0
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (p >= lo) & (p < hi)
        if sel.sum() < 200:
            continue
        mean, var = p[sel].sum(), (p[sel] * (1 - p[sel])).sum()
        z = (a[sel].sum() - mean) / math.sqrt(max(var, 1e-12))
        assert abs(z) < 4.5, (lo, hi, int(sel.sum()), z)
        checked += 1
    assert checked >= 4
    # certain acceptances (logA >= 0) are all taken
    assert np.all(a[p >= 1.0])


def _dl_history(src, dst, n, B, b, seed, beta, sweeps, first_sweep=0):
    """DL after 0..sweeps asynchronous sweeps, each DL recomputed from
    scratch by numpy (the model only supplies the per-sweep decisions)."""
    m = O.Model(O.Graph(n, src, dst), B, b)
    hist = [brute_DL(brute_M(src, dst, b, B), src.size, n)]
    for k in range(sweeps):
        od = m.nodal_decide(seed, first_sweep + k, beta)
        m.set_b(B, od.b_new)
        hist.append(brute_DL(brute_M(src, dst, od.b_new, B), src.size, n))
    return np.array(hist)


def _first_stop(hist, t, max_sweeps):
    for k in range(3, max_sweeps + 1):
        if abs(hist[k - 3] - hist[k]) < t * hist[k]:
            return k
    return max_sweeps


@pytest.mark.parametrize("B,start_seed", [(8, 4), (16, 6)])
def test_mcmc_phase_stops_at_first_converged_sweep(B, start_seed):
    g = make_config("plain_1k")
    b = random_labels(g.n, B, seed=start_seed)
    cap = 40
    p = O.Params(seed=3, max_sweeps=cap)
    ref = _dl_history(g.src, g.dst, g.n, B, b, 3, 3.0, cap, first_sweep=10)
    stops = {}
    for t in (5e-4, 1e-4, 1e-2, 0.0):
        m = O.Model(O.Graph(g.n, g.src, g.dst), B, b)
        ns, hist = m.mcmc_phase(p, 10, t)
        want = _first_stop(ref, t, cap)
        assert ns == want, (t, ns, want)
        assert np.allclose(hist, ref[: ns + 1], rtol=1e-12, atol=0)
        stops[t] = ns
    # the thresholds are exercised: the driver's two stop at different
    # sweeps before the cap, a loose one at the first sweep the rule can
    # stop at, and t = 0 runs to the cap
    assert 3 == stops[1e-2] < stops[5e-4] < stops[1e-4] < stops[0.0] == cap


def _paired_blocks_graph(pairs=3, size=12, seed=0):
    """2*pairs groups of vertices; edges only inside a group and between the
    two groups of a pair.  The planted labels are the groups."""
    rng = np.random.default_rng(seed)
    n = 2 * pairs * size
    src, dst = [], []
    for p in range(pairs):
        a = np.arange(2 * p * size, (2 * p + 2) * size)
        for _ in range(8 * size):
            x, y = rng.choice(a, 2, replace=False)
            src.append(x)
            dst.append(y)
    b = (np.arange(n) // size).astype(np.int32)
    return n, np.array(src, np.int32), np.array(dst, np.int32), b


def test_merge_phase_takes_another_round_when_proposals_run_out():
    # 6 blocks in 3 pairs with no edge between pairs: in round 0 every block's
    # best merge is its partner, so at most 3 links form; asking for 4 needs
    # a second proposal round on the merged model
    n, src, dst, b = _paired_blocks_graph()
    B, n_merges, seed = 6, 4, 5
    p = O.Params(seed=seed)
    G = O.Graph(n, src, dst)
    m = O.Model(G, B, b)
    Bn, rounds = m.merge_phase(p, 20, n_merges)
    assert (Bn, rounds) == (B - n_merges, 2)
    # the same two rounds from the pinned pieces: proposals of round 20, the
    # application (pinned against connected components), the rebuilt model,
    # then proposals of round 21 for the remaining links
    m0 = O.Model(G, B, b)
    bs, bd = m0.merge_proposals(seed, 20, 10)
    done0, map0, B0 = O.merge_apply(B, bs, bd, n_merges)
    assert done0 == 3 and B0 == 3
    b1 = map0[b]
    m1 = O.Model(G, B0, b1)
    bs1, bd1 = m1.merge_proposals(seed, 21, 10)
    done1, map1, B1 = O.merge_apply(B0, bs1, bd1, n_merges - done0)
    assert done1 == 1 and B1 == 2
    assert np.array_equal(m.assignment(), map1[b1])
    assert np.array_equal(m.dense(), brute_M(src, dst, map1[b1], B1))


def test_merge_phase_single_round_when_enough_links():
    n, src, dst, b = _paired_blocks_graph(seed=2)
    m = O.Model(O.Graph(n, src, dst), 6, b)
    assert m.merge_phase(O.Params(seed=1), 0, 3) == (3, 1)


def test_partition_phases_follow_the_bracket_rule():
    # every phase of a full run, replayed through the bracket rule alone
    # (pinned on unimodal curves): its start state and target, t_pre while
    # no lower bracket end exists and t_post after, the exact merge count,
    # and the end of the search
    g = make_config("plain_1k")
    p = O.Params()
    b, B, dl, sweeps, log = O.partition(O.Graph(g.n, g.src, g.dst), p, nthreads=4, phase_log=True)
    br = O.Bracket()
    br.insert(g.n, O.Model(O.Graph(g.n, g.src, g.dst), g.n, np.arange(g.n, dtype=np.int32)).dl())
    seen_post = False
    for row in log:
        B0, target, Bm, t, ns, Bc, dlc = row
        more, Bs, dls, start, tg = br.next(p.reduction)
        assert more
        assert Bs[start] == B0 and tg == target
        assert Bm == target
        if Bs[2] == 0:
            assert t == p.t_pre
        else:
            assert t == p.t_post
            seen_post = True
        assert 1 <= ns <= p.max_sweeps
        assert Bc <= Bm
        br.insert(int(Bc), float(dlc))
    more, Bs, dls, _, _ = br.next(p.reduction)
    assert not more
    assert Bs[1] == B and dls[1] == dl
    assert int(log[:, 4].sum()) == sweeps
    assert seen_post and log[0, 3] == p.t_pre
