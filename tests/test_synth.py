"""The synthetic inputs follow their stated recipe (no GPU): the directed
DCSBM generator (exact edge count, no self-loops or duplicates, planted block
sizes, the intra-block share of the edges, the degree law's truncation,
determinism per seed), the perturbed start of the sweep benchmark, and the
size laws of the batching and serving workloads."""
import numpy as np
import pytest

from synth.dcsbm import CONFIGS, batch_specs, block_sizes, dcsbm, make_config, perturb, serving_specs


def test_edges_distinct_without_self_loops_and_exact_count():
    g = dcsbm(n=3000, e=30000, n_blocks=12, gamma=2.2, kmin=1, kmax=200, ratio=4.0, sizes="lognormal", seed=3)
    assert g.m == 30000
    assert not np.any(g.src == g.dst)
    key = g.src.astype(np.int64) * g.n + g.dst
    assert np.unique(key).size == g.m
    assert g.src.min() >= 0 and g.src.max() < g.n and g.dst.min() >= 0 and g.dst.max() < g.n


@pytest.mark.parametrize("ratio", [1.0, 3.0, 5.0])
def test_intra_block_share_is_ratio_over_one_plus_ratio(ratio):
    # on a sparse graph (few duplicate draws to drop) the share of edges
    # inside a block is ratio / (1 + ratio) up to the binomial spread
    g = dcsbm(n=50_000, e=300_000, n_blocks=20, gamma=2.5, kmin=1, kmax=100, ratio=ratio, seed=5)
    intra = float(np.mean(g.planted[g.src] == g.planted[g.dst]))
    assert intra == pytest.approx(ratio / (1 + ratio), abs=0.01)
    # dense blocks draw more intra-block duplicates, which are dropped and
    # redrawn: the share then falls a little short, never above
    d = dcsbm(n=5000, e=60000, n_blocks=20, gamma=2.5, kmin=1, kmax=100, ratio=ratio, seed=5)
    dense_intra = float(np.mean(d.planted[d.src] == d.planted[d.dst]))
    assert ratio / (1 + ratio) - 0.04 < dense_intra < ratio / (1 + ratio)


def test_block_sizes_equal_and_lognormal():
    rng = np.random.Generator(np.random.Philox(0))
    eq = block_sizes(1000, 8, "equal", 1.0, rng)
    assert eq.sum() == 1000 and eq.max() - eq.min() <= 1
    ln = block_sizes(200_000, 100, "lognormal", 1.0, rng)
    assert ln.sum() == 200_000 and ln.min() >= 1
    # log-normal(sigma = 1) weights: the sizes spread well beyond equal ones
    assert ln.max() / np.median(ln) > 3
    g = dcsbm(n=1000, e=5000, n_blocks=8, gamma=2.5, kmin=1, kmax=100, ratio=5.0, sizes="equal", seed=1)
    assert np.array_equal(np.bincount(g.planted, minlength=8), eq)


def test_degrees_follow_the_truncated_power_law():
    # expected degrees are proportional to theta in [kmin, kmax]: a heavy
    # tail (max far above the mean) yet no vertex's out-degree beyond what
    # the largest weight can draw
    c = dict(CONFIGS["plain_200k"])
    c.update(n=50_000, e=1_000_000)
    g = dcsbm(seed=0, **c)
    dout = np.bincount(g.src, minlength=g.n)
    mean = g.m / g.n
    assert dout.max() > 20 * mean
    # theta_max / mean theta bounds the expected degree ratio; 3x covers the draw
    k = np.arange(c["kmin"], c["kmax"] + 1, dtype=np.float64)
    p = k ** -c["gamma"]
    mean_theta = float((k * p).sum() / p.sum())
    assert dout.max() <= 3 * mean * c["kmax"] / mean_theta
    assert np.mean(dout == 0) < 0.5


def test_generator_is_deterministic_per_seed():
    a = make_config("plain_1k", seed=0)
    b = make_config("plain_1k", seed=0)
    c = make_config("plain_1k", seed=1)
    assert np.array_equal(a.src, b.src) and np.array_equal(a.dst, b.dst) and np.array_equal(a.planted, b.planted)
    assert not np.array_equal(a.src, c.src)
    assert a.n == 1000 and a.m == 10_000 and a.n_blocks == 8


def test_perturbed_start_reassigns_the_stated_share():
    lab = np.repeat(np.arange(10, dtype=np.int32), 1000)
    b = perturb(lab, 10, 0.3, seed=0)
    changed = float(np.mean(b != lab))
    # 30% are redrawn uniformly over 10 blocks, so 90% of them land elsewhere
    assert changed == pytest.approx(0.3 * 0.9, abs=0.02)
    assert b.min() >= 0 and b.max() < 10
    assert np.array_equal(b, perturb(lab, 10, 0.3, seed=0))


def test_batching_and_serving_size_laws():
    specs = batch_specs(4096, seed=0)
    n = np.array([s["n"] for s in specs])
    deg = np.array([s["e"] / s["n"] for s in specs])
    assert n.min() >= 500 and n.max() <= 50_000
    # log-uniform: the median near the geometric mean of the range
    assert np.median(n) == pytest.approx(np.sqrt(500 * 50_000), rel=0.1)
    assert deg.min() >= 8 - 1e-3 and deg.max() <= 32 + 1e-3
    assert all(s["n_blocks"] == max(1, int(round(np.sqrt(s["n"]) / 2))) for s in specs)
    assert all(s["gamma"] == 2.5 and s["ratio"] == 4.0 for s in specs)
    srv = serving_specs(200, seed=0)
    ns = np.array([s["n"] for s in srv])
    assert ns.min() >= 1000 and ns.max() <= 2_000_000
    assert all(s["e"] == 16 * s["n"] for s in srv)
