"""Seeded synthetic directed degree-corrected SBM graphs.

This module only draws inputs: it contains none of the partitioning
arithmetic, so both the CPU oracle and the CUDA path can be fed from it.

The recipe follows the structure the paper describes for its synthetic
graphs (Section IV-A, Tables 3-4): power-law degree sequences truncated to
``[kmin, kmax]``, independent out- and in-degree sequences (the
"non-duplicated" variant of Table 3), a fixed intra:inter edge ratio and
planted community sizes that are either equal or varied.

Steps (all draws from ``numpy.random.Generator(Philox(seed))``):

1. planted block sizes: equal, or log-normal(sigma) weights normalised to
   ``n`` with largest-remainder rounding and a minimum of one vertex;
   vertices are dealt to blocks in a random order;
2. per-vertex weights ``theta_out`` and ``theta_in`` drawn independently
   from the discrete power law ``P(k) ~ k**-gamma`` on ``[kmin, kmax]``;
3. edges: source ~ ``theta_out``; with probability ``ratio / (1 + ratio)``
   the target block is the source's block, otherwise another block chosen in
   proportion to its summed ``theta_in``; the target vertex within the block
   ~ ``theta_in``;
4. self-loops and duplicate edges are dropped and redrawn, so the edge count
   is ``e`` up to a small deficit when the redraw cap is hit.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = ["Graph", "dcsbm", "perturb", "block_sizes", "CONFIGS", "make_config", "batch_specs", "serving_specs"]


@dataclass
class Graph:
    n: int
    src: np.ndarray  # int32[m]
    dst: np.ndarray  # int32[m]
    planted: np.ndarray  # int32[n]
    n_blocks: int

    @property
    def m(self) -> int:
        return int(self.src.shape[0])


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


def block_sizes(n: int, n_blocks: int, sizes: str, sigma: float, rng) -> np.ndarray:
    if n_blocks < 1 or n_blocks > n:
        raise ValueError("need 1 <= n_blocks <= n")
    if sizes == "equal":
        w = np.ones(n_blocks)
    elif sizes == "lognormal":
        w = rng.lognormal(0.0, sigma, n_blocks)
    else:
        raise ValueError(sizes)
    # one vertex per block up front, the rest by largest remainder
    rest = n - n_blocks
    q = w / w.sum() * rest
    base = np.floor(q).astype(np.int64)
    short = rest - int(base.sum())
    order = np.argsort(-(q - base), kind="stable")
    base[order[:short]] += 1
    return base + 1


def _sorted_unique(a: np.ndarray) -> np.ndarray:
    a = np.sort(a)
    if a.size == 0:
        return a
    keep = np.empty(a.size, dtype=bool)
    keep[0] = True
    np.not_equal(a[1:], a[:-1], out=keep[1:])
    return a[keep]


def _powerlaw(rng, size: int, gamma: float, kmin: int, kmax: int) -> np.ndarray:
    k = np.arange(kmin, kmax + 1, dtype=np.float64)
    cdf = np.cumsum(k ** -gamma)
    cdf /= cdf[-1]
    idx = np.searchsorted(cdf, rng.random(size), side="right")
    return k[np.minimum(idx, k.size - 1)]


def dcsbm(
    n: int,
    e: int,
    n_blocks: int,
    gamma: float,
    kmin: int,
    kmax: int,
    ratio: float,
    sizes: str = "equal",
    sigma: float = 1.0,
    seed: int = 0,
    max_redraw: int = 50,
) -> Graph:
    rng = _rng(seed)
    sz = block_sizes(n, n_blocks, sizes, sigma, rng)
    planted = np.repeat(np.arange(n_blocks, dtype=np.int32), sz)
    planted = planted[rng.permutation(n)]

    th_out = _powerlaw(rng, n, gamma, kmin, kmax)
    th_in = _powerlaw(rng, n, gamma, kmin, kmax)

    # vertices grouped by block, with cumulative theta_in inside each block
    by_block = np.argsort(planted, kind="stable")
    blk_start = np.concatenate([[0], np.cumsum(sz)])
    cin = np.cumsum(th_in[by_block])
    blk_cin_start = np.concatenate([[0.0], cin])[blk_start[:-1]]
    blk_tot = np.add.reduceat(th_in[by_block], blk_start[:-1])
    blk_cdf = np.cumsum(blk_tot) / blk_tot.sum()
    out_cdf = np.cumsum(th_out) / th_out.sum()
    p_intra = ratio / (1.0 + ratio)

    def draw(count: int):
        # edge order is irrelevant, so sorted uniforms keep the search cache-friendly
        s = np.searchsorted(out_cdf, np.sort(rng.random(count)), side="right")
        s = np.minimum(s, n - 1)
        sb = planted[s]
        tb = sb.copy()
        inter = rng.random(count) >= p_intra
        if n_blocks > 1:
            pending = np.flatnonzero(inter)
            while pending.size:
                cand = np.minimum(np.searchsorted(blk_cdf, rng.random(pending.size), side="right"), n_blocks - 1)
                ok = cand != sb[pending]
                tb[pending[ok]] = cand[ok]
                pending = pending[~ok]
        x = blk_cin_start[tb] + rng.random(count) * blk_tot[tb]
        o = np.argsort(x)
        pos = np.empty(count, dtype=np.int64)
        pos[o] = np.searchsorted(cin, x[o], side="right")
        pos = np.clip(pos, blk_start[tb], blk_start[tb + 1] - 1)
        d = by_block[pos]
        return s.astype(np.int64), d.astype(np.int64)

    keys = np.empty(0, dtype=np.int64)
    need = e
    for _ in range(max_redraw):
        if need <= 0:
            break
        s, d = draw(need + need // 16 + 16)
        keep = s != d
        k = s[keep] * n + d[keep]
        keys = _sorted_unique(np.concatenate([keys, k]))
        if keys.size > e:
            # drop a random surplus to keep exactly e distinct edges
            drop = rng.choice(keys.size, keys.size - e, replace=False)
            keys = np.delete(keys, drop)
        need = e - keys.size
    order = rng.permutation(keys.size)
    keys = keys[order]
    return Graph(
        n=n,
        src=(keys // n).astype(np.int32),
        dst=(keys % n).astype(np.int32),
        planted=planted.astype(np.int32),
        n_blocks=n_blocks,
    )


def perturb(labels: np.ndarray, n_blocks: int, frac: float, seed: int = 0) -> np.ndarray:
    """Reassign a ``frac`` share of the vertices to uniformly drawn blocks."""
    rng = _rng(seed)
    b = labels.astype(np.int32).copy()
    n = b.size
    pick = rng.permutation(n)[: int(round(frac * n))]
    b[pick] = rng.integers(0, n_blocks, pick.size, dtype=np.int32)
    return b


def random_labels(n: int, n_blocks: int, seed: int = 0) -> np.ndarray:
    """Uniform random block labels in ``[0, n_blocks)``."""
    return _rng(seed).integers(0, n_blocks, n, dtype=np.int32)


# The five workloads: sizes, degree law, structure.
CONFIGS = {
    "plain_1k": dict(n=1_000, e=10_000, n_blocks=8, gamma=2.5, kmin=1, kmax=100, ratio=5.0, sizes="equal"),
    "plain_200k": dict(n=200_000, e=4_000_000, n_blocks=100, gamma=2.1, kmin=1, kmax=2000, ratio=2.0, sizes="lognormal"),
    "dcsbm_1m": dict(n=1_000_000, e=20_000_000, n_blocks=316, gamma=2.1, kmin=1, kmax=2000, ratio=3.0, sizes="lognormal"),
}


def make_config(name: str, seed: int = 0, scale: float = 1.0) -> Graph:
    c = dict(CONFIGS[name])
    if scale != 1.0:
        c["n"] = max(int(c["n"] * scale), c["n_blocks"])
        c["e"] = max(int(c["e"] * scale), 1)
    return dcsbm(seed=seed, **c)


def batch_specs(count: int = 4096, seed: int = 0, n_lo: int = 500, n_hi: int = 50_000) -> list[dict]:
    """The many-small-graphs workload: N log-uniform in [n_lo, n_hi], mean
    out-degree uniform in [8, 32], planted B = round(sqrt(N) / 2), degree
    exponent 2.5 clipped to [1, 100], intra:inter 4:1, equal planted blocks.
    Returns the keyword arguments of ``dcsbm`` for each graph (graph i uses
    seed ``seed * 1_000_003 + i``)."""
    rng = _rng(seed)
    n = np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), count)).astype(np.int64)
    deg = rng.uniform(8.0, 32.0, count)
    out = []
    for i in range(count):
        ni = int(n[i])
        out.append(dict(n=ni, e=int(round(ni * deg[i])), n_blocks=max(1, int(round(np.sqrt(ni) / 2))), gamma=2.5,
                        kmin=1, kmax=100, ratio=4.0, sizes="equal", seed=seed * 1_000_003 + i))
    return out


def serving_specs(count: int, seed: int = 0, n_lo: int = 1_000, n_hi: int = 2_000_000) -> list[dict]:
    """Requests of the serving workload: N log-uniform in [n_lo, n_hi], mean
    out-degree 16, planted B = round(sqrt(N) / 2), degree exponent 2.3 clipped
    to [1, 1000], intra:inter 3:1 (the ratio is not stated for this workload),
    log-normal planted sizes."""
    rng = _rng(seed + 7)
    n = np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), count)).astype(np.int64)
    out = []
    for i in range(count):
        ni = int(n[i])
        out.append(dict(n=ni, e=16 * ni, n_blocks=max(1, int(round(np.sqrt(ni) / 2))), gamma=2.3, kmin=1, kmax=1000,
                        ratio=3.0, sizes="lognormal", seed=seed * 1_000_003 + 500_000 + i))
    return out

