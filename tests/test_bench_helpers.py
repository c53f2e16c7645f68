"""Host-side helpers of bench.py (no GPU): the code hash that keys the
committed DRAM-traffic figure to the kernels it was measured on, and the
algorithmic-bytes formula of the roofline, and the NMI of the full-run
reports."""
import pytest

import bench


def test_code_hash_ignores_comments_and_whitespace_only():
    a = "int f(int x) {\n  // count\n  return x + 1; /* done */\n}\n"
    b = "int f(int x)\n{ return x + 1; }  // reformatted, other comment\n"
    c = "int f(int x) { return x + 2; }\n"
    assert bench.code_only(a) == bench.code_only(b)
    assert bench.code_only(a) != bench.code_only(c)


def test_traffic_figure_only_for_its_form_and_code():
    t = bench.decide_traffic("sparse")
    # the committed figure belongs to the sparse-row form; the dense form has none
    assert bench.decide_traffic("dense") is None
    if t is not None:  # present exactly while the decide-pass code is unchanged
        # the pass must at least stream the movers' rows from DRAM, and the
        # lookups it adds to the algorithmic bytes are served from L2
        assert 0.9 * t["streamed_bytes"] <= t["bytes"] <= t["algorithmic_bytes"]


def test_algorithmic_bytes_formula():
    # the per-sweep bytes of the measurement table: streamed offsets,
    # labels, the proposal's edge and the moving rows; the proposal's
    # inverse-CDF search; four blockmodel counts and two degrees per
    # distinct neighbour block of a moving vertex (hash probes of 8 bytes
    # on sparse rows)
    n, m, B, me, ent = 1000, 5000, 10, 1234, 3000
    dec, streamed, reb = bench.algorithmic_bytes(n, m, B, me, ent)
    assert streamed == 8 * (n + 1) + 16 * n + 8 * me
    assert dec == streamed + 4 * 5 * n + ent * (4 * 4 + 8)  # 2B = 20 prefix entries: 5 halvings
    assert reb == 16 * m + 12 * B * B
    dec_s, streamed_s, _ = bench.algorithmic_bytes(n, m, B, me, ent, sparse=True, nnz=40)
    assert streamed_s == streamed
    assert dec_s == streamed + 4 * 3 * n + ent * (4 * 8 + 8)  # rows and columns of 8 entries on average


def test_nmi_of_the_full_run_reports():
    # the NMI the full-run lines report: 1 for the same partition under any
    # relabelling, near 0 for independent labels, symmetric, and equal to
    # the textbook value on a small hand-worked case
    import numpy as np

    rng = np.random.default_rng(0)
    a = rng.integers(0, 8, 5000)
    perm = rng.permutation(8)
    assert bench.nmi(a, perm[a]) == pytest.approx(1.0, abs=1e-12)
    b = rng.integers(0, 8, 5000)
    assert bench.nmi(a, b) < 0.01
    assert bench.nmi(a, b) == pytest.approx(bench.nmi(b, a), abs=1e-12)
    # a = [0,0,1,1], b = [0,0,0,1]: H(a) = ln 2, H(b) = H(1/4), I = H(b) - H(b|a)
    h = lambda p: -sum(x * np.log(x) for x in p if x > 0)  # noqa: E731
    hb = h([0.75, 0.25])
    mi = hb - 0.5 * h([0.5, 0.5])
    assert bench.nmi([0, 0, 1, 1], [0, 0, 0, 1]) == pytest.approx(2 * mi / (np.log(2) + hb), rel=1e-12)
    assert bench.nmi([3, 3, 3], [1, 1, 1]) == 1.0  # one block on both sides
