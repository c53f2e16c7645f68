"""Host-side helpers of bench.py (no GPU): the code hash that keys the
committed DRAM-traffic figure to the kernels it was measured on, and the
algorithmic-bytes formula of the roofline."""
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
        assert t["bytes"] > t["algorithmic_bytes"] > 0


def test_algorithmic_bytes_formula():
    n, m, B, me = 1000, 5000, 10, 1234
    dec, reb = bench.algorithmic_bytes(n, m, B, me)
    assert dec == 8 * (n + 1) + 12 * n + 8 * me
    assert reb == 16 * m + 12 * B * B
