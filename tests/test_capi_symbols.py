"""The C-ABI library builds for sm_103a, loads, and exports every function
that the headers under include/ declare.  No compute call is made (no GPU
needed), except the host-only checks."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_text():
    """Every header under include/, comments removed."""
    d = os.path.join(ROOT, "include")
    text = ""
    for name in sorted(os.listdir(d)):
        if name.endswith(".h"):
            with open(os.path.join(d, name)) as f:
                text += f.read() + "\n"
    return re.sub(r"/\*.*?\*/", "", text, flags=re.S)


def declared_functions():
    text = header_text()
    names = re.findall(r"\b(?:int|void|size_t)\s+\**(sbp_\w+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["sbp_load_graph", "sbp_build_blockmodel", "sbp_nodal_sweep", "sbp_merge_blocks", "sbp_partition",
                     "sbp_bracket_check"]:
        assert required in names


def test_library_builds_and_exports_every_symbol():
    from paper_2305_18663_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    import paper_2305_18663_gb300 as P

    for n in declared_functions():
        assert hasattr(P, n), n


def test_vertex_dealing_covers_each_vertex_once():
    import numpy as np

    from paper_2305_18663_gb300 import deal_vertices

    rng = np.random.default_rng(0)
    deg = rng.integers(0, 100, 1001)
    for world in (1, 2, 3, 8):
        parts = [deal_vertices(deg, world, r) for r in range(world)]
        allv = np.sort(np.concatenate(parts))
        assert np.array_equal(allv, np.arange(deg.size))
        sizes = [p.size for p in parts]
        assert max(sizes) - min(sizes) <= 2
        # each rank gets both high- and low-degree vertices
        loads = [deg[p].sum() for p in parts]
        assert max(loads) - min(loads) <= deg.max() * 2


def declared_arity():
    """Parameter count of every function the headers declare."""
    text = header_text()
    out = {}
    for m in re.finditer(r"\b(?:int|void|size_t)\s+\**(sbp_\w+)\s*\(([^)]*)\)\s*;", text):
        params = m.group(2).strip()
        out[m.group(1)] = 0 if params in ("", "void") else len(params.split(","))
    return out


def test_binding_signatures_match_the_header():
    # every ctypes prototype takes as many arguments as the C declaration
    import paper_2305_18663_gb300 as P

    lib = P.load()
    arity = declared_arity()
    assert arity, "no declarations parsed"
    for name, n in arity.items():
        fn = getattr(lib, name)
        assert fn.argtypes is not None, name
        assert len(fn.argtypes) == n, (name, len(fn.argtypes), n)


def _search_like_sequence(rng, n0, reduction=0.5):
    """States in the order a golden-ratio search visits them: the next B
    from the host bracket's own plan (read back after each insert), DL a
    noisy convex function of B with its minimum at a random block count."""
    import numpy as np

    import paper_2305_18663_gb300 as P

    best = int(rng.integers(2, max(3, n0 // 4)))
    Bs, dls = [n0], [1e6 * (1 + (np.log(n0) - np.log(best)) ** 2)]
    for _ in range(60):
        out, bad = P.sbp_bracket_check(Bs, dls, reduction)
        assert bad == 0
        if not out[-1, 3]:
            break
        B = int(out[-1, 5])
        Bs.append(B)
        dls.append(1e6 * (1 + (np.log(B) - np.log(best)) ** 2) + rng.normal(0, 1e3))
    return Bs, dls


def test_kernel_bracket_follows_the_host_bracket():
    # the persistent kernel's copy of the golden-ratio bracket (compiled for
    # the host as well) against the host driver's Bracket: the same positions
    # and ids after every insert, the same next phase (start and target), and
    # label slots that never collide; on search-like sequences, on random
    # ones, and with equal DL values (ties go to the same side)
    import numpy as np

    import paper_2305_18663_gb300 as P

    rng = np.random.default_rng(7)
    for trial in range(200):
        n0 = int(rng.integers(2, 5000))
        red = float(rng.choice([0.5, 0.3, 0.7]))
        Bs, dls = _search_like_sequence(rng, n0, red)
        out, bad = P.sbp_bracket_check(Bs, dls, red)
        assert bad == 0, (trial, Bs)
        assert np.array_equal(out[:, :6], out[:, 6:])
        # the search ends: the last plan says no next phase, or the bracket
        # is down to adjacent block counts
        assert not out[-1, 3] or len(Bs) == 61
    for trial in range(200):
        k = int(rng.integers(1, 30))
        Bs = rng.integers(1, 3000, k)
        dls = rng.choice([1.0, 2.0, 3.0], k) if trial % 2 else rng.normal(1e6, 1e4, k)
        out, bad = P.sbp_bracket_check(Bs, dls, 0.5)
        assert bad == 0, trial
    # first insert of B = N with reduction 0.5: merge to ceil(N / 2)
    out, bad = P.sbp_bracket_check([1000], [5.0], 0.5)
    assert bad == 0 and out[0, 3] == 1 and out[0, 4] == 1 and out[0, 5] == 500
    out, bad = P.sbp_bracket_check([1], [5.0], 0.5)
    assert bad == 0 and out[0, 3] == 0  # one block: nothing left to merge
