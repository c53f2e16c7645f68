"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/sbp.h declares.  No compute call is made (no GPU needed)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    with open(os.path.join(ROOT, "include", "sbp.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(?:int|void|size_t)\s+\**(sbp_\w+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["sbp_load_graph", "sbp_build_blockmodel", "sbp_nodal_sweep", "sbp_merge_blocks", "sbp_partition"]:
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
    """Parameter count of every function include/sbp.h declares."""
    with open(os.path.join(ROOT, "include", "sbp.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
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
