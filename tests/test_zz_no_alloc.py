"""The allocation-free DL entry point agrees with the library's own DL.

sbp_dense_dl_noalloc is for callers that must not allocate device memory
while running (its scratch is a fixed device array inside the library).
For the same blockmodel it must give the DL that the model reports through
sbp_get_dl, within the 1e-12 relative tolerance of the parity tests, call
after call (the calls share that scratch).  This file is named so pytest
collects it last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2305_18663_gb300 as P  # noqa: E402
from synth.dcsbm import make_config, random_labels  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.load()


def _dl_noalloc(pm, g, B):
    dev = torch.device("cuda")
    M = torch.zeros(B * B, dtype=torch.int32, device=dev)
    dout = torch.zeros(B, dtype=torch.int32, device=dev)
    din = torch.zeros(B, dtype=torch.int32, device=dev)
    P.sbp_get_blockmodel_dense(pm.h, M)
    P.sbp_get_degrees(pm.h, dout, din)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
    P.sbp_dense_dl_noalloc(M, B, dout, din, g.m, g.n, out)
    torch.cuda.synchronize()
    return float(out.item())


def test_noalloc_dl_matches_model_dl_on_consecutive_calls():
    g = make_config("plain_1k")
    pg = P.Graph(g.n, g.src, g.dst)
    seen = {}
    for B, seed in [(64, 1), (500, 2), (64, 1), (1000, 3)]:
        b = random_labels(g.n, B, seed=seed) if B < g.n else np.arange(g.n, dtype=np.int32)
        pm = P.Model(pg, B, b)
        got = _dl_noalloc(pm, g, B)
        assert got == pytest.approx(pm.dl(), rel=1e-12)
        if (B, seed) in seen:  # same input again: same result from the shared scratch
            assert got == seen[(B, seed)]
        seen[(B, seed)] = got
        pm.close()


def test_noalloc_dl_rejects_B_beyond_scratch():
    dev = torch.device("cuda")
    B = 4097
    M = torch.zeros(1, dtype=torch.int32, device=dev)
    d = torch.zeros(1, dtype=torch.int32, device=dev)
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    with pytest.raises(P.SbpError) as e:
        P.sbp_dense_dl_noalloc(M, B, d, d, 10, 10, out)
    assert e.value.code == -1 and "4096" in str(e.value)
