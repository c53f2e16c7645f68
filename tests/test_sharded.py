"""Sharded nodal pass (Section III-B dealing, Alg. 5 exchange).

CPU: two gloo ranks, each deciding its dealt range with the oracle, exchange
the new labels through `allgather_slices` and apply them; the result equals
the single-rank sweeps bit for bit.  GPU: two model replicas on one device
decide their ranges, trade them through sbp_get_pending / sbp_set_pending and
commit; and two gloo ranks, each with its own replica on the same device, run
`sharded_sweep` (decide, exchange on the host, commit).  Both equal
sbp_nodal_sweep over the whole graph.  The ranks' kernels never wait on one
another: the exchange is a host collective between whole sweeps."""

import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

from synth.dcsbm import dcsbm, perturb

SEED, BETA, SWEEPS = 11, 3.0, 3


def _graph():
    g = dcsbm(n=600, e=6000, n_blocks=6, gamma=2.5, kmin=1, kmax=80, ratio=4.0, seed=5)
    b0 = perturb(g.planted, g.n_blocks, 0.4, seed=6)
    return g, b0


def _relabelled(world):
    from paper_2305_18663_gb300.shard import dealt_order, relabel_edges

    g, b0 = _graph()
    deg = np.bincount(g.src, minlength=g.n) + np.bincount(g.dst, minlength=g.n)
    new_to_old, ranges = dealt_order(deg, world)
    src, dst = relabel_edges(g.src, g.dst, new_to_old)
    return g.n, g.n_blocks, src, dst, b0[new_to_old].astype(np.int32), ranges


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    import oracle as O
    from paper_2305_18663_gb300.shard import allgather_slices

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        n, B, src, dst, b0, ranges = _relabelled(world)
        m = O.Model(O.Graph(n, src, dst), B, b0)
        lo, hi = ranges[rank]
        for k in range(SWEEPS):
            d = m.nodal_decide(SEED, k, BETA, lo, hi)
            full = allgather_slices(torch.from_numpy(d.b_new[lo:hi].copy()), ranges)
            m.set_b(B, full.numpy())
        np.save(os.path.join(out_dir, f"b{rank}.npy"), m.assignment())
        # uneven slices, one of them empty
        uneven = [(0, 0), (0, 5)] if world == 2 else None
        if uneven:
            l, h = uneven[rank]
            got = allgather_slices(torch.arange(l, h, dtype=torch.int32) + 100, uneven)
            np.save(os.path.join(out_dir, f"u{rank}.npy"), got.numpy())
    finally:
        dist.destroy_process_group()


def test_dealt_order_is_a_permutation_with_contiguous_ranks():
    from paper_2305_18663_gb300.shard import deal_vertices, dealt_order

    rng = np.random.default_rng(3)
    deg = rng.integers(0, 50, 101)
    for world in (1, 2, 3, 5):
        new_to_old, ranges = dealt_order(deg, world)
        assert np.array_equal(np.sort(new_to_old), np.arange(deg.size))
        assert ranges[0][0] == 0 and ranges[-1][1] == deg.size
        for r, (lo, hi) in enumerate(ranges):
            assert np.array_equal(new_to_old[lo:hi], deal_vertices(deg, world, r))


def test_two_gloo_ranks_match_the_single_rank_sweeps(tmp_path):
    import oracle as O

    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    assert codes == [0, 0], codes

    n, B, src, dst, b0, _ = _relabelled(world)
    m = O.Model(O.Graph(n, src, dst), B, b0)
    moved = 0
    for k in range(SWEEPS):
        d = m.nodal_decide(SEED, k, BETA)
        moved += int((d.b_new != m.assignment()).sum())
        m.set_b(B, d.b_new)
    assert moved > 0
    want = m.assignment()
    for r in range(world):
        assert np.array_equal(np.load(tmp_path / f"b{r}.npy"), want)
        assert np.array_equal(np.load(tmp_path / f"u{r}.npy"), np.arange(100, 105, dtype=np.int32))


@pytest.mark.gpu
def test_two_replicas_exchange_pending_labels_on_one_gpu():
    import torch

    import paper_2305_18663_gb300 as P

    world = 2
    n, B, src, dst, b0, ranges = _relabelled(world)
    graph = P.Graph(n, src, dst)
    params = P.Params.default(seed=SEED, beta=BETA)
    dev = torch.device("cuda", 0)
    reps = [P.Model(graph, B, b0, params) for _ in range(world)]
    ref = P.Model(graph, B, b0, params)
    for k in range(SWEEPS):
        slices = []
        for r, m in enumerate(reps):
            lo, hi = ranges[r]
            P.sbp_nodal_decide(m.h, k, lo, hi)
            s = torch.empty(hi - lo, dtype=torch.int32, device=dev)
            P.sbp_get_pending(m.h, lo, hi, s)
            slices.append(s)
        full = torch.cat(slices)
        for r, m in enumerate(reps):
            if r == 0:
                P.sbp_set_pending(m.h, 0, n, full)  # device input
            else:
                P.sbp_set_pending(m.h, 0, n, full.cpu().numpy())  # host input
            P.sbp_commit(m.h)
        P.sbp_nodal_sweep(ref.h, k, 0, n)
    want = ref.assignment()
    for m in reps:
        assert np.array_equal(m.assignment(), want)
        assert m.dl() == ref.dl()
    # a host label out of range is refused before anything is written
    bad = np.full(3, B, np.int32)
    with pytest.raises(P.SbpError):
        P.sbp_set_pending(reps[0].h, 0, 3, bad)
    for m in reps + [ref]:
        m.close()


def _gather_main(rank, world, port, out_dir, ranges):
    import torch
    import torch.distributed as dist

    from paper_2305_18663_gb300.shard import allgather_slices

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        lo, hi = ranges[rank]
        got = allgather_slices(torch.arange(lo, hi, dtype=torch.int32) * 3 + 1, ranges)
        np.save(os.path.join(out_dir, f"g{rank}.npy"), got.numpy())
    finally:
        dist.destroy_process_group()


def test_three_gloo_ranks_gather_uneven_slices(tmp_path):
    world = 3
    ranges = [(0, 7), (7, 7), (7, 20)]  # the middle rank holds nothing
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_gather_main, args=(r, world, port, str(tmp_path), ranges)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    assert codes == [0, 0, 0], codes
    want = np.arange(0, 20, dtype=np.int32) * 3 + 1
    for r in range(world):
        assert np.array_equal(np.load(tmp_path / f"g{r}.npy"), want)


def _sharded_gpu_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    import paper_2305_18663_gb300 as P
    from paper_2305_18663_gb300.shard import sharded_sweep

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        P.load()
        n, B, src, dst, b0, ranges = _relabelled(world)
        m = P.Model(P.Graph(n, src, dst), B, b0, P.Params.default(seed=SEED, beta=BETA))
        accepted = 0
        for k in range(SWEEPS):
            accepted += sharded_sweep(m, k, ranges, stats=True).n_accepted
        np.save(os.path.join(out_dir, f"s{rank}.npy"), m.assignment())
        np.save(os.path.join(out_dir, f"dl{rank}.npy"), np.array([m.dl(), accepted], np.float64))
        m.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.gpu
def test_sharded_sweep_two_gloo_ranks_on_one_gpu(tmp_path):
    import torch

    import paper_2305_18663_gb300 as P

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_sharded_gpu_main, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    assert codes == [0, 0], codes
    n, B, src, dst, b0, _ = _relabelled(world)
    ref = P.Model(P.Graph(n, src, dst), B, b0, P.Params.default(seed=SEED, beta=BETA))
    accepted = 0
    for k in range(SWEEPS):
        accepted += P.sbp_nodal_sweep(ref.h, k, 0, n).n_accepted
    assert accepted > 0
    rank_accepted = 0
    for r in range(world):
        assert np.array_equal(np.load(tmp_path / f"s{r}.npy"), ref.assignment())
        dl, acc = np.load(tmp_path / f"dl{r}.npy")
        assert dl == ref.dl()
        rank_accepted += int(acc)  # each rank counts the moves of the range it decided
    assert rank_accepted == accepted
    ref.close()
