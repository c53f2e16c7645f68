#!/usr/bin/env python3
"""Benchmark of the SBP nodal sweep on one GB300 (or N replicas).

Metric: vertex proposals/s per nodal sweep = N / t_sweep, where a step is
one asynchronous-Gibbs nodal pass over all vertices (proposal, Delta DL,
Hastings test) plus the rebuild of M, block degrees and DL from the new
assignment.  Inputs are synthetic directed DCSBM graphs (seeded generator),
standing in for the paper's datasets.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--config dcsbm_1m] [--scale 1.0]

Prints one JSON line (rank 0).  Under torchrun every rank runs its own
replica on its own GPU (the path has no cross-GPU exchange on one box); the
timed region is bracketed by barriers and the slowest rank's time is used.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth.dcsbm import CONFIGS, make_config, perturb  # noqa: E402

METRIC = "vertex proposals/s per nodal sweep"
UNIT = "proposals/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# the translation unit of the decide-pass kernels (nodal.cu and what it includes)
DECIDE_SOURCES = ["paper_2305_18663_gb300/csrc/nodal.cu", "paper_2305_18663_gb300/csrc/nodal_dev.cuh",
                  "paper_2305_18663_gb300/csrc/common.cuh", "include/sbp.h"]


def code_only(text: str) -> str:
    """C/C++ source without comments and whitespace (so that edits of the
    documentation do not count as a change of the kernels)."""
    import re

    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return re.sub(r"\s+", "", text)


def sources_sha256() -> str:
    """Hash of the code the decide-pass kernels are compiled from."""
    import hashlib

    h = hashlib.sha256()
    for name in DECIDE_SOURCES:
        h.update(name.encode())
        with open(os.path.join(ROOT, name)) as f:
            h.update(code_only(f.read()).encode())
    return h.hexdigest()


def decide_traffic(m_form: str):
    """DRAM bytes of one decide pass from the committed ncu summary, when it
    was taken on the current decide-pass sources and this M form; else None."""
    path = os.path.join(ROOT, "profiles", "decide_traffic_dcsbm_1m.txt")
    try:
        kv = {}
        with open(path) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("sources_sha256") != sources_sha256() or kv.get("m_form") != m_form:
            return None
        return {"bytes": float(kv["dram_bytes_per_pass"]), "sweep": kv["sweep"],
                "algorithmic_bytes": float(kv["algorithmic_bytes_of_that_sweep"]),
                "streamed_bytes": float(kv["streamed_bytes_of_that_sweep"])}
    except (OSError, KeyError, ValueError):
        return None


def workload(name: str, scale: float, B: int | None = None):
    """The graph, the block count of the sweeps (the planted count unless
    given) and the start: planted labels with 30% of vertices reassigned
    uniformly over the B blocks."""
    g = make_config(name, seed=0, scale=scale)
    B = B or CONFIGS[name]["n_blocks"]
    b0 = perturb(g.planted, B, 0.3, seed=0)
    return g, B, b0


def describe(name, g, B, scale, m_form="dense"):
    c = CONFIGS[name]
    form = "sparse hashed M rows (CSR+CSC, per-row hash tables)" if m_form == "sparse" else "dense M"
    return {
        "workload": f"{name}: directed DCSBM N={g.n:,} E={g.m:,}, {B} planted {c['sizes']} blocks, "
        f"degree exponent {c['gamma']} clipped [{c['kmin']},{c['kmax']}], intra:inter {c['ratio']:g}:1, "
        f"nodal sweeps at B={B} from planted labels with 30% reassigned, {form}, beta=3",
        "m_form": m_form,
        "n": g.n,
        "e": g.m,
        "B": B,
        "scale": scale,
        "l2": "inputs larger than L2 (CSR out+in with offsets = %.0f MB > 129 MB)" % ((16 * g.m + 8 * (g.n + 1)) / 1e6),
    }


class Clocks:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.proc = None
        self.index = index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        rows = []
        for line in out.strip().splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 7:
                try:
                    rows.append((float(p[0]), float(p[1]), p[3:7]))
                except ValueError:
                    pass
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, x in enumerate(r) if x.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": reasons}


def algorithmic_bytes(n, m, B, move_edges, entries=0, sparse=False, nnz=0):
    """Per-sweep bytes the method has to move, each access counted at its
    element size, in three parts.

    streamed: offsets 8(N+1); labels read and written 8N; the proposal's
    edge and its block 8N; the rows of the vertices whose proposal differs
    from their block, with the block at each far end, 8 per edge end.
    lookups: the proposal's inverse-CDF search, 4 ceil(log2 L) per vertex
    (L = 2B prefix entries, or the mean row plus column length of the sparse
    rows); per distinct neighbour block of a moving vertex (entries) the
    four blockmodel counts (4 bytes each dense, 8 per hash probe sparse)
    and two block degrees (8); per moving vertex the 2x2 corner and four
    degrees.  rebuild (the apply step as a recount): adjacency 4E + both
    blocks 8E + edge sources 4E + zeroing and prefix of M 12 B^2.
    Returns (streamed + lookups, streamed, rebuild)."""
    import math

    streamed = 8 * (n + 1) + 8 * n + 8 * n + 8 * move_edges
    cell = 8 if sparse else 4
    L = max(2.0, 2.0 * nnz / max(B, 1)) if sparse else 2.0 * B
    search = 4 * math.ceil(math.log2(L)) * n
    lookups = search + entries * (4 * cell + 8)
    rebuild = 4 * m + 8 * m + 4 * m + 12 * B * B
    return streamed + lookups, streamed, rebuild


def dl_vs_fp64(P, torch, model, g, B, dev):
    """DL of the final state as the library holds it (exact fixed-point
    sums) against an FP64 evaluation of Eq. 2 from the same counts (the
    library's allocation-free FP64 reduction), as a relative difference."""
    if B > 4096:
        return None
    keys, cnt = model.coo()
    M = np.zeros(B * B, np.int32)
    M[keys] = cnt
    dout, din = model.degrees()
    Md = torch.from_numpy(M).to(dev)
    od = torch.from_numpy(dout).to(dev)
    idg = torch.from_numpy(din).to(dev)
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    P.sbp_dense_dl_noalloc(Md, B, od, idg, g.m, g.n, out, torch.cuda.current_stream(dev).cuda_stream)
    torch.cuda.synchronize(dev)
    dl64 = float(out.item())
    dl = model.dl()
    return {"dl": dl, "dl_fp64": dl64, "rel_error": abs(dl - dl64) / abs(dl64)}


def dense_max_b(args) -> int:
    """dense / auto: M held dense while B <= 4096, sparse hashed rows above
    (auto is the plain configuration's rule); sparse: per-row hashed sparse
    rows at every B (dense_max_B = 1)."""
    return 1 if args.m_form == "sparse" else 4096


def m_form_of(args, B) -> str:
    return "sparse" if args.m_form == "sparse" or B > 4096 else "dense"


def run_ours(args, rank, world, local_rank):
    import torch

    import paper_2305_18663_gb300 as P

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    P.load()
    g, B, b0 = workload(args.config, args.scale, args.B)
    m_form = m_form_of(args, B)
    stream = torch.cuda.current_stream(dev)
    graph = P.Graph(g.n, g.src, g.dst)
    params = P.Params.default(seed=args.seed, dense_max_B=dense_max_b(args), dl_fp32=1 if args.dl == "fp32" else 0,
                              hybrid_h=args.hybrid_h)
    model = P.Model(graph, B, b0, params, stream)

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    sweep_id = 0
    for _ in range(args.warmup):
        P.sbp_nodal_decide(model.h, sweep_id, 0, g.n)
        P.sbp_commit(model.h, stats=False)
        sweep_id += 1
    P.sbp_sync(model.h)
    torch.cuda.synchronize(dev)

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    clocks = Clocks(local_rank)
    barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    launches0 = P.sbp_kernel_launches()
    t_start.record(stream)
    for k in range(args.steps):
        ev[k][0].record(stream)
        P.sbp_nodal_decide(model.h, sweep_id, 0, g.n)
        ev[k][1].record(stream)
        P.sbp_commit(model.h, stats=False)
        ev[k][2].record(stream)
        sweep_id += 1
    t_end.record(stream)
    launches = P.sbp_kernel_launches() - launches0
    torch.cuda.synchronize(dev)
    P.sbp_sync(model.h)
    total_ms = t_start.elapsed_time(t_end)
    decide_ms = [e[0].elapsed_time(e[1]) for e in ev]
    commit_ms = [e[1].elapsed_time(e[2]) for e in ev]

    # The same chain again from the same start, with every sweep's
    # statistics read back (the mover edges and distinct neighbour blocks of
    # exactly the timed sweeps, and the first sweeps' heavy-move regime),
    # repeated until the clock sampler has seen the GPU for a while.
    first = []
    stats_of = {}
    t_clock0 = time.perf_counter()
    reps = 0
    while True:
        replay = P.Model(graph, B, b0, params, stream)
        for k in range(args.warmup + args.steps):
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            P.sbp_nodal_decide(replay.h, k, 0, g.n)
            e1.record(stream)
            rs = P.sbp_commit(replay.h, stats=True)
            e2.record(stream)
            if reps == 0:
                stats_of[k] = rs.as_dict()
                if k < 5:
                    torch.cuda.synchronize(dev)
                    first.append({"sweep": k, "decide_ms": e0.elapsed_time(e1), "commit_ms": e1.elapsed_time(e2),
                                  "n_moves": rs.n_moves, "n_accepted": rs.n_accepted,
                                  "n_move_edges": rs.n_move_edges, "n_entries": rs.n_entries,
                                  "n_recheck": rs.n_recheck})
        replay.close()
        reps += 1
        if time.perf_counter() - t_clock0 >= args.clock_window or reps >= 200:
            break
    torch.cuda.synchronize(dev)
    clock_window_s = time.perf_counter() - t_clock0
    ck = clocks.stop()

    if world > 1:
        import torch.distributed as dist

        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())

    # end to end through the C ABI with host buffers: upload b, sweep (with
    # stats read back), download b
    # pinned host buffers (page-locked: the copies run as DMA)
    host_b = torch.empty(g.n, dtype=torch.int32, pin_memory=True).numpy()
    host_b[:] = model.assignment()
    out_b = torch.empty(g.n, dtype=torch.int32, pin_memory=True).numpy()
    e2e_steps = max(3, min(args.steps, 10))
    barrier()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        P.sbp_set_assignment(model.h, B, host_b)
        P.sbp_nodal_sweep(model.h, sweep_id, 0, g.n, stats=True)
        P.sbp_get_assignment(model.h, out_b)
        sweep_id += 1
    e2e_s = time.perf_counter() - t0
    if world > 1:
        import torch.distributed as dist

        t = torch.tensor([e2e_s], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    st = P.sbp_nodal_sweep(model.h, sweep_id, 0, g.n, stats=True)
    precision = dl_vs_fp64(P, torch, model, g, B, dev)
    nnz = len(model.coo()[0]) if m_form == "sparse" else 0
    model.close()
    dense_comparison = None
    if args.m_form == "sparse" and B <= 4096:
        # the same sweeps with M held dense (the comparison form)
        dm = P.Model(graph, B, b0, P.Params.default(seed=args.seed, dense_max_B=4096, dl_fp32=params.dl_fp32), stream)
        for k in range(args.warmup):
            P.sbp_nodal_decide(dm.h, k, 0, g.n)
            P.sbp_commit(dm.h, stats=False)
        t0e = torch.cuda.Event(enable_timing=True)
        t1e = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        t0e.record(stream)
        for k in range(args.warmup, args.warmup + args.steps):
            P.sbp_nodal_decide(dm.h, k, 0, g.n)
            P.sbp_commit(dm.h, stats=False)
        t1e.record(stream)
        torch.cuda.synchronize(dev)
        dms = t0e.elapsed_time(t1e)
        dense_comparison = {"m_form": "dense", "value": g.n * args.steps / (dms * 1e-3), "unit": UNIT,
                            "ms_per_step": dms / args.steps}
        dm.close()

    res = None
    if rank == 0:
        hbm, hbm_kind = peaks()
        timed = [stats_of[k] for k in range(args.warmup, args.warmup + args.steps)]
        move_edges = statistics.mean(t["n_move_edges"] for t in timed)
        entries = statistics.mean(t["n_entries"] for t in timed)
        dec_b, dec_streamed, reb_b = algorithmic_bytes(g.n, g.m, B, move_edges, entries, m_form == "sparse", nnz)
        dec_avg = statistics.mean(decide_ms)
        achieved = dec_b / (dec_avg * 1e-3) / 1e9
        achieved_streamed = dec_streamed / (dec_avg * 1e-3) / 1e9
        traffic = decide_traffic(m_form) if args.config == "dcsbm_1m" and args.scale == 1.0 and args.B is None else None
        ms_step = total_ms / args.steps
        value = g.n * args.steps * world / (total_ms * 1e-3)
        if ck is not None:
            ck["window_s"] = clock_window_s
            ck["window"] = (f"the timed region, then the same {args.warmup + args.steps}-sweep chain replayed {reps} "
                            "times from the same start with statistics read back")
        res = {
            "metric": METRIC,
            "value": value,
            "unit": UNIT,
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms_step,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": ("fp32 terms + exact fp64 recheck" if args.dl == "fp32" else "f64 / fixed point") + ", int32 counts",
            "data": "synthetic (seeded directed DCSBM generator; the paper's graphs are not available)",
            "config": dict(describe(args.config, g, B, args.scale, m_form), hybrid_h=args.hybrid_h),
            "impl": "ours",
            "e2e": {"value": g.n * e2e_steps * world / e2e_s, "unit": UNIT,
                    # d2h: the labels, the pass counters (9 x 8), the two DLs (16), the
                    # status word (4) and the label check's read-back (4)
                    "h2d_bytes_per_step": 4 * g.n, "d2h_bytes_per_step": 4 * g.n + 96},
            "gpu_launches": launches,
            "roofline": {"kernel": "nodal decide pass (k_propose and the evaluation kernels of the three degree groups)",
                         "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "peak_kind": hbm_kind, "algorithmic_bytes": dec_b,
                         "algorithmic_bytes_note": ("per decide pass, mean over the timed sweeps (replayed with "
                                                    "statistics): streamed bytes plus the proposal search and the "
                                                    "blockmodel and degree lookups of every distinct neighbour block "
                                                    "of a moving vertex"),
                         "streamed_bytes": dec_streamed, "streamed_frac": achieved_streamed / hbm,
                         "sum_D_v": entries, "move_edge_ends": move_edges, "nnz": nnz or None,
                         "traffic": traffic["bytes"] if traffic else None,
                         "traffic_note": (f"ncu DRAM bytes of the decide pass of {traffic['sweep']}, whose "
                                          f"algorithmic bytes are {traffic['algorithmic_bytes']:.4g}") if traffic else None},
            "breakdown_ms": {"decide": dec_avg, "commit": statistics.mean(commit_ms),
                             "decide_min": min(decide_ms), "commit_bytes": reb_b},
            "first_sweeps": first,
            "last_sweep": st.as_dict(),
            "precision": precision,
            "dense_comparison": dense_comparison,
            "clocks": ck,
        }
    return res


def run_cpu_oracle(args, name, scale, steps=3, warmup=0, B=None):
    """The oracle, as it stands, on whole sweeps of the same chain: every
    vertex decided (OpenMP over vertices on all host threads), then M
    rebuilt from the new labels (single-threaded), from the same start as
    the GPU sweeps.  Returns proposals per second over the timed sweeps."""
    import oracle as O

    g, B, b0 = workload(name, scale, B)
    nt = O.max_threads()
    G = O.Graph(g.n, g.src, g.dst)
    om = O.Model(G, B, b0)
    times = []
    for k in range(warmup + steps):
        t0 = time.perf_counter()
        od = om.nodal_decide(args.seed, k, 3.0, nthreads=nt)
        om.set_b(B, od.b_new)
        dt = time.perf_counter() - t0
        if k >= warmup:
            times.append(dt)
    return {"value": g.n * steps / sum(times), "unit": UNIT, "cores": nt, "kind": "oracle",
            "sample": f"{steps} whole sweeps after {warmup} untimed (all {g.n:,} vertices decided on {nt} threads, "
                      f"then M rebuilt single-threaded) from the same start as the GPU sweeps",
            "seconds": sum(times)}, g, B


def nmi(a, b) -> float:
    """Normalised mutual information (arithmetic mean normalisation)."""
    a = np.asarray(a, np.int64)
    b = np.asarray(b, np.int64)
    n = a.size
    _, ai = np.unique(a, return_inverse=True)
    _, bi = np.unique(b, return_inverse=True)
    joint = np.zeros((ai.max() + 1, bi.max() + 1))
    np.add.at(joint, (ai, bi), 1.0)
    pa, pb, pj = joint.sum(1) / n, joint.sum(0) / n, joint / n
    nz = pj > 0
    mi = float(np.sum(pj[nz] * np.log(pj[nz] / np.outer(pa, pb)[nz])))
    ha = -float(np.sum(pa[pa > 0] * np.log(pa[pa > 0])))
    hb = -float(np.sum(pb[pb > 0] * np.log(pb[pb > 0])))
    return 2 * mi / (ha + hb) if ha + hb > 0 else 1.0


def run_partition(args):
    """Full run (golden-ratio search from B = N) on one graph: wall time
    through the C ABI with host buffers (graph upload included)."""
    import torch

    import paper_2305_18663_gb300 as P

    torch.cuda.set_device(0)
    P.load()
    g = make_config(args.config, seed=0, scale=args.scale)
    params = P.Params.default(seed=args.seed)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    graph = P.Graph(g.n, g.src, g.dst)
    b, B, dl, sweeps = graph.partition(params)
    wall = time.perf_counter() - t0
    c = CONFIGS[args.config]
    config = {"workload": f"{args.config}: full partition run (golden-ratio search over B from B = N = {g.n:,}, "
                          f"merge and MCMC phases, beta=3) of a directed DCSBM with E={g.m:,}, {c['n_blocks']} planted "
                          f"{c['sizes']} blocks, degree exponent {c['gamma']} clipped [{c['kmin']},{c['kmax']}], "
                          f"intra:inter {c['ratio']:g}:1; graph upload included",
              "n": g.n, "e": g.m, "scale": args.scale}
    res = {"metric": "full partition runs/s", "value": 1.0 / wall, "unit": "graphs/s", "n_gpus": 1, "steps": 1,
           "warmup": 0, "ms_per_step": wall * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "fp32 terms + exact fp64 recheck, int32 counts", "data": "synthetic", "config": config,
           "result": {"B": B, "dl": dl, "sweeps": sweeps, "nmi_vs_planted": nmi(b, g.planted),
                      "planted_B": CONFIGS[args.config]["n_blocks"]}}
    print(json.dumps(res))


def forms_summary(args, batch_every=64):
    """Small runs of the other forms, reported beside the sweep line: the
    full runs (golden-ratio search from B = N) of the 1k and 200k plain
    configurations, and every batch_every-th graph of the batching workload
    partitioned by one batch call against one sbp_partition per graph."""
    import torch

    import paper_2305_18663_gb300 as P
    from synth.dcsbm import batch_specs

    out = {}
    params = P.Params.default(seed=args.seed)
    for name in ("plain_1k", "plain_200k"):
        try:
            g = make_config(name, seed=0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            graph = P.Graph(g.n, g.src, g.dst)
            b, B, dl, sweeps = graph.partition(params)
            out["full_run_" + name] = {"seconds": time.perf_counter() - t0, "n": g.n, "e": g.m, "B": B, "dl": dl,
                                       "sweeps": sweeps, "nmi_vs_planted": nmi(b, g.planted),
                                       "planted_B": CONFIGS[name]["n_blocks"], "graph_upload_included": True}
        except Exception as e:  # reported, not fatal to the sweep line
            out["full_run_" + name] = {"error": str(e)}
    try:
        specs = batch_specs(4096, seed=args.seed)[::batch_every]
        graphs = [P.Graph(n, src, dst) for n, src, dst in gen_graphs(specs)]
        bp = P.Params.default(seed=args.seed, dense_max_B=P.BatchOptions.default().dense_max_B)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = P.partition_batch(graphs, bp)
        tb = time.perf_counter() - t0
        t0 = time.perf_counter()
        plain = [g.partition(bp) for g in graphs]
        tp = time.perf_counter() - t0
        equal = all(B == pB and dl == pdl and ns == pns and np.array_equal(b, pb)
                    for (b, B, dl, ns, _, _), (pb, pB, pdl, pns) in zip(res, plain))
        out["batch_sample"] = {"graphs": len(graphs), "of": 4096, "every": batch_every,
                               "batched_graphs_per_s": len(graphs) / tb, "plain_graphs_per_s": len(graphs) / tp,
                               "results_equal": equal, "options": "defaults"}
    except Exception as e:
        out["batch_sample"] = {"error": str(e)}
    return out


def _gen(spec):
    from synth.dcsbm import dcsbm

    g = dcsbm(**spec)
    return g.n, g.src, g.dst


def gen_graphs(specs, procs=None):
    """Draws the graphs of specs (a process pool, spawned: no CUDA in it)."""
    import multiprocessing as mp

    procs = procs or min(16, os.cpu_count() or 1)
    if procs <= 1 or len(specs) < 4:
        return [_gen(s) for s in specs]
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(_gen, specs, chunksize=max(1, len(specs) // (4 * procs)))


def run_batch(args):
    """The batching form: many small uneven graphs partitioned (full
    golden-ratio runs) by one batch call against one sbp_partition call per
    graph, on the same graphs, with every result compared."""
    import torch

    import paper_2305_18663_gb300 as P
    from synth.dcsbm import batch_specs

    torch.cuda.set_device(0)
    P.load()
    specs = batch_specs(args.batch_total, seed=args.seed)
    stride = max(1, args.batch_total // args.batch_count)
    chosen = specs[::stride][: args.batch_count]
    t0 = time.perf_counter()
    raw = gen_graphs(chosen)
    t_gen = time.perf_counter() - t0
    graphs = [P.Graph(n, src, dst) for n, src, dst in raw]
    opts = P.BatchOptions.default(**{"workers": args.batch_workers, **json.loads(args.options)})
    tuned = None
    if args.autotune > 0:
        # the autotuner on a sample of the same graphs, before the timed call
        t0 = time.perf_counter()
        opts, rate, trials = P.autotune_batch(graphs, P.Params.default(seed=args.seed), args.autotune, opts)
        tuned = {"sample": min(args.autotune, len(graphs)), "trials": trials, "seconds": time.perf_counter() - t0,
                 "sample_graphs_per_s": rate,
                 "options": {f: getattr(opts, f) for f, _ in P.BatchOptions._fields_}}
    params = P.Params.default(seed=args.seed, dense_max_B=opts.dense_max_B)
    torch.cuda.synchronize()
    bstats = P.BatchStats()
    t0 = time.perf_counter()
    out = P.partition_batch(graphs, params, opts, bstats)
    t_batch = time.perf_counter() - t0
    t0 = time.perf_counter()
    plain = [g.partition(params) for g in graphs]
    t_plain = time.perf_counter() - t0
    mismatch = sum(1 for (b, B, dl, ns, _, _), (pb, pB, pdl, pns) in zip(out, plain)
                   if not (B == pB and dl == pdl and ns == pns and np.array_equal(b, pb)))
    done = np.array([o[5] for o in out])
    nv = sum(g.n for g in graphs)
    ne = sum(g.m for g in graphs)
    res = {"metric": "graphs/s, batched vs plain (full partition runs)", "value": len(graphs) / t_batch,
           "unit": "graphs/s", "n_gpus": 1, "higher_is_better": True, "impl": "ours",
           "plain": {"value": len(graphs) / t_plain, "unit": "graphs/s", "seconds": t_plain},
           "batched_seconds": t_batch, "speedup_vs_plain": t_plain / t_batch, "batch_stats": bstats.as_dict(),
           "phases_batched_share": bstats.phases_batched / max(1, bstats.phases_batched + bstats.phases_per_graph),
           "autotune": tuned,
           "results_equal": mismatch == 0, "mismatches": mismatch,
           "completion_s": {"p50": float(np.percentile(done, 50)), "p99": float(np.percentile(done, 99))},
           "dtype": "f32 terms, exact recheck", "data": "synthetic",
           "config": {"workload": f"{len(graphs)} of {args.batch_total} directed DCSBM graphs (every {stride}th), "
                                  "N log-uniform [500, 50000], mean out-degree uniform [8, 32], "
                                  "planted B = round(sqrt(N)/2), degree exponent 2.5 on [1, 100], intra:inter 4:1",
                      "graphs": len(graphs), "vertices": nv, "edges": ne, "workers": opts.workers,
                      "max_B": opts.max_B, "max_n": opts.max_n, "dense_max_B": opts.dense_max_B,
                      "generation_s": t_gen}}
    print(json.dumps(res))


def run_serve(args):
    """The serving form: Poisson arrivals of partition requests (N
    log-uniform in [1000, 2M], mean out-degree 16) fed to a server while it
    runs, at several rates.  Latency = result time - arrival time.  The plain
    comparison serves the same arrivals one request at a time in arrival
    order (FIFO), with each request's own measured sbp_partition time."""
    import threading

    import torch

    import paper_2305_18663_gb300 as P
    from synth.dcsbm import serving_specs

    torch.cuda.set_device(0)
    P.load()
    specs = serving_specs(args.serve_count, seed=args.seed, n_hi=args.serve_n_hi)
    t0 = time.perf_counter()
    raw = gen_graphs(specs)
    t_gen = time.perf_counter() - t0
    graphs = [P.Graph(n, src, dst) for n, src, dst in raw]
    params = P.Params.default(seed=args.seed)
    # plain: each request alone, timed
    plain, service = [], []
    for g in graphs:
        t0 = time.perf_counter()
        plain.append(g.partition(params))
        service.append(time.perf_counter() - t0)
    rng = np.random.Generator(np.random.Philox(args.seed + 11))
    rates = [float(r) for r in args.serve_rates.split(",")]
    points = []
    equal = True
    for rate in rates:
        gaps = rng.exponential(1.0 / rate, len(graphs))
        arrive = np.cumsum(gaps) - gaps[0]
        srv = P.Server(params, P.BatchOptions.default(**json.loads(args.options)))
        rids = [None] * len(graphs)
        base = time.perf_counter()

        def feed():
            for i, g in enumerate(graphs):
                delay = arrive[i] - (time.perf_counter() - base)
                if delay > 0:
                    time.sleep(delay)
                rids[i] = srv.submit(g)

        th = threading.Thread(target=feed)
        th.start()
        th.join()
        outs = [srv.wait(r) for r in rids]
        srv.close()
        lat = np.array([o[6] - o[4] for o in outs])
        span = max(o[6] for o in outs) - min(o[4] for o in outs)
        for o, pl in zip(outs, plain):
            if not (o[1] == pl[1] and o[2] == pl[2] and o[3] == pl[3] and np.array_equal(o[0], pl[0])):
                equal = False
        # plain FIFO with the measured service times
        fin, t = [], 0.0
        for a, sv in zip(arrive, service):
            t = max(t, a) + sv
            fin.append(t)
        plat = np.array(fin) - arrive
        points.append({"rate_req_s": rate,
                       "served": {"graphs_per_s": len(graphs) / span, "p50_s": float(np.percentile(lat, 50)),
                                  "p99_s": float(np.percentile(lat, 99))},
                       "plain_fifo": {"graphs_per_s": len(graphs) / (fin[-1] - arrive[0]),
                                      "p50_s": float(np.percentile(plat, 50)), "p99_s": float(np.percentile(plat, 99))}})
    top = points[-1]
    res = {"metric": "graphs/s and p99 latency, served (continuous batching) vs plain FIFO",
           "value": top["served"]["graphs_per_s"], "unit": "graphs/s", "n_gpus": 1, "higher_is_better": True,
           "impl": "ours", "p99_s": top["served"]["p99_s"], "points": points, "results_equal": equal,
           "dtype": "f32 terms, exact recheck", "data": "synthetic",
           "config": {"workload": f"{len(graphs)} requests, directed DCSBM, N log-uniform [1000, {args.serve_n_hi}], "
                                  "mean out-degree 16, planted B = round(sqrt(N)/2), degree exponent 2.3 on [1, 1000], "
                                  "intra:inter 3:1, Poisson arrivals",
                      "requests": len(graphs), "vertices": sum(g.n for g in graphs), "edges": sum(g.m for g in graphs),
                      "rates": rates, "generation_s": t_gen, "plain_service_s": float(sum(service))}}
    print(json.dumps(res))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="dcsbm_1m", choices=list(CONFIGS))
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--oracle-sweeps", type=int, default=3, help="whole oracle sweeps timed for cpu_baseline")
    ap.add_argument("--B", type=int, default=None,
                    help="blocks of the timed sweeps (default: the planted count); the start is the planted "
                         "labels with 30%% of vertices reassigned uniformly over B blocks")
    ap.add_argument("--clock-window", type=float, default=2.0,
                    help="seconds of replayed sweeps (same chain, same start) the clock sampler also covers")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the small full-run and batch runs reported under 'forms'")
    ap.add_argument("--mode", default="sweep", choices=["sweep", "partition", "batch", "serve"])
    ap.add_argument("--serve-count", type=int, default=24)
    ap.add_argument("--serve-n-hi", type=int, default=2_000_000)
    ap.add_argument("--serve-rates", default="2,20,200")
    ap.add_argument("--batch-total", type=int, default=4096, help="graphs of the batching workload")
    ap.add_argument("--batch-count", type=int, default=4096,
                    help="graphs actually run (all of them by default; fewer: an evenly strided subset)")
    ap.add_argument("--batch-workers", type=int, default=32)
    ap.add_argument("--options", default="{}",
                    help="batch and serve modes: batch options over the defaults, as JSON (e.g. '{\"max_n\": 4096}')")
    ap.add_argument("--autotune", type=int, default=0,
                    help="batch mode: graphs in the autotuner's sample (0: default options)")
    ap.add_argument("--m-form", default="sparse", choices=["dense", "sparse", "auto"],
                    help="sparse: hashed sparse rows at every B (the M form of the 1M-vertex precision "
                         "configuration; a dense run of the same sweeps is reported beside it); dense or auto: "
                         "M dense while B <= 4096, sparse rows above")
    ap.add_argument("--hybrid-h", type=int, default=0,
                    help="hybrid pass: this many highest-degree vertices sequentially (dense M only)")
    ap.add_argument("--dl", default="fp32", choices=["fp32", "exact"],
                    help="fp32: x ln x terms in FP32 with the exact recheck inside the error band; "
                         "exact: fixed-point/FP64 terms for every proposal")
    args = ap.parse_args()
    if args.mode == "partition":
        run_partition(args)
        return
    if args.mode == "batch":
        run_batch(args)
        return
    if args.mode == "serve":
        run_serve(args)
        return

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))

    if args.impl == "reference":
        if rank != 0:
            return
        cb, g, B = run_cpu_oracle(args, args.config, args.scale, steps=args.steps, warmup=args.warmup, B=args.B)
        res = {"metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": 1e3 * g.n / cb["value"], "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": dict(describe(args.config, g, B, args.scale, m_form_of(args, B)), hybrid_h=args.hybrid_h),
               "impl": "reference", "cpu_baseline": cb,
               "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(res))
        return

    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    res = run_ours(args, rank, world, local_rank)
    if rank == 0:
        if world == 1 and not args.no_forms:
            res["forms"] = forms_summary(args)
        if not args.no_cpu_baseline:
            cb, _, _ = run_cpu_oracle(args, args.config, args.scale, steps=args.oracle_sweeps, B=args.B)
            res["cpu_baseline"] = cb
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
