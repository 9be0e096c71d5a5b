#!/usr/bin/env python
"""Benchmark: queries/sec at recall@10 >= 0.95 on one GB300 (and N replicas).

One step = one batched search (Algorithm 1 per query, all rows of the query
path: rotation, quantization, beam search with implicit re-ranking) over one
batch of the workload's size (10,000 queries at 1M x 128), at the smallest
beam size ef of the sweep whose recall@10 on the first batch reaches 0.95.
The job draws a pool of `--batches` distinct batches (one seeded query
stream) and step s searches batch s mod batches, so no two steps in flight
share a query.  Inputs are resident in HBM before the timed region.  Each
step is one CUDA graph (rotation and search; plus the planning kernel
when k differs per query); the job replays K steps back to back
alternating over three streams (more for batches of a few hundred
queries; the index is larger than L2, so no flush between them), so one
step's tail overlaps the next steps' start.
`step_isolated_ms` is one step alone, L2 flushed before it.  The sweep's
`qps_at_recall` is timed the same way (distinct batches, three streams).
`e2e` repeats the job through the public host-to-host API (pinned H2D of
each step's queries, D2H of ids and distances inside the timed region).

Multi-GPU: queries are independent, so N ranks are N replicas, each with
its own index copy and its own query pool (weak scaling, no collective on
the data path); value = all ranks' queries / the slowest rank's time.

--impl reference times the CPU oracle (oracle/, single-threaded C per query,
run on all host cores) on bounded samples of the same batches, at the same
ef; the index and the ground truth are made beforehand by a separate
process, so the timed process loads no GPU library.
--profile runs two searches of the first batch at --ef (a warm-up and the
one to capture under ncu) and exits.
"""

from __future__ import annotations

import argparse
import concurrent.futures as cf
import hashlib
import json
import os
import pathlib
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = pathlib.Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

from paper_2411_12229_gb300 import synth  # noqa: E402

METRIC = "queries/sec at recall@10>=0.95"
UNIT = "queries/s"


def log(*a):
    print("[bench]", *a, file=sys.stderr, flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched-1m-d128", choices=list(synth.WORKLOADS))
    ap.add_argument("--n", type=int, default=0, help="override N (smaller runs)")
    ap.add_argument("--nq", type=int, default=0, help="override the query count")
    ap.add_argument("--cache", default=os.environ.get("SQG_CACHE", "/tmp/sqg_cache"))
    ap.add_argument("--target", type=float, default=0.95)
    ap.add_argument("--build-iters", type=int, default=3)
    ap.add_argument("--ef-build", type=int, default=400, help="index build: candidate-search beam (the paper's EF)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--ef", type=int, default=0, help="fixed ef: skip the sweep (profiling runs)")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-stop", action="store_true", help="skip the learned-stop comparison")
    ap.add_argument("--stop-train", type=int, default=0,
                    help="training queries for the learned stop (0: the workload's, else 20,000)")
    ap.add_argument("--rotation", default="dense", choices=["dense", "fjlt"],
                    help="index rotation: dense P^-1, or the fast JLT (Sec. 3.1.4; data padded to a power of 2)")
    ap.add_argument("--metric", default="l2", choices=["l2", "cosine"],
                    help="index metric: squared Euclidean, or cosine similarity (unit vectors; the library "
                         "normalizes every query, Sec. 3)")
    ap.add_argument("--graph", default="regular", choices=["regular", "irregular"],
                    help="index graph: degree-aligned by the angle rule, or the w/o GR ablation (Sec. 5) "
                         "with unused slots left empty")
    ap.add_argument("--prep", action="store_true",
                    help="time query preparation alone (rotation + 4-bit quantization), CUDA vs tensor cores")
    ap.add_argument("--batches", type=int, default=20,
                    help="distinct query batches in the job's pool (step s searches batch s mod batches)")
    ap.add_argument("--profile", action="store_true",
                    help="two searches of the first batch at --ef (warm-up, then the one ncu captures); no timing")
    ap.add_argument("--build-only", action="store_true",
                    help="make the index and the ground truth of the pool, then exit")
    return ap.parse_args()


def workload(args):
    w = synth.WORKLOADS[args.workload]
    if args.n:
        w = synth.small(w, args.n, w.n_queries)
    if args.nq:
        w = w.with_(n_queries=args.nq)
    return w


def cache_paths(args, w):
    c = pathlib.Path(args.cache)
    c.mkdir(parents=True, exist_ok=True)
    tag = f"{w.name}-n{w.n}-R{w.degree}-it{args.build_iters}-ef{args.ef_build}"
    if args.metric != "l2":
        tag += f"-{args.metric}"
    gt = c / f"{tag}-gt-q{w.n_queries}"  # the ground truth depends on neither the rotation nor the graph
    if args.rotation != "dense":
        tag += f"-{args.rotation}"
    if args.graph != "regular":
        tag += f"-{args.graph}"
    return c / f"{tag}.sqg", gt


def ensure_index(args, w, device, rank):
    """Build the index once (Algorithm 2 on the GPU) and the exact ground
    truth; cached on disk for the other ranks and later runs."""
    from paper_2411_12229_gb300 import eval as E
    from paper_2411_12229_gb300 import index_builder as ib
    idx, gtp = cache_paths(args, w)
    if rank == 0 and not idx.exists():
        t = time.time()
        base = synth.base(w)
        log(f"building {idx.name}: n={w.n} d={w.d} R={w.degree}")
        info = ib.build_index(str(idx) + ".part", base, w.degree, device=device, init="random",
                              iterations=args.build_iters, ef_build=args.ef_build, cand_k=2 * w.degree,
                              rotation=args.rotation, metric=args.metric, regular=args.graph == "regular",
                              log=log)
        os.replace(str(idx) + ".part", idx)
        secs = time.time() - t
        log(f"built in {secs:.1f}s {info['iterations'][-1]}")
        pathlib.Path(str(idx) + ".build.json").write_text(json.dumps(
            {"seconds": round(secs, 1), "iterations": args.build_iters, "ef_build": args.ef_build,
             "last_iteration": {k: (float(v) if isinstance(v, (int, float, np.floating, np.integer)) else str(v))
                                for k, v in info["iterations"][-1].items()}}))
    return idx, gtp


def build_record(idx):
    """The index build's wall time, if this cache built it."""
    p = pathlib.Path(str(idx) + ".build.json")
    return json.loads(p.read_text()) if p.exists() else None


def ground_truth(args, w, gtp, queries, device, world):
    from paper_2411_12229_gb300 import eval as E
    f = pathlib.Path(f"{gtp}-w{world}.npz")
    if f.exists():
        z = np.load(f)
        return z["ids"], z["dists"]
    t = time.time()
    base = synth.base(w)
    if args.metric == "cosine":  # the most similar = the nearest between unit vectors
        from paper_2411_12229_gb300 import index_builder as ib
        base, queries = ib.unit_rows(base), ib.unit_rows(queries)
    ids, dd = E.ground_truth(base, queries, 100 if w.mixed_k else 10, device=device)
    np.savez(f, ids=ids, dists=dd)
    log(f"ground truth in {time.time() - t:.1f}s")
    return ids, dd


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={device}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in pathlib.Path(self.f.name).read_text().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_digest() -> str:
    """Digest of the search kernel's sources and of its launch planning."""
    h = hashlib.sha256()
    csrc = ROOT / "paper_2411_12229_gb300" / "csrc"
    for p in sorted(list(csrc.glob("search*")) + [csrc / "sqg_api.cu"]):
        h.update(p.read_bytes())
    return h.hexdigest()[:16]


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        z = json.loads(p.read_text())
        return float(z["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def traffic_record(workload_name, ef, metric="l2", rotation="dense", graph="regular"):
    """DRAM bytes per launch of the search kernel from a committed ncu
    summary of the same launch (workload, index metric, rotation, graph and
    ef), used only while the kernel source is unchanged since."""
    p = ROOT / "profiles" / "search_kernel_traffic.json"
    if not p.exists():
        return None
    z = json.loads(p.read_text())
    if (z.get("kernel_digest") != kernel_digest() or z.get("workload") != workload_name or z.get("ef") != ef
            or z.get("metric", "l2") != metric or z.get("rotation", "dense") != rotation
            or z.get("graph", "regular") != graph):
        return None
    return z


def run_oracle(idx_path, queries, k, ef, seconds, threads, max_queries):
    """The oracle as it stands, one query per task on `threads` host
    threads (ctypes releases the GIL), for about `seconds`."""
    from oracle import oracle
    O = oracle.Index(idx_path)
    done, ids = 0, {}
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(threads) as ex:
        it = iter(range(min(max_queries, queries.shape[0])))
        futs = {}
        for _ in range(threads * 2):
            i = next(it, None)
            if i is not None:
                futs[ex.submit(O.search, queries[i], k, ef)] = i
        while futs:
            fin, _ = cf.wait(futs, return_when=cf.FIRST_COMPLETED)
            for f in fin:
                ids[futs.pop(f)] = f.result()[0]
                done += 1
                if time.perf_counter() - t0 < seconds:
                    i = next(it, None)
                    if i is not None:
                        futs[ex.submit(O.search, queries[i], k, ef)] = i
    el = time.perf_counter() - t0
    O.close()
    return done, el, ids


def replica_queries(w, rank: int, world: int, batches: int = 1) -> np.ndarray:
    """Rank `rank`'s own pool of `batches` batches of nq queries: rows
    [rank*B*nq, (rank+1)*B*nq) of one seeded query stream, so the N replicas
    search disjoint pools (weak scaling) and no two batches share a query."""
    per = w.n_queries * batches
    allq = synth.queries(w, per * world)
    return np.ascontiguousarray(allq[rank * per:(rank + 1) * per])


def aggregate_replicas(local_ms, nq: int, world: int, dist, device):
    """Max over ranks of each per-step time (ms), and the whole-job rate:
    all ranks' queries divided by the slowest rank's step time."""
    import torch
    t = torch.tensor(local_ms, dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    worst = [float(x) for x in t.tolist()]
    return worst, [world * nq / (m / 1e3) for m in worst]


def learned_stop_comparison(args, w, ix, pool_d, gt_ids, sweep, ef_sel, device, nq, nb):
    """The learned stop (not in the paper) against the plain fixed-ef search
    at equal recall, both timed like the headline (captured batched
    searches over distinct batches on three streams).

    The network is trained on the GPU from traces of separate training
    queries with the label the stop is built for (the result already holds
    the true top-10) or with "final" (it holds what the search at the cap
    ends with).  Variants: evaluation every 8 or 16 hops, fixed-ef caps from
    the plain operating point up to 1.5x, for the target recall and for
    0.99; each picks its threshold on held-out training queries, then runs
    the test batches at a few thresholds; the plain frontier is the sweep.
    Reported per target recall: the stop's best QPS among points reaching
    it, beside the first plain ef reaching it, and the ratio against the
    plain frontier interpolated to the stop's own recall."""
    from paper_2411_12229_gb300 import eval as E
    from paper_2411_12229_gb300 import learned_stop as L
    t0 = time.time()
    ntrain = args.stop_train or w.n_train or 20000
    tq = synth.train_queries(w, ntrain)
    if ix.d != tq.shape[1]:
        tq = np.ascontiguousarray(np.pad(tq, ((0, 0), (0, ix.d - tq.shape[1]))))
    tg, _ = E.ground_truth(synth.base(w), tq[:, :w.d], 10, device=device)
    nbe = min(nb, 4)  # test batches the comparison runs
    rows, models = [], {}

    def caps_for(ef0):
        # fixed-ef caps from the plain operating point up to 1.5x; where that
        # point runs in the compact kernel, caps stay in its range (ef <= 128,
        # for d <= 256 ef <= 256)
        cs = {ef0, int(round(1.25 * ef0)), int(round(1.5 * ef0))}
        cmax = COMPACT_MAX_EF_SMALL_D if ix.d <= 256 else COMPACT_MAX_EF
        return sorted({min(c, cmax) for c in cs} if ef0 <= cmax else cs)

    # two operating points: the target recall (thresholds chosen for it) and
    # recall 0.99, where the plain search's fixed ef costs the most
    ef99 = next((x["ef"] for x in sweep if x["recall"] >= 0.99), None)
    groups = [(args.target, caps_for(ef_sel))] + ([(0.99, caps_for(ef99))] if ef99 and ef99 != ef_sel else [])
    # label "all": the result holds the true top-10 (the stop's stated
    # target); "final": it holds as many true ids as the traced search at
    # the cap ends with (no later gain), which states that fact directly
    for target, caps in groups:
        for label in ("all", "final"):
            for every in (8, 16):
                for cap in caps:
                    model = L.fit(ix, tq, tg, 10, cap, target, every=every, steps=3000, label=label)
                    name = f"t{target}_{label}_every{every}_cap{cap}"
                    models[name] = {"threshold": model.logit, "positive_rows": round(model.info["positive"], 4)}
                    for thr in (model.logit - 1.0, model.logit - 0.5, model.logit, model.logit + 1.0):
                        kw = dict(stop_mlp=model.params, stop_logit=thr, stop_every=every)
                        r = stop_point(ix, pool_d, gt_ids, nq, nbe, cap, kw)
                        rows.append({"target": target, "label": label, "every": every, "ef_cap": cap, "logit": thr,
                                     **r})
    caps = sorted({c for _, cs in groups for c in cs})
    # the plain frontier on the same test batches (recall over the first 4)
    plain = {t: next((x for x in sweep if x["recall_4"] >= t), None) for t in (0.90, 0.95, 0.99)}
    # what a perfect stop could save at each cap (first expansion holding the
    # true top-10, from traces), and what evaluating the network costs (a
    # threshold it never reaches: the same expansions as the plain search)
    test_q = pool_d[:nq].cpu().numpy()
    bound = [L.perfect_stop(ix, test_q, gt_ids[:nq], 10, cap) for cap in caps]
    m0 = L.fit(ix, tq, tg, 10, ef_sel, args.target, every=8, steps=1000, label="all")
    overhead = {}
    for every in (4, 8, 16):
        r = stop_point(ix, pool_d, gt_ids, nq, nbe, ef_sel, dict(stop_mlp=m0.params, stop_logit=1e30,
                                                                  stop_every=every))
        pl = next(x for x in sweep if x["ef"] == ef_sel)
        overhead[str(every)] = round(1.0 - r["qps"] / pl["qps"], 4)
    # the plain frontier between its sweep points (QPS linear in recall)
    front = sorted((x["recall_4"], x["qps"]) for x in sweep)

    def plain_qps_at(rec):
        for (r0, q0), (r1, q1) in zip(front, front[1:]):
            if r0 <= rec <= r1:
                return q0 + (q1 - q0) * (rec - r0) / max(r1 - r0, 1e-9)
        return None
    at = {}
    for t in (0.90, 0.95, 0.99):
        ok = [x for x in rows if x["recall"] >= t]
        best = max(ok, key=lambda x: x["qps"]) if ok else None
        pl = plain[t]
        fq = plain_qps_at(best["recall"]) if best else None
        at[str(t)] = {"stop": best, "plain": {"ef": pl["ef"], "recall": pl["recall_4"], "qps": pl["qps"],
                                              "hops": pl["hops"]} if pl else None,
                      "qps_ratio": round(best["qps"] / pl["qps"], 4) if best and pl else None,
                      "qps_ratio_vs_frontier_at_its_recall": round(best["qps"] / fq, 4) if fq else None}
    log(f"learned stop in {time.time() - t0:.1f}s: {at}")
    return {"labels": {"all": "the result holds the true top-10",
                       "final": "the result holds what the search at the cap ends with"},
            "train_queries": int(ntrain), "variants": models,
            "perfect_stop_bound": bound, "evaluation_overhead_by_period": overhead,
            "timing": f"graph-captured searches of {nbe} distinct batches of {nq}, {job_streams(nq)} streams (as the headline)",
            "points": rows, "at_recall": at, "qps_ratio_vs_plain": at["0.95"]["qps_ratio"]}


def stop_point(ix, pool_d, gt_ids, nq, nbe, ef, kw):
    """Recall over nbe batches, mean expansions and job QPS of one search
    configuration (graph per batch, three streams)."""
    from paper_2411_12229_gb300 import eval as E
    from paper_2411_12229_gb300.autotune import GraphSearch
    gs, hops = [], []
    for b in range(nbe):
        g = GraphSearch(ix, nq, 10, ef, max_k=10, max_ef=ef, **kw)
        g.q.copy_(pool_d[b * nq:(b + 1) * nq])
        gs.append(g)
        _, _, st = ix.search(pool_d[b * nq:(b + 1) * nq], 10, ef, stats=True, **kw)
        hops.append(st[:, 0].float().mean().item())
    for _ in range(3):
        for g in gs:
            g.graph.replay()
    ms = time_job(gs, 2 * nbe)
    ids = np.concatenate([g.ids.view(nq, 10).cpu().numpy() for g in gs])
    rec = E.recall(ids, gt_ids[:nbe * nq], 10)
    return {"recall": round(rec, 4), "qps": round(nq / (ms / 1e3)), "hops": round(float(np.mean(hops)), 2)}


L2_BYTES = 129_000_000  # GB300 L2, 129 MB
COMPACT_MAX_EF = 128  # the largest beam the compact search kernel takes (sqg_search_params.kernel)
COMPACT_MAX_EF_SMALL_D = 256  # ... and for d <= 256


def l2_note(ix, flushed: str) -> str:
    """How the job's steps stand to the L2: the index larger than it (no
    flush needed between steps) or resident in it (the small workload)."""
    size = ix.n * ix.block_bytes
    where = "larger than L2" if size > L2_BYTES else "fits in L2 (L2-resident by design)"
    return f"index ({size / 1e9:.2f} GB) {where}, no flush between job steps; {flushed}"


def job_streams(nq: int) -> int:
    """Streams the job's steps alternate over: 3 for batches of thousands of
    queries (1 / 2 / 3 / 4 streams: 0.310 / 0.223 / 0.214 / 0.214 ms per
    1M x 128 step of 10,000), more for small batches, whose single launch
    occupies a fraction of the GPU's resident warps (16 for 200 queries)."""
    return min(16, max(3, 8000 // max(nq, 1)))


def e2e_depth(nq: int) -> int:
    """Slots (streams) of the end-to-end host pipeline: one more than the
    device job's streams for batches of thousands, since each slot also
    holds its batch's copies (1M x 128, 10k batches: 45.9 / 47.3 M q/s with
    3 / 4 slots)."""
    return max(4, job_streams(nq))


def time_job(graphs, steps: int, nstreams: int | None = None) -> float:
    """Device ms per step of `steps` steps back to back: step s replays
    graphs[s % len(graphs)] (each graph owns its query batch and buffers)
    on stream s % nstreams, bracketed by events on the launching stream."""
    import torch
    nstreams = nstreams or job_streams(graphs[0].q.shape[0])
    cur = torch.cuda.current_stream()
    streams = [torch.cuda.Stream() for _ in range(min(nstreams, len(graphs)))]
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(cur)
    for st in streams:
        st.wait_stream(cur)
    for s in range(steps):
        with torch.cuda.stream(streams[s % len(streams)]):
            graphs[s % len(graphs)].graph.replay()
    for st in streams:
        cur.wait_stream(st)
    b.record(cur)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def isolated_steps(graph, steps: int, flush) -> float:
    """Mean device ms of one step alone, L2 flushed before it."""
    import torch
    ms = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        graph.graph.replay()
        b.record()
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return float(np.mean(ms))


def launches_per_step(d: int, metric: str = "l2", ragged: bool = False) -> int:
    """Library kernels per search call: rotation (tensor cores plus the
    exact quantization from d = 512 up, else one CUDA-core kernel), search;
    the planning kernel when k differs per query (ragged outputs); on a
    cosine index also the query normalization."""
    return (3 if d >= 512 else 2) + ragged + (metric == "cosine")


def bench_mixed(args, w, ix, pool_d, pool, gt_ids, rank, world, dist, local, nb):
    """Batches with per-query k and ef (the persistent work-queue form):
    autotune the launch knobs on the first batch, then time the job over nb
    distinct batches (each with its own k and ef draws); recall per k group.
    Also a fixed-ef sweep of the k = 10 queries, which shows the beam the
    k = 10 group would need for recall@10 >= 0.95 on this graph."""
    import torch

    from paper_2411_12229_gb300 import autotune
    from paper_2411_12229_gb300 import eval as E
    nq = w.n_queries
    kq, efq = synth.query_k_ef(w, nq * nb)
    max_k, max_ef = int(kq.max()), int(efq.max())
    q0 = pool_d[:nq]
    kt0, et0 = torch.from_numpy(kq[:nq]).cuda(), torch.from_numpy(efq[:nq]).cuda()
    tune = autotune.autotune(ix, q0, kt0, et0, reps=3, knobs=None, save=False)
    knobs = tune["best"]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    graphs = []
    for b in range(nb):
        sl = slice(b * nq, (b + 1) * nq)
        g = autotune.GraphSearch(ix, nq, kq[sl], efq[sl], max_k=max_k, max_ef=max_ef, **knobs)
        g.q.copy_(pool_d[sl])
        graphs.append(g)
    for _ in range(max(3, args.warmup)):
        for g in graphs:
            g.graph.replay()
    iso_ms = isolated_steps(graphs[0], args.steps, flush)
    clocks = Clocks(local)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms_local = time_job(graphs, args.steps)
    if dist:
        dist.barrier()
    clk = clocks.stop()
    (ms,), (value,) = aggregate_replicas([ms_local], nq, world, dist, "cuda")  # slowest rank
    total0 = int(kq[:nq].sum())
    out = (torch.empty(total0, dtype=torch.int32, device="cuda"), torch.empty(total0, device="cuda"))
    _, _, st = ix.search(q0, kt0, et0, out=out, stats=True, max_k=max_k, max_ef=max_ef, **knobs)
    if not torch.equal(out[0], graphs[0].ids):
        raise RuntimeError("graph replay and direct search disagree")
    used = min(nb, args.steps)
    rec, per_k = {}, {}
    for b in range(used):
        ids = graphs[b].ids.cpu().numpy()
        kb = kq[b * nq:(b + 1) * nq]
        off = np.concatenate([[0], np.cumsum(kb)])
        for kk in sorted(set(kb.tolist())):
            sel = np.nonzero(kb == kk)[0]
            got = np.stack([ids[off[i]:off[i + 1]] for i in sel])
            per_k.setdefault(kk, []).append((E.recall(got, gt_ids[b * nq + sel], kk), len(sel)))
    for kk, v in per_k.items():
        rec[str(kk)] = round(sum(r * n for r, n in v) / sum(n for _, n in v), 4)
    # fixed ef for the k = 10 queries of the first batch
    sel10 = np.nonzero(kq[:nq] == 10)[0]
    q10 = pool_d[:nq][torch.from_numpy(sel10).cuda()]
    k10_sweep = []
    for ef in (20, 40, 80, 120, 160, 240, 320, 480):
        ids10, _ = ix.search(q10, 10, ef)
        r = E.recall(ids10.cpu().numpy(), gt_ids[sel10], 10)
        k10_sweep.append({"ef": ef, "recall": round(r, 4)})
        if r >= 0.99:
            break
    hops = st[:, 0].double().cpu().numpy()
    alg = float(hops.sum() * ix.block_bytes + nq * 4 * ix.d + 8 * total0)
    peak, src = measured_peaks()
    stop = None
    if not args.skip_stop:  # the same job with the learned stop on (each query's ef is its cap)
        stop = mixed_stop(args, w, ix, pool_d, gt_ids, kq, efq, nq, nb, max_k, max_ef, knobs, rec, value, local)
    line = {"metric": "queries/sec, mixed k and ef in one launch", "value": round(value, 1),
            "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "n": w.n, "d": w.d, "degree": w.degree, "k": "U{1,10,100}",
                       "ef": "U[k, 8k]", "queries_per_step": nq, "knobs": knobs},
            "recall_per_k": rec,
            "k10_fixed_ef_sweep": k10_sweep,
            "timing": {"l2": l2_note(ix, "isolated steps flushed (512 MiB write)"),
                       "batches": f"{nb} distinct batches of {nq} queries, own k and ef draws; step s searches "
                                  f"batch s mod {nb}",
                       "launch": f"one CUDA graph per batch, steps alternating over {job_streams(nq)} streams",
                       "step_isolated_ms": round(iso_ms, 4)},
            "roofline": {"bound": "hbm", "achieved": round(alg / (ms / 1e3) / 1e9, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(alg / (ms / 1e3) / 1e9 / peak, 4), "peak_source": src,
                         "note": "job step time (plan + rotation + search), not the search kernel alone"},
            "learned_stop": stop,
            "autotune": sorted(tune["table"], key=lambda r: r["ms"])[:6], "clocks": clk,
            "hops_mean": round(float(hops.mean()), 2),
            "gpu_launches": launches_per_step(w.d, args.metric, ragged=True) * args.steps}
    if rank == 0:
        print(json.dumps(line), flush=True)


def mixed_stop(args, w, ix, pool_d, gt_ids, kq, efq, nq, nb, max_k, max_ef, knobs, rec, plain_qps, device):
    """The mixed batch with the learned stop on: one network for k in
    {1, 10, 100} (traces at each group's largest beam, 8k), its threshold
    the most aggressive whose held-out recall@min(k, 10) stays within 0.005
    of the plain search's at the same beams in every group; then the job
    again with the stop (each query's own ef as its cap)."""
    import torch

    from paper_2411_12229_gb300 import autotune
    from paper_2411_12229_gb300 import eval as E
    from paper_2411_12229_gb300 import learned_stop as L
    t0 = time.time()
    tq = synth.train_queries(w, args.stop_train or 8000)
    tg, _ = E.ground_truth(synth.base(w), tq, 100, device=device)
    groups = [(kk, min(8 * kk, max_ef)) for kk in sorted(set(kq.tolist()))]
    model = L.fit_mixed(ix, tq, tg, groups, None, every=8, steps=2000, max_loss=0.005)
    kw = dict(stop_mlp=model.params, stop_logit=model.logit, stop_every=model.every)
    graphs = []
    for b in range(nb):
        sl = slice(b * nq, (b + 1) * nq)
        g = autotune.GraphSearch(ix, nq, kq[sl], efq[sl], max_k=max_k, max_ef=max_ef,
                                 **{**knobs, "team": 32}, **kw)
        g.q.copy_(pool_d[sl])
        graphs.append(g)
    for _ in range(3):
        for g in graphs:
            g.graph.replay()
    ms = time_job(graphs, 2 * nb)
    per_k = {}
    for b in range(nb):
        ids = graphs[b].ids.cpu().numpy()
        kb = kq[b * nq:(b + 1) * nq]
        off = np.concatenate([[0], np.cumsum(kb)])
        for kk in sorted(set(kb.tolist())):
            sel = np.nonzero(kb == kk)[0]
            got = np.stack([ids[off[i]:off[i + 1]] for i in sel])
            per_k.setdefault(kk, []).append((E.recall(got, gt_ids[b * nq + sel], kk), len(sel)))
    srec = {str(kk): round(sum(r * n for r, n in v) / sum(n for _, n in v), 4) for kk, v in per_k.items()}
    qps = nq / (ms / 1e3)
    return {"threshold": model.logit, "every": model.every, "groups": groups, "recall_per_k": srec,
            "qps": round(qps, 1), "qps_ratio_vs_plain": round(qps / plain_qps, 4),
            "seconds": round(time.time() - t0, 1)}


def bench_serving(args, w, ix, q, gt_ids, device):
    """The serving loop (continuous batching, serve.Server) over Poisson
    arrivals at the workload's offered loads, k in {10, 100}: p50/p99
    latency, achieved QPS and recall@10, with the learned stop on and, for
    comparison, off.  Each k gets the smallest ef of the sweep (>= k) whose
    recall@10 on the test queries reaches the target; with the stop, k = 10
    requests may search up to twice that beam, within the compact kernel's
    range for d <= 256 (ef 256)."""
    import torch

    from paper_2411_12229_gb300 import eval as E
    from paper_2411_12229_gb300 import learned_stop as L
    from paper_2411_12229_gb300.serve import Server
    t0 = time.time()
    qd = torch.from_numpy(q).cuda()
    ef_for = {}
    for k in (10, 100):
        for ef in [e for e in w.ef if e >= k] + [768, 1024]:
            ids, _ = ix.search(qd, k, ef)
            if E.recall(ids.cpu().numpy()[:, :10], gt_ids, 10) >= args.target:
                break
        ef_for[k] = ef
    big_ef = COMPACT_MAX_EF_SMALL_D if ix.d <= 256 else COMPACT_MAX_EF
    caps = {10: max(ef_for[10], min(2 * ef_for[10], big_ef)), 100: ef_for[100]}
    tq = synth.train_queries(w, args.stop_train or 20000)
    tg, _ = E.ground_truth(synth.base(w), tq, 100, device=device)
    model = L.fit_mixed(ix, tq, tg, [(10, caps[10]), (100, caps[100])], args.target, every=4)
    loads = (50_000, 100_000, 200_000, 500_000, 1_000_000, 2_000_000)
    rng = np.random.default_rng(5)
    table = {"stop": [], "plain": []}
    for mode in ("stop", "plain"):
        efmap = caps if mode == "stop" else ef_for
        srv = Server(ix, max_k=100, max_ef=max(efmap.values()), mem_budget=256 << 20, streams=8, max_batch=8192,
                     stop_model=model if mode == "stop" else None)
        for load in loads:
            m = int(min(200_000, max(4000, load * 1.0)))
            sel = rng.integers(0, q.shape[0], size=m)
            ks = np.where(rng.integers(0, 2, size=m) == 0, 10, 100).astype(np.int32)
            efs = np.array([efmap[int(k)] for k in ks], dtype=np.int32)
            r = srv.run(q[sel], ks, efs, synth.poisson_arrivals(float(load), m))
            sm = r.summary()
            got = np.full((m, 10), -1, np.int64)
            for i in range(m):
                got[i] = r.ids[i][:10]
            sm.update(offered_qps=load, recall_at_10=round(E.recall(got, gt_ids[sel], 10), 4))
            table[mode].append(sm)
            log(f"serving {mode} {load}: {sm}")
    ok = [x for x in table["stop"] if x["recall_at_10"] >= args.target]
    best = max(ok, key=lambda x: x["qps"]) if ok else None
    okp = [x for x in table["plain"] if x["recall_at_10"] >= args.target]
    bestp = max(okp, key=lambda x: x["qps"]) if okp else None
    line = {"metric": "queries/sec at recall@10>=0.95, serving loop (Poisson arrivals, continuous batching)",
            "value": best["qps"] if best else None, "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "n": w.n, "d": w.d, "degree": w.degree, "k": "{10, 100}",
                       "ef_for_k": ef_for, "stop_caps": caps, "streams": 8, "mem_budget_mb": 256,
                       "offered_loads": list(loads)},
            "learned_stop": {"threshold": model.logit, "every": model.every, "positive_rows": model.info["positive"]},
            "table": table, "plain_best_qps": bestp["qps"] if bestp else None,
            "seconds": round(time.time() - t0, 1)}
    print(json.dumps(line), flush=True)


def bench_reference(args):
    """CPU oracle arm: the same metric, workload and ef as the GPU arm, each
    step a bounded sample of one distinct batch.  The index and the ground
    truth come from a separate process (GPU build), so this one loads the
    oracle's library only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload(args)
    nb = max(1, args.batches)
    idx, gtp = cache_paths(args, w)
    gtf = pathlib.Path(f"{gtp}-r0-b{nb}-w1.npz")
    if not idx.exists() or not gtf.exists():
        cmd = [sys.executable, str(ROOT / "bench.py"), "--build-only", "--workload", args.workload,
               "--cache", args.cache, "--build-iters", str(args.build_iters), "--ef-build", str(args.ef_build),
               "--rotation", args.rotation, "--metric", args.metric, "--graph", args.graph, "--batches", str(nb)]
        if args.n:
            cmd += ["--n", str(args.n)]
        if args.nq:
            cmd += ["--nq", str(args.nq)]
        env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
        subprocess.run(cmd, check=True, env=env)
    gt_ids = np.load(gtf)["ids"]
    pool = replica_queries(w, 0, 1, nb)
    if args.rotation == "fjlt":  # the index's data were zero-padded to a power of 2
        d2 = 1 << (w.d - 1).bit_length()
        pool = np.ascontiguousarray(np.pad(pool, ((0, 0), (0, d2 - w.d))))
    nq, k = w.n_queries, 10
    threads = os.cpu_count() or 1
    # the GPU arm's rule on the same queries: the smallest ef of the sweep
    # whose recall@10 on the first batch reaches the target
    ef_sel, sweep = None, []
    for ef in ([args.ef] if args.ef else w.ef):
        done, el, ids = run_oracle(idx, pool[:nq], k, ef, 1e9, threads, nq)
        got = np.stack([ids[i] for i in range(done)]).astype(np.int64)
        r = E_recall(got, gt_ids[:done], k)
        sweep.append({"ef": ef, "recall": round(r, 4), "qps": round(done / el, 1)})
        if r >= args.target:
            ef_sel = ef
            break
    ef_sel = args.ef or ef_sel or sweep[-1]["ef"]
    per_step = min(nq, 2000)
    sample = lambda s: pool[(s % nb) * nq:(s % nb) * nq + per_step]  # noqa: E731
    for s in range(args.warmup):
        run_oracle(idx, sample(s), k, ef_sel, 1e9, threads, threads)
    tot_q, tot_t = 0, 0.0
    for s in range(args.steps):
        done, el, _ = run_oracle(idx, sample(s), k, ef_sel, 1e9, threads, per_step)
        tot_q += done
        tot_t += el
    v = tot_q / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": headline_config(w, args, k, ef_sel, nq, 1),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"the first {per_step} queries of batch s mod {nb} per step (of {nq}), "
                                       f"ef={ef_sel}, one query per task on {threads} threads"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "sweep": sweep}
    print(json.dumps(line), flush=True)


def E_recall(ids, gt, k):
    """Mean |G cap S| / K (Sec. 5.1) without importing the GPU package."""
    return float(np.mean([len(np.intersect1d(ids[i][:k], gt[i][:k])) for i in range(len(ids))])) / k


def bench_prep(args):
    """Query preparation alone: q' = P^-1 q and its exact 4-bit
    quantization, on the CUDA cores and on the tensor cores (plus the exact
    pass), for the workload's dimension and query count.  The index is a
    small one (--n, default 1000 vertices, exact kNN graph built on the
    host): the rotation does not depend on n."""
    import torch

    from paper_2411_12229_gb300 import index_builder as ib
    from paper_2411_12229_gb300.api import Index
    w = synth.WORKLOADS[args.workload]
    n, nq, d = args.n or 1000, args.nq or w.n_queries, w.d
    ws = synth.small(w, n, 64)
    x = synth.base(ws)
    path = pathlib.Path(args.cache) / f"prep-{w.name}-n{n}-{args.rotation}-{args.metric}.sqg"
    path.parent.mkdir(parents=True, exist_ok=True)
    if not path.exists():
        ib.build_index(path, x, w.degree, rotation=args.rotation, metric=args.metric)
    ix = Index(path, 0)
    q = ix.fit_queries(torch.from_numpy(synth.queries(w.with_(n_queries=nq))).cuda())
    if ix.fjlt:  # the fast transform (no dense contraction, no tensor-core path)
        flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
        for _ in range(max(3, args.warmup)):
            ix.prepare_queries(q)
        ms = []
        for _ in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            ix.prepare_queries(q)
            b.record()
            b.synchronize()
            ms.append(a.elapsed_time(b))
        t = float(np.median(ms))
        traffic = 2.0 * 4 * nq * ix.d  # read q, write q' (the planes are small)
        peak_hbm = json.loads((ROOT / "MEASURED_PEAKS.json").read_text())["hbm_gbs"] \
            if (ROOT / "MEASURED_PEAKS.json").exists() else 6800.0
        print(json.dumps({"metric": "query preparation time (fast JLT + 4-bit quantization)", "unit": "ms",
                          "workload": w.name, "d": w.d, "d_padded": ix.d, "queries": nq, "fjlt_ms": round(t, 4),
                          "roofline": {"bound": "hbm", "achieved": round(traffic / (t / 1e3) / 1e9, 1),
                                       "peak": peak_hbm, "unit": "GB/s",
                                       "frac": round(traffic / (t / 1e3) / 1e9 / peak_hbm, 4)},
                          "l2": "flushed (512 MiB write) before each call"}), flush=True)
        return
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    res = {}
    for name, fn in (("cuda_cores", lambda: ix.prepare_queries(q)), ("tensor_cores", lambda: ix.prepare_queries_tc(q))):
        for _ in range(max(3, args.warmup)):
            out = fn()
        ms = []
        for _ in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            out = fn()
            b.record()
            b.synchronize()
            ms.append(a.elapsed_time(b))
        res[name] = (float(np.median(ms)), out)
    same = bool(torch.equal(res["cuda_cores"][1][1], res["tensor_cores"][1][1]) and
                torch.equal(res["cuda_cores"][1][2], res["tensor_cores"][1][2]))
    rec = int(res["tensor_cores"][1][3].item())
    flop = 2.0 * nq * d * d
    peak = json.loads((ROOT / "MEASURED_PEAKS.json").read_text())["bf16_tflops"] * (1.1 / 2.25) \
        if (ROOT / "MEASURED_PEAKS.json").exists() else 1900.0 * (1.1 / 2.25)
    t_tc = res["tensor_cores"][0]
    line = {"metric": "query preparation time (rotation + 4-bit quantization)", "unit": "ms", "workload": w.name,
            "d": d, "queries": nq, "cuda_core_ms": round(res["cuda_cores"][0], 4), "tensor_core_ms": round(t_tc, 4),
            "speedup": round(res["cuda_cores"][0] / t_tc, 3), "planes_identical": same,
            "recomputed_fraction": round(rec / (nq * d), 5),
            "roofline": {"bound": "tensor", "achieved": round(3 * flop / (t_tc / 1e3) / 1e12, 1),
                         "peak": round(peak, 1), "unit": "TFLOP/s",
                         "frac": round(3 * flop / (t_tc / 1e3) / 1e12 / peak, 4),
                         "note": "3xTF32 FLOP over the tensor-core rotation and the exact pass together; "
                                 "peak = measured bf16 x nominal tf32/bf16 ratio (1.1/2.25)"},
            "l2": "flushed (512 MiB write) before each call"}
    print(json.dumps(line), flush=True)


def headline_config(w, args, k: int, ef: int, nq: int, world: int) -> dict:
    """The workload a step runs, the same in both arms."""
    return {"workload": w.name, "n": w.n, "d": w.d, "degree": w.degree, "rotation": args.rotation,
            "metric": args.metric, "graph": args.graph, "k": k, "ef": ef, "queries_per_step": nq,
            "parallelism": f"replicas{world}"}


def graphs_for(ix, pool, nq: int, k: int, ef: int, nb: int):
    """One captured search per batch: graph b holds batch b of the pool."""
    from paper_2411_12229_gb300.autotune import GraphSearch
    gs = []
    for b in range(nb):
        g = GraphSearch(ix, nq, k, ef, max_k=k, max_ef=ef)
        g.q.copy_(pool[b * nq:(b + 1) * nq])
        gs.append(g)
    return gs


def profile_run(args, w, ix, qd, k: int):
    """Two searches of the first batch at --ef: a warm-up and the launch an
    ncu capture takes (-k regex:search_kernel -s 1 -c 1)."""
    import torch
    ef = args.ef or 40
    for _ in range(2):
        ix.search(qd, k, ef)
    torch.cuda.synchronize()
    log(f"profile: 2 searches of {qd.shape[0]} queries at ef={ef} on {w.name}")


def main():
    args = parse()
    if args.impl == "reference":
        return bench_reference(args)
    import torch

    from paper_2411_12229_gb300 import build as build_mod
    build_mod.build()
    if args.prep:
        return bench_prep(args)
    from paper_2411_12229_gb300 import eval as E
    from paper_2411_12229_gb300.api import Index

    rank, world = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = workload(args)
    idx, gtp = ensure_index(args, w, local, rank)
    if dist:
        dist.barrier()
    nb = 1 if args.profile else (min(4, max(1, args.batches)) if w.mixed_k else max(1, args.batches))
    # each rank serves its own pool of nb distinct batches (replicas, weak scaling)
    pool = replica_queries(w, rank, world, nb)
    nq = w.n_queries
    if args.profile:
        ix = Index(idx, local)
        return profile_run(args, w, ix, ix.fit_queries(torch.from_numpy(pool[:nq]).cuda()), 10)
    gt_ids, gt_d = ground_truth(args, w, f"{gtp}-r{rank}-b{nb}", pool, local, world)
    if args.build_only:
        return
    ix = Index(idx, local)
    if ix.d != pool.shape[1]:  # a fast-JLT index: data and queries zero-padded to a power of 2
        pool = np.ascontiguousarray(np.pad(pool, ((0, 0), (0, ix.d - pool.shape[1]))))
    pool_d = torch.from_numpy(pool).cuda()
    q, qd = pool[:nq], pool_d[:nq]
    if w.name.startswith("serving"):
        return bench_serving(args, w, ix, pool[:nq], gt_ids[:nq], local)
    if w.mixed_k:
        return bench_mixed(args, w, ix, pool_d, pool, gt_ids, rank, world, dist, local, nb)
    k = 10
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    # ---- sweep (untimed for the metric): recall on the first batch (where
    # the operating point is chosen) and on the whole pool, hops, and QPS
    # timed like the job (distinct batches, three streams)
    sweep = []
    nb_sweep = min(nb, 4)
    for ef in ([args.ef] if args.ef else w.ef):
        ids_all, hops_all = [], []
        for b in range(nb):
            ids, _, st = ix.search(pool_d[b * nq:(b + 1) * nq], k, ef, stats=True)
            ids_all.append(ids.cpu().numpy())
            hops_all.append(st[:, 0].float().cpu().numpy())
        ids_all = np.concatenate(ids_all)
        rec0 = E.recall(ids_all[:nq], gt_ids[:nq], k)
        recp = E.recall(ids_all, gt_ids, k)
        gs = graphs_for(ix, pool_d, nq, k, ef, nb_sweep)
        for _ in range(3):
            for g in gs:
                g.graph.replay()
        ms = time_job(gs, 2 * nb_sweep)
        del gs
        rec4 = E.recall(ids_all[:min(nb, 4) * nq], gt_ids[:min(nb, 4) * nq], k)
        sweep.append({"ef": ef, "recall": round(rec0, 4), "recall_4": round(rec4, 4), "recall_pool": round(recp, 4),
                      "qps": round(nq / (ms / 1e3)), "hops": round(float(np.concatenate(hops_all).mean()), 1)})
        if rank == 0:
            log(f"ef={ef} recall@10={rec0:.4f} (pool {recp:.4f}) hops={sweep[-1]['hops']} qps={sweep[-1]['qps']}")
        if rec0 >= 0.995:
            break
    pick = lambda t: next((s["ef"] for s in sweep if s["recall"] >= t), None)  # noqa: E731
    ef_sel = args.ef or pick(args.target) or sweep[-1]["ef"]
    stop_cmp = None
    if rank == 0 and not args.skip_stop and not args.ef:
        stop_cmp = learned_stop_comparison(args, w, ix, pool_d, gt_ids, sweep, ef_sel, local, nq, nb)
    if dist:
        t = torch.tensor([ef_sel], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ef_sel = int(t.item())

    # ---- timed steps: step s replays the graph of batch s mod nb (rotation,
    # search); three streams, so one step's tail overlaps the next steps'
    # start, and no two steps in flight share a query
    graphs = graphs_for(ix, pool_d, nq, k, ef_sel, nb)
    for _ in range(max(3, args.warmup)):
        for g in graphs[:2]:
            g.graph.replay()
    for g in graphs[2:]:
        g.graph.replay()
    iso_ms = isolated_steps(graphs[0], args.steps, flush)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    job_ms = time_job(graphs, args.steps)
    if dist:
        dist.barrier()
    used = min(nb, args.steps)  # batches the job searched
    job_ids = np.concatenate([g.ids.view(nq, k).cpu().numpy() for g in graphs[:used]])
    rec_job = E.recall(job_ids, gt_ids[:used * nq], k)
    # ---- the search kernel alone: events around its launch, L2 flushed,
    # batch s mod nb, outside a graph
    out2 = (torch.empty(nq * k, dtype=torch.int32, device="cuda"), torch.empty(nq * k, device="cuda"))
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in kev:  # create the underlying CUDA events
        a.record()
        b.record()
    sts = []
    for s in range(args.steps):
        flush.zero_()
        b = s % nb
        _, _, st = ix.search(pool_d[b * nq:(b + 1) * nq], k, ef_sel, out=out2, stats=True, timing_events=kev[s])
        sts.append(st)
        if not torch.equal(out2[0], graphs[b].ids):
            raise RuntimeError("graph replay and direct search disagree")
    torch.cuda.synchronize()
    kern_ms = [a.elapsed_time(b) for a, b in kev]
    hops_launch = [float(st[:, 0].double().sum().item()) for st in sts]
    hops = torch.cat(sts)[:, 0].double().cpu().numpy()
    # ---- end to end through host buffers: every step copies its batch in
    # from pinned host memory and its (ids, dists) back, through the public
    # pipelined API (e2e_depth slots: one step's copies overlap another's search);
    # host wall clock over all steps, device idle at both ends
    qh = [torch.from_numpy(pool[b * nq:(b + 1) * nq]).pin_memory() for b in range(nb)]
    e2e_ms, rec_e2e = [], None
    if not args.skip_e2e:
        pipe = ix.host_pipeline(nq, k, ef_sel, depth=e2e_depth(nq))
        for s in range(max(3, args.warmup)):
            pipe.submit(qh[s % nb])
        pipe.drain()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        got = [r for r in (pipe.submit(qh[s % nb]) for s in range(args.steps)) if r is not None]
        got += pipe.drain()
        e2e_ms = [(time.perf_counter() - t0) * 1e3 / args.steps]
        e2e_ids = np.concatenate([got[s][0] for s in range(used)])
        rec_e2e = E.recall(e2e_ids, gt_ids[:used * nq], k)
    clk = clocks.stop()

    (step_max, e2e_max), (value, e2e_value) = aggregate_replicas(
        [job_ms, float(np.mean(e2e_ms)) if e2e_ms else job_ms], nq, world, dist, "cuda")
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # ---- roofline of the search kernel: algorithmic bytes / its event time
    bb = ix.block_bytes
    alg_bytes = float(np.mean(hops_launch) * bb + nq * (4 * ix.d + 8 * k))
    kern_mean = float(np.mean(kern_ms))
    achieved = alg_bytes / (kern_mean / 1e3) / 1e9
    peak, peak_src = measured_peaks()
    tr = traffic_record(w.name, ef_sel, args.metric, args.rotation, args.graph)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_source": peak_src,
                "traffic": tr["dram_bytes_per_launch"] if tr else None,
                "algorithmic_bytes_per_launch": alg_bytes, "kernel_ms": round(kern_mean, 4),
                "kernel": search_kernel_name(ix, k, ef_sel, args),
                "job_frac": round(alg_bytes / (job_ms / 1e3) / 1e9 / peak, 4)}

    cpu = None
    if world == 1 and not args.skip_cpu:
        threads = os.cpu_count() or 1
        done, el, ids_o = run_oracle(idx, q, k, ef_sel, args.cpu_seconds, threads, nq)
        cpu = {"value": round(done / el, 2), "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"first {done} of the first batch's {nq} queries at ef={ef_sel}, {el:.1f}s on "
                         f"{threads} threads"}
        g0 = graphs[0].ids.view(nq, k).cpu().numpy().view(np.uint32)
        same = sum(np.array_equal(ids_o[i], g0[i]) for i in ids_o)
        cpu["ids_identical_to_gpu"] = f"{same}/{len(ids_o)}"
        # one thread, the paper's own search protocol (a few seconds)
        d1, e1, _ = run_oracle(idx, q, k, ef_sel, 3.0, 1, nq)
        cpu["single_thread_value"] = round(d1 / e1, 2)
        cpu["single_thread_sample"] = f"first {d1} queries, {e1:.1f}s on 1 thread"

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(step_max, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": headline_config(w, args, k, ef_sel, nq, world),
        "recall@10": {"first_batch": round(pick_rec(sweep, ef_sel), 4), "job": round(rec_job, 4)},
        "timing": {"l2": l2_note(ix, "isolated steps and kernel launches flushed (512 MiB write)"),
                   "batches": f"{nb} distinct batches of {nq} queries; step s searches batch s mod {nb}",
                   "launch": f"one CUDA graph per batch, steps alternating over {job_streams(nq)} streams",
                   "step_isolated_ms": round(iso_ms, 4),
                   "step_isolated_qps": round(nq / (iso_ms / 1e3), 1)},
        "e2e": {"value": round(e2e_value, 1), "unit": UNIT, "h2d_bytes_per_step": int(nq * ix.d * 4),
                "d2h_bytes_per_step": int(nq * k * 8),
                "recall@10": round(rec_e2e, 4) if rec_e2e is not None else None,
                "api": f"Index.host_pipeline ({e2e_depth(nq)} streams) over the same distinct batches, host wall clock"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "gpu_launches": launches_per_step(w.d, args.metric) * args.steps,
        "clocks": clk,
        "qps_at_recall": {str(t): next((s["qps"] for s in sweep if s["recall"] >= t), None)
                          for t in (0.90, 0.95, 0.99)},
        "ef_at_recall": {str(t): pick(t) for t in (0.90, 0.95, 0.99)},
        "hops_mean": round(float(hops.mean()), 2),
        "index_build": build_record(idx),
        "learned_stop": stop_cmp,
        "sweep": sweep,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def search_kernel_name(ix, k: int, ef: int, args) -> str:
    """The search kernel a default search of this shape runs (the compact
    kernel's range: d <= 1024, degree 32 or 64, k <= 32, ef <= 128; for
    d <= 256 k <= 128, ef <= 256)."""
    small = ix.d <= 256
    if (ix.d <= 1024 and ix.degree in (32, 64) and k <= (128 if small else 32)
            and ef <= (COMPACT_MAX_EF_SMALL_D if small else COMPACT_MAX_EF)):
        return "sqg::search_compact_kernel"
    return "sqg::search_kernel"


def pick_rec(sweep, ef):
    return next(s["recall"] for s in sweep if s["ef"] == ef)


if __name__ == "__main__":
    main()
