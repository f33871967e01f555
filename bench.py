#!/usr/bin/env python
"""Benchmark: exact labeled subgraph matching on one GB300 (or N replicas).

One step = the whole device pipeline (plan, filter, exploration, refinement,
candidate-edge tables, join, sort) over one batch of queries: by default the
10,000 queries of 3-12 vertices (half of them cyclic) on the 4M-vertex /
32M-edge graph, as one batch.  Prints one JSON line.

  value   queries/s of the batched pipeline, inputs resident in HBM
          (CUDA events on the launching stream; L2 flushed between steps)
  e2e     the same metric through the C ABI (gs_match_batch_shared) with
          host buffers: queries packed in host memory, counts, fingerprints
          and rows back in host memory (upload and download inside the timed
          region); also through the Python binding (gs.match_batch)
  one_at_a_time   queries/s when the same device pipeline runs each query
                  as its own wave (the baseline the batching is measured against),
                  on a sample of the queries when the workload is large
  serving  p50/p99/p999 latency and sustained queries/s of the serving loop
           under Poisson arrivals (for the 4M-vertex graph: 1k, 5k, 20k and
           50k queries/s of queries of 3-12 vertices)

--impl reference times the CPU oracle (test infrastructure) on the same
workload on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "queries/s and embeddings/s, batched vs one-at-a-time (exact); serving p50/p99 ms"
# queries the CPU oracle times per workload (all of them for the two small
# workloads; a seeded sample of the large ones, labelled "sampled")
CPU_SAMPLE = {"batch-4m": 200, "serve-4m": 200, "stress-16m": 50}
# queries of the one-at-a-time comparison (a sample where one step of all of
# them would take seconds)
ONE_SAMPLE = {"batch-4m": 1000, "serve-4m": 1000}
L2_FLUSH_BYTES = 512 << 20


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl != "reference" else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock and throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i, v in enumerate(r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# source section (banner name in gs_kernels.cu) of each kernel kind the bench reports
KIND_SECTION = {"sort_large": "sort + gather", "gather": "sort + gather", "join_count": "join", "join_write": "join",
                "ec_count": "edge tables", "ec_write": "edge tables"}


def kernel_section_sha(kind):
    """Hash of the source of one kernel kind: the shared device helpers at the
    top of gs_kernels.cu (before the first banner) plus the text between its
    '// ====... <section>' banner and the next one.  A stored DRAM-traffic
    figure is used only while this still matches."""
    import hashlib
    src = open(os.path.join(ROOT, "paper_1807_08804_gb300", "csrc", "gs_kernels.cu")).read()
    banner = "// " + "=" * 60 + " "
    i = src.find(banner + KIND_SECTION.get(kind, kind) + "\n")
    if i < 0:
        return None
    j = src.find(banner, i + len(banner))
    head = src[:src.find(banner)]
    return hashlib.sha256((head + src[i:j if j > 0 else len(src)]).encode()).hexdigest()[:16]


def stored_traffic(kind, workload):
    """DRAM bytes per launch of `kind` on `workload` from a committed ncu
    summary (a 'traffic-record:' line under profiles/), or None when there
    is none or the kernel's source changed since the capture."""
    import glob
    import re
    sha = kernel_section_sha(kind)
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for line in open(path):
            m = re.match(r"traffic-record: kind=(\S+) workload=(\S+) bytes_per_launch=(\d+) section_sha=(\S+)", line)
            if m and m.group(1) == kind and m.group(2) == workload and m.group(4) == sha:
                return int(m.group(3))
    return None


def refinement_ablation(gs, dg, qs, cap, gmode, sh, stream, flush, steps, want):
    """The refinement variants the thesis compares (converged in visit order,
    converged in reversed order, one reversed round, none) plus one reversed
    round that skips degree-1 query vertices: batched time per step, run and
    finish (CUDA events, L2 flushed between steps), and the partial-embedding words of the
    join levels (sum over queries of every level before the last, and the
    largest level of any query).  Every variant must give the same counts and
    fingerprints."""
    import torch
    variants = [("converged", 0, 64), ("converged-reversed", gs.GS_REFINE_REVERSED, 64),
                ("one-round-reversed", gs.GS_REFINE_REVERSED, 1), ("none", gs.GS_REFINE_OFF, 1),
                ("one-round-reversed-skip-degree-1", gs.GS_REFINE_REVERSED | gs.GS_REFINE_LOW(1), 1),
                ("baseline-outgoing-graph-tree-only", gs.GS_REFINE_BASELINE, 1)]
    out = []
    for name, refine, rounds in variants:
        b = gs.Batch(dg, qs, cap=cap, mode=gmode, stream=sh, max_refine_rounds=rounds, refine=refine)
        for _ in range(3):
            b.run()
            b.finish()
        res = b.fetch()
        same = all((r.count, r.fingerprint) == (x.count, x.fingerprint) for r, x in zip(res, want))
        tot, peak = b.join_sizes()
        ms = 0.0
        for _ in range(steps):
            flush.fill_(1)
            stream.wait_stream(torch.cuda.current_stream())
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.run()
            b.finish()  # queries sent to the chunked path finish inside the timed region
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        out.append({"variant": name, "ms_per_step": ms / steps, "queries_per_s": len(qs) * steps / (ms / 1e3),
                    "partial_words_total": int(tot.sum()), "partial_words_peak": int(peak.max()) if len(peak) else 0,
                    "results_identical": same, "fallback_queries": b.counters().get("fallback_queries", 0)})
        b.close()
    return out


class SubBatches:
    """The workload's queries as `parts` prepared batches run at once, each on
    its own stream (gs_batch_run_all), behind the interface of one batch; one
    part is a plain batch on the main stream."""

    def __init__(self, gs, dg, qs, parts, main_stream, **kw):
        import torch
        self.gs, self.main = gs, main_stream
        n = len(qs)
        self.streams = [torch.cuda.Stream() for _ in range(parts)] if parts > 1 else []
        sh = [st.cuda_stream for st in self.streams] if parts > 1 else [main_stream]
        self.bs = [gs.Batch(dg, qs[n * i // parts: n * (i + 1) // parts], stream=sh[i], **kw) for i in range(parts)]

    def run(self):
        if len(self.bs) == 1:
            self.bs[0].run()
        else:
            self.gs.run_all(self.bs, self.main)

    def finish(self):
        for b in self.bs:
            b.finish()

    def fetch(self):
        return [r for b in self.bs for r in b.fetch()]

    def counters(self):
        out = {}
        for b in self.bs:
            for k, v in b.counters().items():
                out[k] = out.get(k, 0) + v
        return out

    def stats_enable(self, on=True):
        for b in self.bs:
            b.stats_enable(on)

    def stats_reset(self):
        for b in self.bs:
            b.stats_reset()

    def stats(self):
        out = {}
        for b in self.bs:
            for k, v in b.stats().items():
                a = out.setdefault(k, {"launches": 0, "ms": 0.0, "bytes": 0})
                for f in a:
                    a[f] += v[f]
        return out

    def busy(self):
        """Per kind, ms during which some launch of it ran (overlaps once)."""
        return self.gs.stats_busy(self.bs)

    def close(self):
        for b in self.bs:
            b.close()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def cpu_sample(qs, n, seed):
    """A seeded sample of n of the queries (all of them when n >= len(qs))."""
    import numpy as np
    if n >= len(qs):
        return list(qs), "all"
    idx = np.sort(np.random.default_rng(seed).choice(len(qs), n, replace=False))
    return [qs[i] for i in idx], f"a seeded sample of {n}"


def cpu_baseline(workload, g, qs, sample_n=None, min_seconds=10.0, max_repeats=30):
    """The oracle as it stands, counts and fingerprints, on every host core:
    the sample is run repeatedly until at least min_seconds have passed (at
    most max_repeats times), so that the rate rests on 10-30 s of CPU work."""
    import oracle
    og = oracle.OracleGraph.from_graph(g)
    sample, how = cpu_sample(qs, len(qs) if sample_n is None else sample_n, workload.seed + 0x5A)
    reps, done, emb, timed_out, used = 0, 0, 0, 0, 0
    t = time.perf_counter()
    while reps < max_repeats and (reps == 0 or time.perf_counter() - t < min_seconds):
        cnt, fp, st, used = oracle.match_many(og, sample, threads=0, time_limit_s=60.0)
        reps += 1
        done += len(sample)
        emb += int(cnt.sum())
        timed_out += int((st == 2).sum())
    dt = time.perf_counter() - t
    return {"value": done / dt, "unit": "queries/s", "cores": int(used), "kind": "oracle",
            "sample": f"{how} of the {len(qs)} queries of {workload.name} (counts and fingerprints, "
                      f"all embeddings enumerated), run {reps} times in {dt:.2f} s, {timed_out} timed out"
                      + ("" if how == "all" else "; sampled"),
            "embeddings_per_s": emb / dt}


def serve_measure(gs, dg, qs, rate_qps, duration_s, cap, seed=1, warmup_s=1.0, warmup_min=4096):
    """Poisson arrivals at rate_qps for duration_s into the serving loop,
    after warmup_s of arrivals at the same rate (at least warmup_min of
    them) whose results are dropped: the slots capture their pipelines for
    each query size and size their pools then.  Latency is
    submit-to-completion as the server observes it."""
    from paper_1807_08804_gb300 import inputs as I
    pack = gs._QueryPack(qs)
    srv = gs.Server(dg, slots=4, max_batch=256)
    nw = max(int(rate_qps * warmup_s), warmup_min) if warmup_s > 0 else 0
    if nw:
        warr = I.make_arrivals(nw, rate_qps, seed=seed + 1000)
        wt, t0 = [], time.perf_counter()
        for i in range(nw):
            while time.perf_counter() - t0 < warr[i]:
                pass
            wt.append(srv.submit_packed(pack, (i * 7919) % len(qs), cap=cap))
        deadline = time.perf_counter() + 120
        while wt and time.perf_counter() < deadline:
            wt = [t for t in wt if srv.poll(t) is None]
    n = max(1, int(rate_qps * duration_s))
    arr = I.make_arrivals(n, rate_qps, seed=seed)
    tickets, t_sub = [], []
    t0 = time.perf_counter()
    for i in range(n):
        while time.perf_counter() - t0 < arr[i]:
            pass
        t_sub.append(time.perf_counter() - t0)
        tickets.append(srv.submit_packed(pack, i % len(qs), cap=cap))
    submit_end = time.perf_counter() - t0
    lat, done_at = [], []
    pending = list(range(n))
    deadline = time.perf_counter() + 120
    while pending and time.perf_counter() < deadline:
        rest = []
        for i in pending:
            r = srv.poll(tickets[i])
            if r is None:
                rest.append(i)
            else:
                lat.append(r[1])
                done_at.append(t_sub[i] + r[1])  # the server's completion time
        pending = rest
    srv.close()
    lat.sort()
    q = lambda p: 1e3 * lat[min(len(lat) - 1, int(p * len(lat)))] if lat else None
    # sustained rate from the server's own completion times (the polling
    # loop here is slower than the server at the highest rates)
    last = max(done_at) if done_at else float("inf")
    return {"offered_qps": rate_qps, "requests": n, "completed": len(lat), "p50_ms": q(0.50), "p99_ms": q(0.99),
            "p999_ms": q(0.999), "sustained_qps": len(lat) / max(last, submit_end), "submit_s": submit_end,
            "warmup_requests": nw}


def run_reference(args, world, rank):
    from paper_1807_08804_gb300 import inputs as I
    import oracle
    if rank != 0:
        return
    w = I.WORKLOADS[args.workload]
    g = w.graph()
    qs = w.queries(g)
    og = oracle.OracleGraph.from_graph(g)
    n_ref = args.ref_sample if args.ref_sample is not None else CPU_SAMPLE.get(w.name, len(qs))
    per_step, how = cpu_sample(qs, n_ref, w.seed + 0x5A)
    for _ in range(args.warmup):
        oracle.match_many(og, per_step, threads=0, time_limit_s=60.0)
    times, used, emb = [], 1, 0
    for _ in range(args.steps):
        t = time.perf_counter()
        cnt, fp, st, used = oracle.match_many(og, per_step, threads=0, time_limit_s=60.0)
        times.append(time.perf_counter() - t)
        emb = int(cnt.sum())
    tot = sum(times)
    value = len(per_step) * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": w.name, "vertices": w.V, "edges": w.E, "queries": len(per_step),
                       "query_vertices": [w.kmin, w.kmax], "p_bind": w.p_bind, "cap": w.cap},
            "embeddings_per_s": emb * args.steps / tot,
            "cpu_baseline": {"value": value, "unit": "queries/s", "cores": int(used), "kind": "oracle",
                             "sample": f"{how} of the {len(qs)} queries of {w.name} per step, counts and "
                                       f"fingerprints" + ("" if how == "all" else "; sampled")},
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


KHOP_METRIC = "domain-graph exploration: adjacency entries scanned/s (k-hop from seed concepts)"


def run_khop(args, world, rank, local):
    """Domain-graph exploration (k hops from seed concepts, both directions)
    on a workload's graph: seeds and the level array resident on the device;
    each step is one whole exploration (level array reset, seeds, every
    level), timed with CUDA events on the library's stream with L2 flushed
    between steps; e2e runs the same call from host buffers (seeds in, the
    V-byte level array out)."""
    import numpy as np
    import torch
    import paper_1807_08804_gb300 as gs
    from paper_1807_08804_gb300 import inputs as I
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = I.WORKLOADS[args.workload]
    g = w.graph()
    dg = gs.DeviceGraph(g)
    rng = np.random.default_rng(w.seed + 0x6B)
    seeds = rng.choice(g.num_vertices, args.khop_seeds, replace=False).astype(np.uint32)
    L = args.khop
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream
    ts = torch.tensor(seeds.astype(np.int32), device=dev)
    tl = torch.empty(g.num_vertices, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    run = lambda: gs.khop(dg, None, L, device=(ts.data_ptr(), len(seeds), tl.data_ptr()), stream=sh)
    for _ in range(max(args.warmup, 3)):
        _, cnt, edges = run()
    lv, hc, he = gs.khop(dg, seeds, L)  # the host path gives the same exploration
    assert hc.tolist() == cnt.tolist() and he == edges and (torch.from_numpy(lv).to(dev) == tl).all().item()
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        stream.wait_stream(torch.cuda.current_stream())
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    tot_ms = max_over_ranks(sum(ms), world, dev)
    value = edges * world * args.steps / (tot_ms / 1e3)
    t = time.perf_counter()
    e2e_steps = max(2, args.steps // 2)
    for _ in range(e2e_steps):
        gs.khop(dg, seeds, L)
    e2e_s = max_over_ranks(time.perf_counter() - t, world, dev)
    # algorithmic bytes of one exploration: level array fill and visited
    # bitmap clear, per frontier vertex its list entry and one row-offset pair
    # per direction, 4 bytes per adjacency entry scanned, per reached vertex
    # its level byte and next-frontier entry
    V = g.num_vertices
    front = int(cnt[:L].sum())
    reached = int(cnt.sum())
    algo = V + V // 8 + front * (4 + 2 * 16) + 4 * edges + 5 * reached
    peak, peak_kind = measured_peaks()
    achieved = algo / (tot_ms / args.steps / 1e3) / 1e9
    line = {"metric": KHOP_METRIC, "value": value, "unit": "edges/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": w.name, "vertices": V, "edges": w.E, "seeds": len(seeds), "levels": L,
                       "directions": "both", "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MB write)",
                       "parallelism": f"replicas x{world}"},
            "vertices_per_level": [int(x) for x in cnt], "edges_scanned_per_step": edges,
            "e2e": {"value": edges * world * e2e_steps / e2e_s, "unit": "edges/s",
                    "h2d_bytes_per_step": 4 * len(seeds), "d2h_bytes_per_step": V + 8 * (L + 1) + 8},
            "gpu_launches": 2 + L,
            "roofline": {"bound": "hbm", "kernel": "khop (one exploration)", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind, "traffic": None,
                         "bytes_per_step": algo},
            "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    dg.free()


COMPRESS_METRIC = "queries/s through a multi-level compressed graph (exact), with the compression ratio"


def run_compressed(args, world, rank, local):
    """Matching through a multi-level compression (the compress-* workloads):
    the compression is built once (offline, untimed; its time is reported),
    then each step matches every query through the compressed graph from host
    buffers (weighted-graph stage, data-graph stage, results to the host),
    timed with CUDA events on the library's work and wall clock around the
    call.  The same queries on the uncompressed graph are timed beside it."""
    import torch
    import paper_1807_08804_gb300 as gs
    from paper_1807_08804_gb300 import inputs as I
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = I.WORKLOADS[args.workload]
    g = w.graph()
    qs = w.queries(g)
    n = len(qs)
    t = time.perf_counter()
    cg = gs.CompressedGraph(g, w.deltas)
    build_s = time.perf_counter() - t
    info = cg.info()
    dg = gs.DeviceGraph(g)
    for _ in range(max(args.warmup, 3)):
        res = cg.match_batch(qs, cap=w.cap)
    plain = gs.match_batch(dg, qs, cap=w.cap)
    assert all((a.count, a.fingerprint) == (b.count, b.fingerprint) for a, b in zip(res, plain)), "paths disagree"
    embeddings = sum(r.count for r in res)
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(args.steps):
        res = cg.match_batch(qs, cap=w.cap)
    torch.cuda.synchronize()
    dt = max_over_ranks(time.perf_counter() - t, world, dev)
    barrier(world)
    clk = clocks.stop()
    t = time.perf_counter()
    for _ in range(args.steps):
        plain = gs.match_batch(dg, qs, cap=w.cap)
    torch.cuda.synchronize()
    dt_plain = max_over_ranks(time.perf_counter() - t, world, dev)
    value = n * world * args.steps / dt
    line = {"metric": COMPRESS_METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": w.name, "vertices": w.V, "edges": w.E, "queries": n, "deltas": list(w.deltas),
                       "target_s": w.target_s, "copy_p": w.copy_p, "cap": w.cap,
                       "parallelism": f"replicas x{world}"},
            "compression": {**info, "build_s": build_s},
            "embeddings_per_step": embeddings,
            "e2e": {"value": value, "unit": "queries/s", "note": "host buffers in and out each step"},
            "uncompressed": {"value": n * world * args.steps / dt_plain, "unit": "queries/s"},
            "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    cg.free()
    dg.free()


def run_profile_once(args):
    """One small program for ncu captures: the workload's batch (or its first
    --queries queries) run --runs times, with no timing, comparison modes,
    serving or CPU baseline, so that a capture of a few kernels ends
    quickly.  The batch is split into sub-batches run together as the timed
    step splits it (--parts; 4 from 4,096 queries), so every launch does the
    work of one launch of the step."""
    import torch
    import paper_1807_08804_gb300 as gs
    from paper_1807_08804_gb300 import inputs as I
    w = I.WORKLOADS[args.workload]
    g = w.graph()
    qs = w.queries(g, args.queries or None)
    dg = gs.DeviceGraph(g)
    if args.group or args.rounds:
        gs.tune_set(dg, args.group, args.rounds)
    stream = torch.cuda.Stream()
    parts = args.parts if args.parts else (4 if len(qs) >= 4096 else 1)
    b = SubBatches(gs, dg, qs, parts, stream.cuda_stream, cap=w.cap)
    if args.stats:
        b.stats_enable(True)
    for _ in range(args.runs):
        b.run()
        b.finish()
    res = b.fetch()
    print(f"{len(qs)} queries, {sum(r.count for r in res)} embeddings, {sum(r.status != 0 for r in res)} not ok",
          flush=True)
    if args.stats:  # algorithmic bytes and launches per kernel kind over the runs
        print(json.dumps({k: v for k, v in b.stats().items() if v["launches"]}), flush=True)
    b.close()
    dg.free()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gs", choices=["gs", "reference"])
    ap.add_argument("--workload", default="batch-4m")
    ap.add_argument("--one-steps", type=int, default=2, help="steps of the one-query-at-a-time comparison")
    ap.add_argument("--ref-sample", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=4.0, help="seconds of arrivals per serving rate (0 = skip)")
    ap.add_argument("--one-sample", type=int, default=None,
                    help="queries in the one-at-a-time comparison (default: all, or 1,000 of the 4M workloads)")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (library defaults)")
    ap.add_argument("--tune-cache", default=os.path.join(ROOT, "paper_1807_08804_gb300", "_build", "tune_cache.txt"),
                    help="autotuner cache file: a choice made once for this graph, GPU and load is reused")
    ap.add_argument("--mode", default=None, choices=["enumerate", "count", "chunked"],
                    help="enumerate rows (default), count only (default for stress-16m), or stream every "
                         "embedding through the chunk callback (chunked enumeration)")
    ap.add_argument("--ablation", action="store_true",
                    help="also time the refinement variants (converged, reversed order, one round, none, "
                         "low-connectivity skip) and report their partial-embedding words")
    ap.add_argument("--khop", type=int, default=0,
                    help="time the domain-graph exploration instead: this many hops from --khop-seeds seeds")
    ap.add_argument("--khop-seeds", type=int, default=16)
    ap.add_argument("--project", default=None,
                    help="comma-separated query vertices whose distinct tuples are returned (projection)")
    ap.add_argument("--parts", type=int, default=0,
                    help="sub-batches run at once for the timed step (0 = 4 for 4,096 queries or more, else 1)")
    ap.add_argument("--profile-once", action="store_true",
                    help="run the workload's batch --runs times and nothing else (for ncu captures)")
    ap.add_argument("--queries", type=int, default=0, help="--profile-once: the first this many queries (0 = all)")
    ap.add_argument("--stats", action="store_true", help="--profile-once: print bytes and launches per kernel kind")
    ap.add_argument("--runs", type=int, default=1, help="--profile-once: runs of the batch")
    ap.add_argument("--group", type=int, default=0, help="--profile-once: lanes per work item (0 = default)")
    ap.add_argument("--rounds", type=int, default=0,
                    help="--profile-once: refinement rounds (0 = default, 4294967295 = none)")
    args = ap.parse_args()
    if args.profile_once:
        run_profile_once(args)
        return
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.khop:
        run_khop(args, world, rank, local)
        return
    from paper_1807_08804_gb300 import inputs as _inputs
    if _inputs.WORKLOADS[args.workload].deltas:
        run_compressed(args, world, rank, local)
        return

    import numpy as np
    import torch
    import paper_1807_08804_gb300 as gs
    from paper_1807_08804_gb300 import inputs as I

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = I.WORKLOADS[args.workload]
    g = w.graph()
    qs = w.queries(g)
    n = len(qs)
    mode = args.mode or ("count" if w.shapes or w.anchored or w.count_only else "enumerate")
    gmode = {"count": gs.GS_COUNT_ONLY, "chunked": gs.GS_CHUNKED}.get(mode, gs.GS_ENUMERATE)
    cap = 0 if mode != "enumerate" else w.cap
    streamed = [0]  # rows delivered to the chunk callback (chunked mode)

    def on_chunk(ptr, n_rows, k, query):  # device pointer, nothing copied
        streamed[0] += n_rows

    chunk_cb = on_chunk if mode == "chunked" else None
    project = [int(x) for x in args.project.split(",")] if args.project else None
    chunk_bytes = (8 << 30) if mode == "chunked" else 0  # 8 GB output chunks
    dg = gs.DeviceGraph(g)
    tuned = None
    if not args.no_tune:  # untimed
        os.makedirs(os.path.dirname(os.path.abspath(args.tune_cache)), exist_ok=True)
        # chunked mode runs the count-only pipeline on the device and streams
        # on the chunked join, so it is tuned as count-only
        tuned = gs.tune(dg, qs, cap=cap, mode=gs.GS_COUNT_ONLY if mode == "chunked" else gmode,
                        cache_path=args.tune_cache)
    # A dedicated stream: the library launches on it and the CUDA events are
    # recorded on it (the legacy default stream would not order with it).
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    sh = stream.cuda_stream
    assert sh != 0
    # large batches run as concurrent sub-batches, as gs_match_batch runs them
    parts = args.parts if args.parts else (4 if n >= 4096 else 1)
    b = SubBatches(gs, dg, qs, parts, sh, cap=cap, mode=gmode, chunk_bytes=chunk_bytes, on_chunk=chunk_cb,
                   raw_chunks=True, project=project)
    n_one = args.one_sample if args.one_sample is not None else ONE_SAMPLE.get(w.name, n)
    one_qs = qs[:n_one]
    one = gs.Batch(dg, one_qs, cap=cap, mode=gmode, wave_queries=1, stream=sh, chunk_bytes=chunk_bytes,
                   on_chunk=chunk_cb, project=project, raw_chunks=True)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    for _ in range(max(args.warmup, 3)):
        b.run()
        b.finish()  # finishes queries that need the chunked path too
    res = b.fetch()
    embeddings = sum(r.count for r in res)
    proj_rows = sum(r.rows.shape[0] for r in res)  # distinct projected tuples returned
    bad = [i for i, r in enumerate(res) if r.status != 0]
    # queries that finish on the chunked path (and, in chunked mode, the
    # streaming itself) run inside the timed steps
    fallback_needed = b.counters().get("fallback_queries", 0) > 0 or mode == "chunked"
    if args.one_steps:
        one.run()
        one.finish()
        ref = one.fetch()
        assert len(ref) == len(one_qs)
        assert all((x.count, x.fingerprint) == (y.count, y.fingerprint) for x, y in zip(res, ref)), "modes disagree"

    # ---- timed region: batched pipeline, device-resident inputs
    b.stats_enable(True)
    b.run()
    b.finish()
    b.stats_reset()
    launches0 = b.counters()["kernel_launches"]
    streamed[0] = 0
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    step_ms = []
    for _ in range(args.steps):
        flush.zero_()
        stream.wait_stream(torch.cuda.current_stream())  # the flush ends before the timed work starts
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.run()
        if fallback_needed:
            b.finish()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    streamed_timed = streamed[0]
    if not fallback_needed:
        b.finish()
    launches = b.counters()["kernel_launches"] - launches0
    stats = b.stats()
    busy = b.busy()
    tot_ms = max_over_ranks(sum(step_ms), world, dev)
    value = n * world * args.steps / (tot_ms / 1e3)

    # ---- one query at a time through the same pipeline
    one_ms = []
    for _ in range(args.one_steps if args.one_steps else 0):
        flush.zero_()
        stream.wait_stream(torch.cuda.current_stream())
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        one.run()
        e1.record(stream)
        e1.synchronize()
        one_ms.append(e0.elapsed_time(e1))
    if args.one_steps:
        one.finish()
    one_tot = max_over_ranks(sum(one_ms), world, dev)
    one_qps = len(one_qs) * world * args.one_steps / (one_tot / 1e3) if args.one_steps else None

    # ---- end to end through the C ABI with host buffers: gs_match_batch_shared
    # on the queries packed once as gs_query structs over host arrays; the
    # counts, fingerprints and sorted rows come back in host memory (rows in
    # the library's page-locked buffers, released after each step)
    import ctypes
    pack = gs.QueryPack(qs)
    ccb = gs.chunk_callback(chunk_cb, True)
    copts = gs.match_opts(cap, gmode, 0, chunk_bytes, on_chunk=ccb, project=project)
    cres = (gs.ResultDesc * n)()

    def c_step():
        blk = gs.P()
        gs.check(gs.lib().gs_match_batch_shared(dg._h, pack.arr, n, ctypes.byref(copts), cres, ctypes.byref(blk)))
        got = int(np.frombuffer(cres, gs.RES_DTYPE, count=n)["count"].sum())  # the result, read on the host
        gs.lib().gs_results_free(cres, n)  # rows a result owns (none when all are shared)
        if blk:
            gs.lib().gs_rows_release(blk)
        return got

    c_step()  # warm the reusable pools
    h0, d0 = dg.io_bytes()
    barrier(world)
    torch.cuda.synchronize()
    t = time.perf_counter()
    e2e_steps = max(2, args.steps)
    for _ in range(e2e_steps):
        got = c_step()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t, world, dev)
    h1, d1 = dg.io_bytes()
    assert got == embeddings
    # the same through the Python binding (Query objects in, MatchResult
    # objects with row views out)
    out = gs.match_batch(dg, qs, cap=cap, mode=gmode, chunk_bytes=chunk_bytes, on_chunk=chunk_cb, project=project,
                         raw_chunks=True)
    del out
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(e2e_steps):
        out = gs.match_batch(dg, qs, cap=cap, mode=gmode, chunk_bytes=chunk_bytes, on_chunk=chunk_cb, raw_chunks=True,
                             project=project)
    torch.cuda.synchronize()
    py_s = max_over_ranks(time.perf_counter() - t, world, dev)
    assert sum(r.count for r in out) == embeddings
    del out

    # ---- serving: continuous batching under Poisson arrivals (on the 4M
    # graph, the serving workload's own queries and rates)
    sw = I.WORKLOADS["serve-4m"] if w.name in ("batch-4m", "serve-4m") else w
    sqs = qs if sw is w else sw.queries(g)
    rates = sw.qps if sw.qps else (20000.0,)
    serving = ([serve_measure(gs, dg, sqs, r, args.serve_seconds, sw.cap) for r in rates]
               if args.serve_seconds > 0 and not w.shapes and mode == "enumerate" and not project else [])

    # ---- roofline of the dominant kernel
    peak, peak_kind = measured_peaks()
    # The sub-batches' launches of one kind overlap: a kind's time is the
    # time some launch of it was running (the union of the launches'
    # event intervals), and its achieved bandwidth is its algorithmic bytes
    # over that time.
    kinds = {k: v for k, v in stats.items() if v["launches"] and v["bytes"]}
    dom = max(kinds, key=lambda k: busy.get(k, 0.0)) if kinds else None
    roof = None
    if dom:
        achieved = kinds[dom]["bytes"] / (busy[dom] / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind, "traffic": stored_traffic(dom, w.name),
                "bytes_per_launch": kinds[dom]["bytes"] / kinds[dom]["launches"],
                "launches_per_step": kinds[dom]["launches"] / args.steps,
                "busy_ms_per_step": busy[dom] / args.steps,
                "ms_per_launch": kinds[dom]["ms"] / kinds[dom]["launches"],
                "timing": "bytes over the time some launch of the kernel ran (overlapping launches of the "
                          "concurrent sub-batches count once), CUDA events on the launching streams, timed steps"}

    line = {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": w.name, "vertices": w.V, "edges": w.E, "queries": n, "mode": mode,
                       "query_vertices": [w.kmin, w.kmax], "p_bind": w.p_bind, "cap": cap,
                       "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MB write)",
                       "parallelism": f"replicas x{world}", "tuned": tuned, "sub_batches": parts,
                       **({"project": project} if project else {})},
            "embeddings_per_s": embeddings * world * args.steps / (tot_ms / 1e3),
            "embeddings_per_step": embeddings,
            **({"streamed_rows_per_step": streamed_timed / args.steps} if mode == "chunked" else {}),
            **({"projected_rows_per_step": proj_rows} if project else {}),
            "one_at_a_time": ({"value": one_qps, "unit": "queries/s", "ms_per_step": one_tot / args.one_steps,
                               "queries": len(one_qs), "speedup_batched": value / one_qps,
                               "sample": "all" if len(one_qs) == n else f"the first {len(one_qs)} queries; sampled"}
                              if one_qps else None),
            "e2e": {"value": n * world * e2e_steps / e2e_s, "unit": "queries/s",
                    "h2d_bytes_per_step": (h1 - h0) // e2e_steps, "d2h_bytes_per_step": (d1 - d0) // e2e_steps,
                    "call": "gs_match_batch_shared, queries packed in host memory, results read on the host",
                    "python_api": {"value": n * world * e2e_steps / py_s, "unit": "queries/s",
                                   "call": "gs.match_batch: Query objects in, MatchResult objects out"}},
            "gpu_launches": launches,
            "serving": serving,
            "roofline": roof,
            "clocks": clk,
            # per kind: time some launch of it ran (busy) and the launches' summed durations
            "kernel_ms_per_step": {k: busy.get(k, 0.0) / args.steps for k, v in stats.items() if v["launches"]},
            "kernel_launch_ms_per_step": {k: v["ms"] / args.steps for k, v in stats.items() if v["launches"]},
            "kernel_bytes_per_step": {k: v["bytes"] // args.steps for k, v in stats.items() if v["bytes"]},
            "fallback_queries": b.counters().get("fallback_queries", 0), "failed_queries": len(bad)}
    if args.ablation:
        line["ablation"] = refinement_ablation(gs, dg, qs, cap, gmode, sh, stream, flush, args.steps, res)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, g, qs, sample_n=CPU_SAMPLE.get(w.name))
    if rank == 0:
        print(json.dumps(line), flush=True)
    b.close()
    one.close()
    dg.free()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
