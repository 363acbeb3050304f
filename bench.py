#!/usr/bin/env python3
"""Benchmark of the EmbedJoin hot path on one GPU (or N independent replicas).

Default workload (long DNA-like strings): n = 20000 strings over {A,C,G,T}, 2000
clusters of 10, base length uniform in [4500, 5500], each member carrying
Poisson(rate * length) random edits with rate uniform in [1%, 8%]. One step =
the whole join (validate -> pack -> random tables -> CGK walk + signatures ->
buckets -> pairs -> dedup -> verify -> sorted output) at K = 50, 150 and 250
(r = 7, m = 20 functions, z = 15/14/13 positions, L = 5000), inputs resident in
HBM. --workload protein / text select the protein-like (n=200000, K=40,60) and
text-like (n=350000, K=100,200,300) sets instead.

The headline runs the step through ej_batch: the joins of a step captured once
as a CUDA graph (each join on its own stream, one merged verifier launch over
all joins' candidates) and replayed every step, outputs read back sorted; the
roofline is that merged launch's, timed with CUDA events inside the batch.
Beside it the same step is timed through one ej_join call per K (whose
per-stage events give the stage breakdown and a per-launch verify roofline)
and through the plain per-stage calls ej_embed -> ej_sign -> ej_lsh_candidates
-> ej_verify; all three must return the same pair sets. --batch-eager issues
the batch's work without a graph (the same work, for per-kernel profilers).

Metric: candidate pairs verified per second of whole-step wall time (the
"verified pairs/s" of the headline metric; join wall time and band cells/s are
reported beside it). The L2 cache is flushed (256 MiB write) before every timed
step, outside the timed events.

--impl reference times the CPU oracle (plain single-threaded C) on a bounded
sample of the same workload, the same metric.
"""
from __future__ import annotations

import argparse
import dataclasses
import datetime
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "verified pairs/s (candidate pairs verified per second of whole-join wall time)"
# GB300: 152 SMs; the integer ALU pipe (add, logic, shift) retires 16 lanes per clock
# per SM sub-partition, 64 per SM, at up to 2070 MHz
SMS, ALU_LANES_PER_SM, MAX_SM_MHZ = 152, 64, 2070.0
INT_OPS_PER_WORD_COLUMN = 26   # 32-bit ops of one 64-bit word of the bit-parallel step
VERIFY_SOURCE = os.path.join(ROOT, "paper_1702_00093_gb300", "csrc", "ej_verify_pq.cu")
# DRAM bytes per verify launch (dram__bytes_read.sum + dram__bytes_write.sum) from
# one ncu capture of the long-DNA workload: "merged" = the batch's merged launch,
# "join" = mean over the K=50/150/250 launches of ej_join; valid only while the
# verify source is the one that was captured
VERIFY_TRAFFIC = {"source_sha256_prefix": "543eb403d5eb9127", "bytes_per_launch": {"merged": 11593472, "join": None}}


def workloads():
    from paper_1702_00093_gb300 import synth
    return {
        "long_dna": dict(
            make=lambda seed, args: synth.long_dna(n_clusters=args.clusters, seed=seed),
            seed=1002, params=synth.long_dna_params, Ks=(50, 150, 250),
            sample=lambda args: synth.long_dna(n_clusters=args.sample_clusters, seed=1002),
            desc=lambda ss, args: (f"long DNA-like self-join: n={ss.n} over ACGT, {args.clusters} clusters of 10, "
                                   f"length U[4500,5500], member edit rate U[1%,8%]")),
        "protein": dict(
            make=lambda seed, args: synth.protein_like(seed, args.n or 200000), seed=1003, params=synth.protein_params,
            Ks=synth.PROTEIN_KS, sample=lambda args: synth.protein_like(1003, 20 * args.sample_clusters),
            desc=lambda ss, args: (f"protein-like self-join: n={ss.n} over 25 letters (Zipf 1), log-normal "
                                   f"length (median 400) in [100,2000], 20% near-duplicates")),
        "text": dict(
            make=lambda seed, args: synth.text_like(seed, args.n or 350000), seed=1004, params=synth.text_params,
            Ks=synth.TEXT_KS, sample=lambda args: synth.text_like(1004, 3 * args.sample_clusters),
            desc=lambda ss, args: (f"text-like self-join: n={ss.n} over 37 symbols, length U[800,3000], "
                                   f"clusters of 2-20 at edit rate U[2%,20%]")),
    }


def verify_traffic(kind):
    with open(VERIFY_SOURCE, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()
    if VERIFY_TRAFFIC["source_sha256_prefix"] and sha.startswith(VERIFY_TRAFFIC["source_sha256_prefix"]):
        return VERIFY_TRAFFIC["bytes_per_launch"][kind]
    return None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["long_dna", "protein", "text", "serving"], default="long_dna")
    ap.add_argument("--index-size", type=int, default=1_000_000, help="serving: strings in the index")
    ap.add_argument("--queries", type=int, default=4000, help="serving: queries in the stream")
    ap.add_argument("--rates", type=str, default="500,2000,8000,32000,128000", help="serving: offered queries/s")
    ap.add_argument("--clusters", type=int, default=2000, help="clusters of 10 strings (long DNA)")
    ap.add_argument("--n", type=int, default=0, help="protein / text: number of strings (0 = the workload's)")
    ap.add_argument("--Ks", type=str, default="", help="comma-separated K values (default: the workload's)")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--plain-steps", type=int, default=3, help="timed steps of the plain per-stage path")
    ap.add_argument("--autotune", action="store_true", help="autotune each join of the batch")
    ap.add_argument("--batch-eager", action="store_true",
                    help="issue the batch's work without a CUDA graph (same work; for per-kernel profilers)")
    ap.add_argument("--paths", type=str, default="batch,join,plain",
                    help="paths to time (batch = the graph-captured headline; without it the ej_join path heads "
                         "the line, e.g. for profilers that do not follow stream capture)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sample-clusters", type=int, default=100)
    return ap.parse_args()


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce(x: float, world: int, op: str) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 20 ms; summary() keeps
    the samples taken inside the marked (timed) windows."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []
        self.windows = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def mark(self, t0: float, t1: float):
        self.windows.append((t0, t1))

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.05)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons, inside = [], MAX_SM_MHZ, set(), 0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                clk, mx = float(parts[1]), float(parts[2])
            except ValueError:
                continue
            if not any(t0 - 0.025 <= ts <= t1 + 0.025 for t0, t1 in self.windows):
                continue
            inside += 1
            sm.append(clk)
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": inside}


def cpu_baseline(wl: dict, args, Ks) -> dict:
    """The oracle as it stands (single-threaded C) on a bounded sample."""
    import oracle
    oracle.build()
    ss = wl["sample"](args)
    cand, t, per_k = 0, 0.0, {}
    for K in Ks:
        p = wl["params"](K)
        t0 = time.perf_counter()
        res = oracle.join(ss.data, ss.offsets, ss.alphabet, K=K, r=p["r"], m=p["m"], z=p["z"],
                          seed=p["seed"], L=p["L"], keep_candidates=False)
        dt = time.perf_counter() - t0
        cand += res.n_candidates
        t += dt
        per_k[str(K)] = {"s": round(dt, 3), "candidates": res.n_candidates, "out": int(res.pairs.shape[0]),
                         "embed_s": round(res.t_embed, 3), "sign_s": round(res.t_sign, 3),
                         "candidates_s": round(res.t_candidates, 3), "verify_s": round(res.t_verify, 3)}
    return {"value": cand / t, "unit": "pairs/s", "cores": 1, "kind": "oracle",
            "sample": f"{ss.n} strings of the same recipe, K={','.join(map(str, Ks))}, one join each; "
                      f"{t:.1f} s single-threaded",
            "per_K": per_k}


def run_reference(args, rank, world):
    if rank != 0:
        return
    wl = workloads()[args.workload]
    Ks = tuple(int(k) for k in args.Ks.split(",")) if args.Ks else wl["Ks"]
    for _ in range(args.warmup):
        cpu_baseline(wl, args, Ks)
    total_t, total_c, last = 0.0, 0.0, None
    for _ in range(args.steps):
        t0 = time.perf_counter()
        last = cpu_baseline(wl, args, Ks)
        total_t += time.perf_counter() - t0
        total_c += sum(v["candidates"] for v in last["per_K"].values())
    value = total_c / total_t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total_t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"{args.workload} join sample: {last['sample']}", "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": 1, "kind": "oracle",
                             "sample": last["sample"]},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_serving(args, rank, world, local):
    """Search against a resident index: the query stream as one offline batch,
    then as Poisson arrivals at each offered rate through the continuous-batching
    server (p50/p99 latency and achieved queries/s per rate)."""
    import random

    import numpy as np
    import torch

    from paper_1702_00093_gb300 import embedjoin as ej
    from paper_1702_00093_gb300 import synth

    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    idx_ss = synth.serving_index(args.index_size, seed=1005 + rank)
    qs, ks = synth.serving_queries(idx_ss, args.queries, seed=1006 + rank)
    ctx = ej.Context(local)
    t0 = time.perf_counter()
    index = ej.Index(ctx, ej.Strings.from_set(idx_ss, dev), ej.Params(K=0, alphabet=idx_ss.alphabet,
                                                                      **synth.SERVING_PARAMS))
    build_s = time.perf_counter() - t0
    index.search(qs[:64], ks[:64])                        # warm-up
    t0 = time.perf_counter()
    offline = index.search(qs, ks)
    offline_s = time.perf_counter() - t0
    per_q = {}
    for v in offline:
        per_q.setdefault(int(v) >> 32, []).append(int(v) & 0xFFFFFFFF)
    rates = []
    identical = True
    with ClockSampler(local) as clk:
        for rate in [float(x) for x in args.rates.split(",") if x]:
            n = min(len(qs), max(200, int(rate * 4.0)))
            srv = ej.Server(index, max_batch=256, inflight=4)
            rnd = random.Random(7)
            done = {}
            sub = {}

            def submitter():
                t = time.perf_counter()
                for q in range(n):
                    t += rnd.expovariate(rate)
                    d = t - time.perf_counter()
                    if d > 0:
                        time.sleep(d)
                    sub[srv.submit(qs[q], int(ks[q]))] = q

            th = threading.Thread(target=submitter)
            w0 = time.time()
            th.start()
            deadline = time.time() + 120
            while len(done) < n and time.time() < deadline:
                for rid, status, matches, lat, queue in srv.poll(1024, 2000):
                    done[rid] = (status, matches, lat, queue)
            th.join()
            clk.mark(w0, time.time())
            st = srv.stats()
            srv.close()
            lats = [v[2] for v in done.values()]
            for rid, (status, matches, _, _) in done.items():
                identical &= status == 0 and list(matches) == per_q.get(sub[rid], [])
            rates.append({"offered_qps": rate, "queries": n, "completed": len(done),
                          "achieved_qps": st["queries_per_s"], "p50_ms": float(np.percentile(lats, 50)),
                          "p99_ms": float(np.percentile(lats, 99)), "mean_batch": st["mean_batch"],
                          "batches": st["batches"], "deferred": st["deferred"], "retries": st["retries"]})
    if rank == 0:
        best = max(rates, key=lambda r: r["achieved_qps"]) if rates else None
        line = {
            "metric": "queries/s (edit-similarity search against a resident index, continuous batching)",
            "value": best["achieved_qps"] if best else None, "unit": "queries/s", "n_gpus": world,
            "steps": len(rates), "warmup": 1, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"serving: index of {idx_ss.n} ACGT strings, length U[900,1100], 10% planted "
                                   f"near-duplicates; {len(qs)} queries, half mutated index strings (rate "
                                   f"U[1%,10%]), half random of length U[200,5000], K = U[1%,10%] of the length; "
                                   f"r=7, m=7, z=8, L=1000; Poisson arrivals",
                       "index_build_s": build_s, "parallelism": "single GPU"},
            "offline_batch": {"queries": len(qs), "seconds": offline_s, "queries_per_s": len(qs) / offline_s,
                              "matches": int(offline.shape[0])},
            "rates": rates, "identical_to_offline": bool(identical), "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    index.close()
    ctx.close()


def main():
    args = parse()
    rank, world, local = dist_init()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "serving":
        run_serving(args, rank, world, local)
        return
    import torch

    from paper_1702_00093_gb300 import embedjoin as ej

    assert torch.cuda.is_available(), "bench.py --impl ours needs a GPU"
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    wl = workloads()[args.workload]
    Ks = tuple(int(k) for k in args.Ks.split(",")) if args.Ks else wl["Ks"]
    ss = wl["make"](wl["seed"] + rank, args)   # an independent problem per rank
    params = []
    for K in Ks:
        p = wl["params"](K)
        params.append(ej.Params(K=K, r=p["r"], m=p["m"], z=p["z"], seed=p["seed"], L=p["L"], alphabet=ss.alphabet))
    strings = ej.Strings.from_set(ss, dev)
    ctx = ej.Context(local)
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    warm = max(args.warmup, 3)

    def timed(step, n_steps, clk):
        """n_steps of step() on `stream`, L2 flushed before each, CUDA events."""
        total = 0.0
        for _ in range(n_steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            barrier(world)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            w0 = time.time()
            e0.record(stream)
            step()
            e1.record(stream)
            torch.cuda.synchronize()
            if clk is not None:
                clk.mark(w0, time.time())
            total += e0.elapsed_time(e1)
        return total

    with torch.cuda.stream(stream), ClockSampler(local) as clk:
        paths = set(args.paths.split(","))
        use_batch = "batch" in paths
        batch_ms, cand_step, launches_step, result_pairs, e2e = None, 0, 0, None, None
        merged_ms, merged_word_cols, eager_ms, same_eager = [], 0, None, None
        if use_batch:
            # ---- headline: all joins of the step as one CUDA graph -------------------
            batch = ctx.batch(strings, params, autotune=args.autotune, stream=stream, eager=args.batch_eager)
            outs = [torch.empty(1 << 16, dtype=torch.int64, device=dev) for _ in params]
            bstats = {}

            def batch_step(b=None):
                b = b or batch
                b.run(stream)
                for i in range(len(params)):
                    while True:
                        try:
                            bstats[i] = b.result_into(i, outs[i], stream)
                            break
                        except ej.EJError as e:
                            if getattr(e, "needed", None) is None:
                                raise
                            outs[i] = torch.empty(e.needed + 1024, dtype=torch.int64, device=dev)

            for _ in range(warm):
                batch_step()
            batch_ms = timed(batch_step, args.steps, clk)
            cand_step = sum(st.n_candidates for _, st in bstats.values())
            launches_step = batch.kernel_count + sum(st.kernel_launches for _, st in bstats.values())
            result_pairs = [outs[i][:bstats[i][0]].clone() for i in range(len(params))]

            # ---- end to end through the public API with host buffers -------------------
            e2e = None
            if args.e2e_steps > 0:
                h_data = torch.from_numpy(ss.data).pin_memory()
                h_off = torch.from_numpy(ss.offsets).pin_memory()
                h_outs = [torch.empty(max(int(o.shape[0]), 1), dtype=torch.int64).pin_memory().numpy() for o in outs]
                h_t, h_cand, d2h = 0.0, 0, 0
                for it in range(args.e2e_steps + 1):
                    torch.cuda.synchronize()
                    barrier(world)
                    t0 = time.perf_counter()
                    strings.data.copy_(h_data, non_blocking=True)
                    strings.offsets.copy_(h_off, non_blocking=True)
                    batch.run(stream)
                    step_c, step_out = 0, 0
                    for i in range(len(params)):
                        n, st = batch.result_into(i, h_outs[i], stream)
                        step_c += st.n_candidates
                        step_out += n
                    dt = time.perf_counter() - t0
                    if it > 0:   # the first pass warms the host staging
                        h_t += dt
                        h_cand += step_c
                        d2h += step_out * 8
                h_t = allreduce(h_t, world, "max")
                h_cand = allreduce(h_cand, world, "sum")
                e2e = {"value": h_cand / h_t, "unit": "pairs/s",
                       "h2d_bytes_per_step": int(ss.data.nbytes + ss.offsets.nbytes),
                       "d2h_bytes_per_step": int(d2h / args.e2e_steps), "steps": args.e2e_steps,
                       "ms_per_step": 1e3 * h_t / args.e2e_steps, "api": "ej_batch_run + ej_batch_result, host buffers"}
            batch.close()   # its scratch is not needed by the other paths

            # ---- the same batch issued without a graph: times the merged verifier ----
            # launch with CUDA events on its stream (a graph replay cannot be timed
            # per kernel), for the roofline of the step's dominant kernel
            if not args.batch_eager:
                eb = ctx.batch(strings, params, autotune=args.autotune, stream=stream, eager=True)

                def eager_step():
                    batch_step(eb)
                    try:
                        merged_ms.append(eb.verify_ms())
                    except ej.EJError:
                        pass

                for _ in range(warm):
                    eager_step()
                merged_ms.clear()
                eager_ms = timed(eager_step, args.steps, clk)
                merged_word_cols = sum(st.verify_word_columns for _, st in bstats.values())
                same_eager = all(torch.equal(outs[i][:bstats[i][0]], result_pairs[i]) for i in range(len(params)))
                eb.close()

        # ---- the same step through ej_join (stage timings, verify roofline) --------
        ctx.set_timing(True)
        jout = torch.empty(1 << 16, dtype=torch.int64, device=dev)
        jstats = []

        def join_step():
            nonlocal jout
            for p in params:
                while True:
                    try:
                        n, st = ctx.join_into(strings, p, jout, stream)
                        break
                    except ej.EJError as e:
                        if e.status != ej.EJ_ERR_CAPACITY:
                            raise
                        jout = torch.empty(e.needed + 1024, dtype=torch.int64, device=dev)
                jstats.append((p.K, n, st.as_dict()))

        for _ in range(warm):
            join_step()
        jstats.clear()
        join_ms = timed(join_step, args.steps, None if use_batch else clk)
        same_join = True
        join_pairs = []
        for i, p in enumerate(params):
            n, _ = ctx.join_into(strings, p, jout, stream)
            join_pairs.append(jout[:n].clone())
        if use_batch:
            same_join = all(torch.equal(a, b) for a, b in zip(join_pairs, result_pairs))
        else:
            # the ej_join path heads the line
            result_pairs = join_pairs
            batch_ms = join_ms
            cand_step = sum(s_["n_candidates"] for _, _, s_ in jstats) // args.steps
            launches_step = sum(s_["kernel_launches"] for _, _, s_ in jstats) // args.steps

        plain_ms, same_plain, cand_plain = None, None, 0
        if "plain" in paths:
            # ---- the plain per-stage path (on a fresh context) --------------------------
            ctx.close()
            ctx = ej.Context(local)
            plain = [dataclasses.replace(p, out_len=p.L) for p in params]   # the walk is causal: prefix L
            infos = [ctx.plan(strings, p, stream) for p in plain]
            emb = torch.empty(max(i.embedding_bytes for i in infos) // 4 + 1, dtype=torch.int32, device=dev)
            we = torch.empty(max(i.walk_end_count for i in infos) + 1, dtype=torch.int32, device=dev)
            keys = torch.empty(max(i.key_count for i in infos) + 1, dtype=torch.int64, device=dev)
            cand_buf = torch.empty(1 << 16, dtype=torch.int64, device=dev)
            pout = torch.empty(1 << 16, dtype=torch.int64, device=dev)
            plain_res = {}

            def plain_step():
                nonlocal cand_buf, pout
                for i, p in enumerate(plain):
                    ctx.embed(strings, p, emb, we, stream)
                    ctx.sign(strings, p, emb, we, keys, stream)
                    while True:
                        try:
                            nc, _ = ctx.lsh_candidates(strings, p, keys, cand_buf, stream)
                            break
                        except ej.EJError as e:
                            if e.status != ej.EJ_ERR_CAPACITY:
                                raise
                            cand_buf = torch.empty(e.needed + 1024, dtype=torch.int64, device=dev)
                            pout = torch.empty(e.needed + 1024, dtype=torch.int64, device=dev)
                    k = ctx.verify(strings, p, cand_buf[:nc], pout, stream)
                    plain_res[i] = (nc, pout[:k].clone())

            plain_step()
            plain_ms = timed(plain_step, args.plain_steps, None)
            same_plain = all(torch.equal(plain_res[i][1], result_pairs[i]) for i in range(len(params)))
            cand_plain = sum(plain_res[i][0] for i in range(len(params)))
    clocks = clk.summary()

    batch_ms_max = allreduce(batch_ms, world, "max")
    value = allreduce(cand_step * args.steps, world, "sum") / (batch_ms_max / 1e3)

    # verify kernel roofline, from the ej_join pass (events around each verify launch)
    verify_ms = sum(s["ms_verify"] for _, _, s in jstats)
    word_cols = sum(s["verify_word_columns"] for _, _, s in jstats)
    n_verify = sum(1 for _, _, s in jstats if s["n_candidates"] > 0)
    ach_ops = word_cols * INT_OPS_PER_WORD_COLUMN / (verify_ms / 1e3) if verify_ms else 0.0
    peak_ops = SMS * ALU_LANES_PER_SM * MAX_SM_MHZ * 1e6
    per_k = {}
    for K in Ks:
        rows = [s for k, _, s in jstats if k == K]
        per_k[str(K)] = {
            "join_ms": statistics.mean(s["ms_total"] for s in rows),
            "prepare_ms": statistics.mean(s["ms_prepare"] for s in rows),
            "embed_sign_ms": statistics.mean(s["ms_embed_sign"] for s in rows),
            "candidates_ms": statistics.mean(s["ms_candidates"] for s in rows),
            "verify_ms": statistics.mean(s["ms_verify"] for s in rows),
            "candidates": rows[0]["n_candidates"], "raw_pairs": rows[0]["n_raw_pairs"],
            "out_pairs": rows[0]["n_out"], "max_bucket": rows[0]["max_bucket"],
            "band_cells": rows[0]["band_cells"],
        }
    cells_step = sum(v["band_cells"] for v in per_k.values())
    join_roofline = {"kernel": "the verifier of ej_join, one launch per join (persistent verify_pq_kernel for "
                               "mean string length >= 2048, else grid-strided verify_bd_kernel)", "bound": "alu",
                     "achieved": ach_ops / 1e12, "peak": peak_ops / 1e12, "unit": "Tops/s (32-bit integer ops)",
                     "frac": ach_ops / peak_ops, "traffic": verify_traffic("join"),
                     "launches": n_verify, "avg_launch_ms": verify_ms / max(n_verify, 1),
                     "ops_per_word_column": INT_OPS_PER_WORD_COLUMN, "word_columns": word_cols,
                     "measured_in": "the ej_join pass (CUDA events around each verify launch, its stream)",
                     "peak_basis": "integer ALU pipe: 152 SMs x 64 lanes/clock x 2070 MHz (derived)"}
    roofline = join_roofline
    if merged_ms:
        m_ms = statistics.mean(merged_ms)
        m_ops = merged_word_cols * INT_OPS_PER_WORD_COLUMN / (m_ms / 1e3)
        roofline = {"kernel": "verify_pq_kernel (the batch's merged launch over all joins' candidates)",
                    "bound": "alu", "achieved": m_ops / 1e12, "peak": peak_ops / 1e12,
                    "unit": "Tops/s (32-bit integer ops)", "frac": m_ops / peak_ops,
                    "traffic": verify_traffic("merged"), "launches": len(merged_ms), "avg_launch_ms": m_ms,
                    "ops_per_word_column": INT_OPS_PER_WORD_COLUMN, "word_columns": merged_word_cols,
                    "word_columns_basis": "columns advanced x 64-bit words of each join's own band",
                    "measured_in": "the batch issued without a graph (same kernels), timed steps: CUDA events "
                                   "around the merged launch, on its stream",
                    "peak_basis": "integer ALU pipe: 152 SMs x 64 lanes/clock x 2070 MHz (derived)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": warm, "ms_per_step": batch_ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"{wl['desc'](ss, args)}; K={','.join(map(str, Ks))}; "
                                   f"r={params[0].r}, m={params[0].m}, z={'/'.join(str(p.z) for p in params)}, "
                                   f"L={params[0].L}; one step = one join per K" +
                                   (", the joins of a step captured as one CUDA graph (ej_batch)" if use_batch
                                    else ", one ej_join call per K"),
                       "n": ss.n, "Ks": list(Ks), "l2": "flushed before each timed step (256 MiB write)",
                       "parallelism": "replicas" if world > 1 else "single GPU", "autotune": args.autotune},
            "join_wall_s_per_step": batch_ms_max / args.steps / 1e3,
            "band_cells_per_s": allreduce(cells_step * args.steps, world, "sum") / (batch_ms_max / 1e3),
            "join_path": {"value": cand_step * args.steps / (join_ms / 1e3), "ms_per_step": join_ms / args.steps,
                          "api": "ej_join per K", "identical_output": bool(same_join)},
            "plain_path": None if plain_ms is None else {
                "value": cand_plain * args.plain_steps / (plain_ms / 1e3), "ms_per_step": plain_ms / args.plain_steps,
                "steps": args.plain_steps, "api": "ej_embed -> ej_sign -> ej_lsh_candidates -> ej_verify per K",
                "identical_output": bool(same_plain)},
            "eager_batch_path": None if eager_ms is None else {
                "ms_per_step": eager_ms / args.steps, "value": cand_step * args.steps / (eager_ms / 1e3),
                "api": "ej_batch with EJ_BATCH_EAGER (the same work issued every step without a graph)",
                "identical_output": bool(same_eager)},
            "per_K": per_k,
            "roofline": roofline,
            "join_path_roofline": join_roofline,
            "clocks": clocks,
            "gpu_launches": int(launches_step * args.steps),
            "e2e": e2e,
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(wl, args, Ks)
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
