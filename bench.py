#!/usr/bin/env python3
"""Benchmark of the EmbedJoin hot path on one GPU (or N independent replicas).

Workload (long DNA-like strings): n = 20000 strings over {A,C,G,T}, 2000
clusters of 10, base length uniform in [4500, 5500], each member carrying
Poisson(rate * length) random edits with rate uniform in [1%, 8%]. One step =
the whole join (validate -> random tables -> CGK embed -> sign -> sort/bucket/
dedup -> verify -> compact) at K = 50, 150 and 250 (r = 7, m = 20 functions,
z = 15/14/13 positions, L = 5000), inputs resident in HBM.

Metric: candidate pairs verified per second of whole-join wall time (the
"verified pairs/s" of the headline metric; join wall time and band cells/s are
reported beside it). The L2 cache is flushed (256 MiB write) before every timed
step, outside the timed events.

--impl reference times the CPU oracle (plain single-threaded C) on a bounded
sample of the same workload (1000 strings = 100 clusters), the same metric.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

KS = (50, 150, 250)
METRIC = "verified pairs/s (candidate pairs verified per second of whole-join wall time)"
# GB300: 152 SMs; the integer ALU pipe (add, logic, shift) retires 16 lanes per clock
# per SM sub-partition, 64 per SM, at up to 2070 MHz
SMS, ALU_LANES_PER_SM, MAX_SM_MHZ = 152, 64, 2070.0
INT_OPS_PER_WORD_COLUMN = 26   # 32-bit ops of one 64-bit word of the bit-parallel step
# DRAM bytes per verify launch (dram__bytes_read.sum + dram__bytes_write.sum, mean
# over the K=50/150/250 launches of one ncu capture of this workload), valid only
# while the verify source is the one that was captured
VERIFY_TRAFFIC = {"source_sha256_prefix": "65da4c7da4e3b0fd", "bytes_per_launch": 8193621}


def verify_traffic():
    import hashlib
    src = os.path.join(ROOT, "paper_1702_00093_gb300", "csrc", "ej_verify.cu")
    with open(src, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()
    if sha.startswith(VERIFY_TRAFFIC["source_sha256_prefix"]):
        return VERIFY_TRAFFIC["bytes_per_launch"]
    return None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--clusters", type=int, default=2000, help="clusters of 10 strings")
    ap.add_argument("--Ks", type=str, default="50,150,250")
    ap.add_argument("--e2e-steps", type=int, default=3)
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


def allreduce_max(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def params_for(K: int, ej, alphabet: bytes):
    from paper_1702_00093_gb300 import synth
    p = synth.long_dna_params(K)
    return ej.Params(K=K, r=p["r"], m=p["m"], z=p["z"], seed=p["seed"], L=p["L"], alphabet=alphabet)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], MAX_SM_MHZ, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(sample_clusters: int, Ks) -> dict:
    """The oracle as it stands (single-threaded C) on a bounded sample."""
    import oracle
    from paper_1702_00093_gb300 import synth
    oracle.build()
    ss = synth.long_dna(n_clusters=sample_clusters, seed=1002)
    cand = 0
    t = 0.0
    per_k = {}
    for K in Ks:
        p = synth.long_dna_params(K)
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
            "sample": f"{ss.n} strings ({sample_clusters} clusters of 10) of the same recipe, "
                      f"K={','.join(map(str, Ks))}, one join each; {t:.1f} s single-threaded",
            "per_K": per_k}


def run_reference(args, rank, world):
    if rank != 0:
        return
    Ks = tuple(int(k) for k in args.Ks.split(","))
    for _ in range(args.warmup):
        cpu_baseline(args.sample_clusters, Ks)
    vals = []
    total_t, total_c = 0.0, 0.0
    last = None
    for _ in range(args.steps):
        t0 = time.perf_counter()
        last = cpu_baseline(args.sample_clusters, Ks)
        dt = time.perf_counter() - t0
        total_t += dt
        total_c += last["value"] * sum(v["s"] for v in last["per_K"].values())
        vals.append(dt)
    value = total_c / total_t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total_t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"long DNA-like join sample: {last['sample']}",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": 1, "kind": "oracle",
                             "sample": last["sample"]},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_init()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch

    from paper_1702_00093_gb300 import embedjoin as ej
    from paper_1702_00093_gb300 import synth

    assert torch.cuda.is_available(), "bench.py --impl ours needs a GPU"
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    Ks = tuple(int(k) for k in args.Ks.split(","))
    ss = synth.long_dna(n_clusters=args.clusters, seed=1002 + rank)   # independent problem per rank
    params = [params_for(K, ej, ss.alphabet) for K in Ks]
    strings = ej.Strings.from_set(ss, dev)
    ctx = ej.Context(local)
    ctx.set_timing(True)
    out = torch.empty(1 << 16, dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step(collect=None):
        nonlocal out
        for p in params:
            while True:
                try:
                    n, st = ctx.join_into(strings, p, out)
                    break
                except ej.EJError as e:
                    if e.status != ej.EJ_ERR_CAPACITY:
                        raise
                    out = torch.empty(e.needed + 1024, dtype=torch.int64, device=dev)
            if collect is not None:
                collect.append((p.K, n, st.as_dict()))

    warm = max(args.warmup, 3)       # at least three untimed steps
    for _ in range(warm):
        step()
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    total_ms = 0.0
    stats = []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            barrier(world)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(stats)
            e1.record(stream)
            torch.cuda.synchronize()
            total_ms += e0.elapsed_time(e1)
    clocks = clk.summary()
    total_ms_max = allreduce_max(total_ms, world)
    cand_local = sum(s["n_candidates"] for _, _, s in stats)
    cand_all = allreduce_sum(cand_local, world)
    value = cand_all / (total_ms_max / 1e3)

    # verify kernel roofline (integer ALU, issue-slot ceiling)
    verify_ms = sum(s["ms_verify"] for _, _, s in stats)
    word_cols = sum(s["verify_word_columns"] for _, _, s in stats)
    cells = sum(s["band_cells"] for _, _, s in stats)
    n_verify = sum(1 for _, _, s in stats if s["n_candidates"] > 0)
    ach_ops = word_cols * INT_OPS_PER_WORD_COLUMN / (verify_ms / 1e3) if verify_ms else 0.0
    peak_ops = SMS * ALU_LANES_PER_SM * MAX_SM_MHZ * 1e6
    per_k = {}
    for K in Ks:
        rows = [s for k, _, s in stats if k == K]
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

    # end to end through the C ABI with host buffers (pinned), copies inside
    e2e = None
    if args.e2e_steps > 0:
        h_data = torch.from_numpy(ss.data).pin_memory()
        h_off = torch.from_numpy(ss.offsets).pin_memory()
        hs = ej.Strings(h_data.numpy(), h_off.numpy())
        h_out = torch.empty(out.shape[0], dtype=torch.int64).pin_memory().numpy()
        h_cand, h_t, d2h = 0, 0.0, 0
        for it in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            barrier(world)
            t0 = time.perf_counter()
            step_c, step_out = 0, 0
            for p in params:
                n, st = ctx.join_into(hs, p, h_out)
                step_c += st.n_candidates
                step_out += n
            dt = time.perf_counter() - t0
            if it > 0:   # first pass warms the staging buffers
                h_t += dt
                h_cand += step_c
                d2h += step_out * 8
        h_t = allreduce_max(h_t, world)
        h_cand = allreduce_sum(h_cand, world)
        steps_e = args.e2e_steps
        e2e = {"value": h_cand / h_t, "unit": "pairs/s",
               "h2d_bytes_per_step": int(len(Ks) * (ss.data.nbytes + ss.offsets.nbytes)),
               "d2h_bytes_per_step": int(d2h / steps_e), "steps": steps_e,
               "ms_per_step": 1e3 * h_t / steps_e}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": warm, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"long DNA-like self-join: n={ss.n} over ACGT, {args.clusters} clusters of 10, "
                                   f"length U[4500,5500], member edit rate U[1%,8%]; K={','.join(map(str, Ks))}; "
                                   f"r=7, m=20, z=15/14/13, L=5000; one step = one join per K",
                       "n": ss.n, "Ks": list(Ks), "l2": "flushed before each timed step (256 MiB write)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "join_wall_s_per_step": total_ms_max / args.steps / 1e3,
            "band_cells_per_s": allreduce_sum(cells, world) / (total_ms_max / 1e3),
            "per_K": per_k,
            "roofline": {"kernel": "verify_bd_kernel", "bound": "alu", "achieved": ach_ops / 1e12,
                         "peak": peak_ops / 1e12, "unit": "Tops/s (32-bit integer ops)",
                         "frac": ach_ops / peak_ops, "traffic": verify_traffic(),
                         "launches": n_verify, "avg_launch_ms": verify_ms / max(n_verify, 1),
                         "ops_per_word_column": INT_OPS_PER_WORD_COLUMN,
                         "word_columns": word_cols,
                         "peak_basis": "integer ALU pipe: 152 SMs x 64 lanes/clock x 2070 MHz (derived)"},
            "clocks": clocks,
            "gpu_launches": int(sum(s["kernel_launches"] for _, _, s in stats)),
            "e2e": e2e,
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.sample_clusters, Ks)
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
