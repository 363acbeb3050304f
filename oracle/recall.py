"""Recall of EmbedJoin against the brute-force join (Section 1's definition), on
seeded samples of each workload. The method's pair set comes from the oracle's
join (Alg. 3 with Alg. 2; the GPU path is bit-identical to it). The true pair
set is every pair with ED <= K, from the brute-force join with the cutoff DP.
Test infrastructure: it calls only the oracle and the seeded input generators.

    python -m oracle.recall            # one JSON line per (workload, K), then serving
    python -m oracle.recall --write    # the same, also written to oracle/recall_samples.json
    python -m oracle.recall --sweep-z  # long DNA and text-like: recall and candidates per z
"""
import json
import os
import sys
import time

import oracle
from paper_1702_00093_gb300 import synth


def samples():
    """(name, string set, Ks, params(K)) for every join workload, at sizes the
    brute force finishes in seconds."""
    small = synth.SMALL_DNA_PARAMS
    yield ("small_dna", "small DNA, n=1000 (the full workload)", synth.small_dna(), [small["K"]],
           lambda K: dict(r=small["r"], m=small["m"], z=small["z"], seed=small["seed"], L=0))
    yield ("long_dna", "long DNA, 20 clusters of 10 (n=200)", synth.long_dna(n_clusters=20, seed=1002),
           [50, 150, 250], synth.long_dna_params)
    yield ("protein", "protein-like, n=1000", synth.protein_like(1003, 1000), list(synth.PROTEIN_KS),
           synth.protein_params)
    yield "text", "text-like, n=300", synth.text_like(1004, 300), list(synth.TEXT_KS), synth.text_params


def serving_recall(n_index: int = 2000, n_queries: int = 100):
    """Search against an index (the serving workload's recipe at a small size): the
    method's matches (each query walked and signed with the index's tables, index
    strings sharing a key in some table within K_q of the query's length, exact
    ED <= K_q) against every index string within K_q by the cutoff DP."""
    import numpy as np
    prm = synth.SERVING_PARAMS
    idx = synth.serving_index(n_index, seed=1005)
    qs, ks = synth.serving_queries(idx, n_queries, seed=1006)
    n = idx.n
    allset = synth.pack([idx.get(i) for i in range(n)] + list(qs), idx.alphabet)
    emb, we = oracle.embed(allset.data, allset.offsets, allset.alphabet, prm["r"], prm["L"], prm["seed"])
    pos = oracle.positions(prm["seed"], prm["r"], prm["m"], prm["z"], prm["L"])
    keys = oracle.sign(emb, we, pos, len(allset.alphabet))
    lens = allset.lengths()
    got, want = set(), set()
    for q in range(len(qs)):
        K = int(ks[q])
        near = np.nonzero(np.abs(lens[:n] - lens[n + q]) <= K)[0]
        hit = np.zeros(n, dtype=bool)
        for t in range(keys.shape[0]):
            hit |= keys[t, :n] == keys[t, n + q]
        for i in near:
            if oracle.ed_banded_cutoff(qs[q], idx.get(int(i)), K) <= K:
                want.add((q, int(i)))
                if hit[i]:
                    got.add((q, int(i)))
    found = len(got)
    row = {"key": "serving", "workload": f"serving search, index n={n}, {len(qs)} queries", "K": "per query",
           "n": n, "true_pairs": len(want), "found": found, "recall": found / len(want) if want else None,
           "precision": 1.0}
    print(json.dumps(row), flush=True)
    return row


def sweep_z():
    """Recall and candidate count of the long-DNA and text-like samples for each
    number of samples per function z (r, m, L and the seed as in the workload)."""
    for _, name, ss, Ks, params in list(samples())[1::2]:
        for K in Ks:
            truth = set(oracle.join_bruteforce(ss.data, ss.offsets, K, cutoff=True).tolist())
            p = params(K)
            for z in range(max(2, p["z"] - 8), p["z"] + 1):
                res = oracle.join(ss.data, ss.offsets, ss.alphabet, K=K, r=p["r"], m=p["m"], z=z, seed=p["seed"],
                                  L=p.get("L", 0), keep_candidates=False)
                found = len(set(res.pairs.tolist()) & truth)
                print(json.dumps({"workload": name, "K": K, "z": z, "paper_rule_z": p["z"], "true_pairs": len(truth),
                                  "found": found, "recall": found / len(truth) if truth else None,
                                  "candidates": res.n_candidates}), flush=True)


def main():
    oracle.build()
    if "--sweep-z" in sys.argv:
        sweep_z()
        return
    rows = []
    for key, name, ss, Ks, params in samples():
        for K in Ks:
            p = params(K)
            t0 = time.perf_counter()
            res = oracle.join(ss.data, ss.offsets, ss.alphabet, K=K, r=p["r"], m=p["m"], z=p["z"], seed=p["seed"],
                              L=p.get("L", 0), keep_candidates=False)
            t1 = time.perf_counter()
            truth = oracle.join_bruteforce(ss.data, ss.offsets, K, cutoff=True)
            t2 = time.perf_counter()
            got, want = set(res.pairs.tolist()), set(truth.tolist())
            found = len(got & want)
            row = {"key": key, "workload": name, "K": K, "n": ss.n, "true_pairs": len(want), "found": found,
                   "recall": found / len(want) if want else None, "precision": found / len(got) if got else None,
                   "candidates": res.n_candidates, "join_s": round(t1 - t0, 2), "bruteforce_s": round(t2 - t1, 2)}
            rows.append(row)
            print(json.dumps(row), flush=True)
    rows.append(serving_recall())
    if "--write" in sys.argv:
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "recall_samples.json")
        with open(path, "w") as f:
            json.dump({"written_by": "python -m oracle.recall --write", "rows": rows}, f, indent=1)
            f.write("\n")


if __name__ == "__main__":
    main()
