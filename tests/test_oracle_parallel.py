"""The process-parallel drivers of the oracle give exactly the single-threaded
oracle's results: keys over string ranges, verification over pair chunks, the
composed join, and the per-string expected pairs used for sampled checks of
full-size workloads."""
import numpy as np

import oracle
from oracle import parallel
from paper_1702_00093_gb300 import synth


def test_parallel_keys_and_join_equal_single_process():
    ss = synth.small_dna(scale=0.3)
    p = dict(K=6, r=3, m=10, z=12, seed=1)
    L = 3 * int(ss.lengths().max())
    want_k = oracle.keys(ss.data, ss.offsets, ss.alphabet, p["r"], p["m"], p["z"], L, p["seed"])
    got_k = parallel.keys(ss.data, ss.offsets, ss.alphabet, p["r"], p["m"], p["z"], L, p["seed"], procs=2)
    assert np.array_equal(got_k, want_k)
    ref = oracle.join(ss.data, ss.offsets, ss.alphabet, **p)
    pairs, nc = parallel.join(ss.data, ss.offsets, ss.alphabet, L=L, procs=2, **p)
    assert nc == ref.n_candidates and np.array_equal(pairs, ref.pairs)
    flags = parallel.verify(ss.data, ss.offsets, ref.candidates, 6, procs=2, cutoff=False)
    assert np.array_equal(flags, oracle.verify(ss.data, ss.offsets, ref.candidates, 6))


def test_expected_pairs_of_sampled_strings_equal_the_join_restricted_to_them():
    ss = synth.protein_like(5, 400, median=120, lo=20, hi=400)
    L = int(2 * ss.lengths().mean())
    K, r, m, z, seed = 12, 4, 6, 6, 3
    ref = oracle.join(ss.data, ss.offsets, ss.alphabet, K=K, r=r, m=m, z=z, seed=seed, L=L,
                      out_len=max(L, 3 * int(ss.lengths().max())))
    keys = oracle.keys(ss.data, ss.offsets, ss.alphabet, r, m, z, L, seed)
    rng = np.random.default_rng(2)
    ids = sorted(set(rng.integers(0, ss.n, size=12).tolist()) | {int(ref.pairs[0] >> 32)})
    got = parallel.expected_pairs_of(ss.data, ss.offsets, keys, K, ids, procs=1)
    assert np.array_equal(got, parallel.pairs_of(ref.pairs, ids))
    assert got.shape[0] > 0
