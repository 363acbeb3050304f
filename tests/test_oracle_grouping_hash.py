"""Pins of the oracle's fidelity options of Section 4: the two-level hash
<u, v> mod P of a signature in place of the exact key, and grouping by length
(Section 4.1) in place of truncation."""
import math

import numpy as np

import oracle
from paper_1702_00093_gb300 import synth


def _embed(ss, r, out_len, seed):
    return oracle.embed(ss.data, ss.offsets, ss.alphabet, r, out_len, seed)


def test_one_sample_per_function_hash_is_the_exact_key():
    # u -> u * v mod P is one-to-one for v != 0 and u < P: with z = 1 the
    # hashed buckets are the exact ones
    ss = synth.small_dna(scale=0.3)
    P = 1000003
    assert all(oracle.hash_coefficient(4, l, f, 0, P) != 0 for l in range(3) for f in range(10))
    a = oracle.join(ss.data, ss.offsets, ss.alphabet, K=6, r=3, m=10, z=1, seed=4)
    b = oracle.join(ss.data, ss.offsets, ss.alphabet, K=6, r=3, m=10, z=1, seed=4, key_P=P)
    assert np.array_equal(a.candidates, b.candidates) and np.array_equal(a.pairs, b.pairs)


def test_hashed_candidates_contain_the_exact_ones():
    for seed, P in [(1, 1000003), (2, 101), (3, 13)]:
        ss = synth.dna_clusters(seed, 20, 6, 40, 80, edits_mean=3.0)
        a = oracle.join(ss.data, ss.offsets, ss.alphabet, K=5, r=2, m=4, z=6, seed=seed)
        b = oracle.join(ss.data, ss.offsets, ss.alphabet, K=5, r=2, m=4, z=6, seed=seed, key_P=P)
        assert set(a.candidates.tolist()) <= set(b.candidates.tolist())
        assert set(a.pairs.tolist()) <= set(b.pairs.tolist())
        if P < 1000:
            assert b.n_candidates > a.n_candidates
        truth = set(oracle.join_bruteforce(ss.data, ss.offsets, 5).tolist())
        assert set(b.pairs.tolist()) <= truth


def test_distinct_signatures_collide_at_one_over_P():
    # equal signatures always share the hashed key; distinct ones share it with
    # probability 1/P over the random vector v
    rng = np.random.default_rng(2)
    lut = np.frombuffer(b"ACGT", np.uint8)
    ss = synth.pack([lut[rng.integers(0, 4, size=30)].tobytes() for _ in range(120)], b"ACGT")
    P, r, m, z, L = 101, 4, 12, 4, 60
    emb, we = _embed(ss, r, L, 9)
    pos = oracle.positions(9, r, m, z, L)
    exact = oracle.sign(emb, we, pos, 4)
    hashed = oracle.sign_modp(emb, we, pos, 4, 9, P)
    same, coll, distinct = 0, 0, 0
    for t in range(r * m):
        e, h = exact[t], hashed[t]
        eq_e = e[:, None] == e[None, :]
        eq_h = h[:, None] == h[None, :]
        iu = np.triu_indices(ss.n, 1)
        assert np.all(eq_h[iu][eq_e[iu]])
        distinct += int((~eq_e[iu]).sum())
        coll += int((eq_h[iu] & ~eq_e[iu]).sum())
    rate = coll / distinct
    sd = math.sqrt((1 / P) * (1 - 1 / P) / distinct)
    assert distinct > 100000
    # the pairs of one table are not independent; allow a wider margin
    assert abs(rate - 1 / P) < 8 * sd + 0.002, rate


def test_groups_cover_every_pair_within_K():
    for N in (1, 5, 37, 100, 101):
        for K in (1, 2, 7, 40, 150):
            G = oracle.group_count(N, K)
            assert G >= 1
            for a in range(N + 1):
                member = [g for g in range(1, G + 1) if oracle.in_group(a, g, K)]
                assert 1 <= len(member) <= 2, (N, K, a, member)
                for b in range(a, min(N, a + K) + 1):
                    assert any(oracle.in_group(b, g, K) for g in member), (N, K, a, b)


def test_one_group_is_embedjoin():
    ss = synth.small_dna(scale=0.2)
    K = int(ss.lengths().max())      # K >= N: a single group
    pairs, nc = oracle.join_grouped(ss.data, ss.offsets, ss.alphabet, K=K, r=2, m=6, z=8, seed=3)
    ref = oracle.join(ss.data, ss.offsets, ss.alphabet, K=K, r=2, m=6, z=8, seed=3)
    assert oracle.group_count(int(ss.lengths().max()), K) == 1
    assert nc == ref.n_candidates and np.array_equal(pairs, ref.pairs)


def test_grouped_join_is_precise_and_finds_most_pairs():
    ss = synth.dna_clusters(5, 30, 8, 40, 120, edits_mean=2.0)
    pairs, nc = oracle.join_grouped(ss.data, ss.offsets, ss.alphabet, K=4, r=3, m=8, z=8, seed=1)
    truth = set(oracle.join_bruteforce(ss.data, ss.offsets, 4).tolist())
    got = set(pairs.tolist())
    assert got <= truth and len(got) >= 0.8 * len(truth) and nc >= len(got)
