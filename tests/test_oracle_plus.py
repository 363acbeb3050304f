"""Pins of the oracle's EmbedJoin+ (Section 5, Algorithms 4 and 5).

- With one substring per string and T = 1 it is EmbedJoin (Section 5 states
  that EmbedJoin+ degenerates to EmbedJoin then): same candidates, same output.
- Its candidate set equals the set definition computed by brute force from the
  signatures of every suffix: pairs within K in length with some substring pair
  that matches in at least T tables.
- The chance that a substring pair gets at least T matched signatures follows
  the binomial p_T of Section 5 when the per-table collision probability is p
  (fixed walks, sampled positions drawn afresh).
- On strings shifted by an inserted prefix (the case Section 5 is built for)
  it finds pairs that plain EmbedJoin misses."""
import itertools
import math

import numpy as np

import oracle
from paper_1702_00093_gb300 import synth


def _suffix_set(ss, S, delta):
    """Every string's substrings s[(k-1)delta:] for k = 1..S, string-major."""
    out = []
    for i in range(ss.n):
        s = ss.get(i)
        for k in range(S):
            out.append(s[min(k * delta, len(s)):])
    return synth.pack(out, ss.alphabet)


def test_one_substring_and_T1_is_embedjoin():
    for ss, K, r, m, z, L in [(synth.small_dna(scale=0.3), 6, 3, 10, 12, 0),
                              (synth.protein_like(4, 300, median=120, lo=20, hi=400), 12, 4, 6, 6, 240),
                              (synth.dna_clusters(3, 12, 6, 30, 60, edits_mean=3.0), 0, 2, 5, 4, 0)]:
        a = oracle.join(ss.data, ss.offsets, ss.alphabet, K=K, r=r, m=m, z=z, seed=2, L=L)
        b = oracle.join_plus(ss.data, ss.offsets, ss.alphabet, K=K, r=r, m=m, z=z, seed=2, L=L,
                             delta=max(K, 1), T=1)
        assert oracle.plus_substrings(K, max(K, 1)) == 1 and b.T == 1
        assert b.n_candidates == a.n_candidates and np.array_equal(b.candidates, a.candidates)
        assert np.array_equal(b.pairs, a.pairs)
        assert a.n_candidates > 0


def test_candidates_equal_the_set_definition():
    for seed, (K, delta, T, alphabet) in enumerate([(8, 3, 2, b"ACGT"), (8, 3, 1, b"ACGT"), (10, 4, 2, b"ACGT"),
                                                   (12, 5, 3, synth.TEXT)]):
        rng = np.random.default_rng(seed)
        lut = np.frombuffer(alphabet, np.uint8)
        sigma = len(alphabet)
        strs = []
        for _ in range(8):
            b = rng.integers(0, sigma, size=int(rng.integers(10, 40))).astype(np.uint8)
            for _ in range(5):
                c = synth.mutate(rng, b, int(rng.integers(0, 4)), sigma)
                pre = rng.integers(0, sigma, size=int(rng.integers(0, 6))).astype(np.uint8)
                strs.append(lut[np.concatenate([pre, c])].tobytes())
        ss = synth.pack(strs, alphabet)
        r, m, z = 2, 3, 3
        L = 2 * int(ss.lengths().max())
        res = oracle.join_plus(ss.data, ss.offsets, alphabet, K=K, r=r, m=m, z=z, seed=seed, L=L,
                               out_len=3 * int(ss.lengths().max()), delta=delta, T=T)
        S = oracle.plus_substrings(K, delta)
        sfx = _suffix_set(ss, S, delta)
        keys = oracle.keys(sfx.data, sfx.offsets, alphabet, r, m, z, L, seed).reshape(r * m, ss.n, S)
        lens = ss.lengths()
        want = []
        for a, b in itertools.combinations(range(ss.n), 2):
            if abs(int(lens[a]) - int(lens[b])) > K:
                continue
            counts = (keys[:, a, :, None] == keys[:, b, None, :]).sum(axis=0)   # [S][S]
            if counts.max() >= T:
                want.append((a << 32) | b)
        assert np.array_equal(res.candidates, np.array(want, dtype=np.uint64)), (K, delta, T)
        assert len(want) > 10


def _p_T(m, p, T):
    return 1.0 - sum(math.comb(m, i) * p ** i * (1 - p) ** (m - i) for i in range(T))


def test_matched_signature_threshold_follows_binomial_p_T():
    # two strings with fixed walks (explicit random bits); the m sampled
    # positions of each function are drawn afresh, uniformly from [0, L)
    rng = np.random.default_rng(11)
    lut = np.frombuffer(b"ACGT", np.uint8)
    x = lut[rng.integers(0, 4, size=60)].tobytes()
    y = bytearray(x)
    y[40] = int(lut[(b"ACGT".index(x[40]) + 1) % 4])    # one edit: the walks agree on a long prefix
    y = bytes(y)
    ss = synth.pack([x, y], b"ACGT")
    L, z, m = 120, 4, 6
    bits = np.array([[[oracle.walk_bit(5, 0, j, c) for c in b"ACGT"] for j in range(L)]], dtype=np.uint8)
    emb, we = oracle.embed(ss.data, ss.offsets, b"ACGT", 1, L, 5, pi_inject=bits)
    h = int((emb[0, 0] != emb[0, 1]).sum())
    p = (1.0 - h / L) ** z
    assert 0.3 < p < 0.8
    draws = 1500
    for T in (2, 4, 6):
        hits = 0
        for d in range(draws):
            pos = rng.integers(0, L, size=(1, m, z)).astype(np.uint32)
            res = oracle.join_plus(ss.data, ss.offsets, b"ACGT", K=60, r=1, m=m, z=z, seed=5, L=L, out_len=L,
                                   delta=60, T=T, pi_inject=bits, pos_inject=pos)
            hits += res.n_candidates
        want = _p_T(m, p, T)
        sd = math.sqrt(want * (1 - want) / draws)
        assert abs(hits / draws - want) < 4 * sd + 1e-9, (T, hits / draws, want)


def test_shifted_pairs_found_by_plus_and_missed_by_plain():
    # y = an inserted prefix of 15-30 symbols + x with a few edits: the shift
    # that Section 5 says plain EmbedJoin's walks do not absorb
    rng = np.random.default_rng(3)
    lut = np.frombuffer(b"ACGT", np.uint8)
    strs = []
    for _ in range(40):
        x = rng.integers(0, 4, size=400).astype(np.uint8)
        y = np.concatenate([rng.integers(0, 4, size=int(rng.integers(15, 31))).astype(np.uint8),
                            synth.mutate(rng, x, 3, 4)])
        strs += [lut[x].tobytes(), lut[y].tobytes()]
    ss = synth.pack(strs, b"ACGT")
    K, r, m, z, L = 40, 7, 16, 12, 400
    truth = {(2 * i) << 32 | (2 * i + 1) for i in range(40)}
    assert all(oracle.ed_banded(ss.get(2 * i), ss.get(2 * i + 1), K) <= K for i in range(40))
    plain = oracle.join(ss.data, ss.offsets, b"ACGT", K=K, r=r, m=m, z=z, seed=1, L=L)
    plus = oracle.join_plus(ss.data, ss.offsets, b"ACGT", K=K, r=r, m=m, z=z, seed=1, L=L, delta=10)
    rec_plain = len(truth & set(plain.pairs.tolist())) / len(truth)
    rec_plus = len(truth & set(plus.pairs.tolist())) / len(truth)
    assert plus.T == 2
    assert rec_plus >= 0.8 and rec_plus >= rec_plain + 0.3, (rec_plain, rec_plus)
