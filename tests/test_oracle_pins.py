"""Pins of the CPU oracle against values fixed by the paper and by mathematics.

None of these checks re-types the oracle's own formulas: they use the paper's
printed examples (Section 1 and Section 4, Tables 2-4), the published
SplitMix64 outputs, edit distances found by enumerating edit neighbourhoods,
closed-form LSH collision probabilities (Theorem 1 with AND/OR amplification),
and structural invariants of Algorithm 1.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1702_00093_gb300 import synth


def _pairs(arr):
    return [(int(p >> 32), int(p & 0xFFFFFFFF)) for p in arr]


# ---------------------------------------------------------------------------
# Random bits
# ---------------------------------------------------------------------------

def test_splitmix64_published_outputs(golden):
    g = golden("splitmix64_seed0.json")
    gamma = int(g["gamma"], 16)
    state = 0
    for want in g["outputs_from_state_0"]:
        # the oracle's function is the output step applied to (state); the
        # generator advances state by gamma between outputs
        assert oracle.splitmix64(state) == int(want, 16)
        state = (state + gamma) & 0xFFFFFFFFFFFFFFFF


def test_walk_bits_are_fair_and_independent_of_neighbours():
    # Alg. 1 draws each pi_j(sigma) as a fair coin: mean 1/2, no correlation
    # between consecutive steps or between symbols.
    bits = np.array([[oracle.walk_bit(7, 0, j, s) for s in b"ACGT"] for j in range(4000)])
    n = bits.size
    mean = bits.mean()
    assert abs(mean - 0.5) < 4.0 * math.sqrt(0.25 / n)
    a, b = bits[:-1, 0], bits[1:, 0]
    corr = np.corrcoef(a, b)[0, 1]
    assert abs(corr) < 4.0 / math.sqrt(a.size)
    corr_sym = np.corrcoef(bits[:, 1], bits[:, 2])[0, 1]
    assert abs(corr_sym) < 4.0 / math.sqrt(bits.shape[0])


def test_positions_uniform_in_range():
    L = 37
    pos = oracle.positions(3, 4, 50, 20, L).ravel()
    assert pos.min() >= 0 and pos.max() < L
    counts = np.bincount(pos, minlength=L)
    exp = pos.size / L
    chi2 = ((counts - exp) ** 2 / exp).sum()
    # chi-square with 36 dof: 99.9% quantile is about 67.98
    assert chi2 < 68.0


# ---------------------------------------------------------------------------
# Running example of Section 4 (Tables 2-4)
# ---------------------------------------------------------------------------

def _running_example(golden):
    g = golden("running_example_sec4.json")
    alphabet = g["alphabet"].encode()
    ss = synth.pack([s.encode() for s in g["strings"]], alphabet)
    pi = np.zeros((2, 10, 4), dtype=np.uint8)
    for l, name in enumerate(["R1", "R2"]):
        for c, ch in enumerate(g["alphabet"]):
            pi[l, :, c] = g["pi_steps_1_to_10"][name][ch]
    f = g["functions_1based_positions"]
    pos = np.array([[f["f1^1"], f["f2^1"]], [f["f1^2"], f["f2^2"]]], dtype=np.uint32) - 1
    return g, ss, pi, pos


def test_running_example_embeddings_table4a(golden):
    g, ss, pi, _ = _running_example(golden)
    emb, we = oracle.embed(ss.data, ss.offsets, ss.alphabet, 2, 10, seed=0, pi_inject=pi)
    for i in range(4):
        for l in range(2):
            got = "".join("ACGT"[c] for c in emb[l, i])
            assert got == g["embedded_prefixes"][f"t{i + 1}^{l + 1}"]
            assert we[l, i] == 10      # no walk finishes within 10 steps


def test_running_example_signatures_table4b(golden):
    g, ss, pi, pos = _running_example(golden)
    emb, we = oracle.embed(ss.data, ss.offsets, ss.alphabet, 2, 10, seed=0, pi_inject=pi)
    keys = oracle.sign(emb, we, pos, 4)           # [r*m][n]
    for i in range(4):
        for col in range(4):
            sig = g["signatures"][str(i + 1)][col]
            want = "ACGT".index(sig[0]) + 5 * "ACGT".index(sig[1])
            assert int(keys[col, i]) == want
    # equal keys exactly where the printed signatures are equal
    for col in range(4):
        for a, b in itertools.combinations(range(4), 2):
            same = g["signatures"][str(a + 1)][col] == g["signatures"][str(b + 1)][col]
            assert (keys[col, a] == keys[col, b]) == same


def test_running_example_candidates_and_output(golden):
    g, ss, pi, pos = _running_example(golden)
    res = oracle.join(ss.data, ss.offsets, ss.alphabet, K=g["K"], r=2, m=2, z=2, seed=0,
                      L=10, out_len=10, pi_inject=pi, pos_inject=pos)
    assert [(a + 1, b + 1) for a, b in _pairs(res.candidates)] == [tuple(p) for p in g["candidates_1based"]]
    assert [(a + 1, b + 1) for a, b in _pairs(res.pairs)] == [tuple(p) for p in g["output_1based"]]


# ---------------------------------------------------------------------------
# Worked example of Section 1 and edit distance
# ---------------------------------------------------------------------------

def test_worked_example_bruteforce(golden):
    g = golden("worked_example_sec1.json")
    ss = synth.pack([s.encode() for s in g["strings"]], g["alphabet"].encode())
    got = _pairs(oracle.join_bruteforce(ss.data, ss.offsets, g["K"]))
    assert got == [tuple(p) for p in g["expected_pairs_0based"]]


def test_worked_example_embedjoin_precision_and_recall(golden):
    g = golden("worked_example_sec1.json")
    ss = synth.pack([s.encode() for s in g["strings"]], g["alphabet"].encode())
    want = [tuple(p) for p in g["expected_pairs_0based"]]
    # precision is always 100%; with many short signatures the candidate stage
    # keeps every true pair for this seed
    res = oracle.join(ss.data, ss.offsets, ss.alphabet, K=g["K"], r=7, m=16, z=2, seed=5)
    assert _pairs(res.pairs) == want
    for seed in range(10):
        res = oracle.join(ss.data, ss.offsets, ss.alphabet, K=g["K"], r=2, m=3, z=4, seed=seed)
        assert set(_pairs(res.pairs)) <= set(want)


def test_edit_distance_textbook(golden):
    for x, y, d in golden("edit_distance_textbook.json")["cases"]:
        assert oracle.ed_full(x.encode(), y.encode()) == d
        assert oracle.ed_banded(x.encode(), y.encode(), d) == d
        assert oracle.ed_banded(x.encode(), y.encode(), d + 3) == d
        if d > 0:
            assert oracle.ed_banded(x.encode(), y.encode(), d - 1) == d   # capped at K+1


def _neighbourhood_distances(x: bytes, alphabet: bytes, depth: int) -> dict:
    """Breadth-first search over single edits: the definition of edit distance."""
    dist = {x: 0}
    frontier = [x]
    for d in range(1, depth + 1):
        nxt = []
        for s in frontier:
            cands = set()
            for i in range(len(s) + 1):
                for a in alphabet:
                    cands.add(s[:i] + bytes([a]) + s[i:])          # insertion
            for i in range(len(s)):
                cands.add(s[:i] + s[i + 1:])                        # deletion
                for a in alphabet:
                    if a != s[i]:
                        cands.add(s[:i] + bytes([a]) + s[i + 1:])  # substitution
            for c in cands:
                if c not in dist:
                    dist[c] = d
                    nxt.append(c)
        frontier = nxt
    return dist


def test_edit_distance_equals_edit_neighbourhood_search():
    alphabet = b"ACG"
    strings = [b""] + [bytes(t) for L in range(1, 4) for t in itertools.product(alphabet, repeat=L)]
    for x in [b"", b"A", b"AC", b"CGA", b"AAG"]:
        dist = _neighbourhood_distances(x, alphabet, 3)
        for y in strings:
            d = dist.get(y, 4)            # beyond the search depth: at least 4
            full = oracle.ed_full(x, y)
            assert min(full, 4) == d, (x, y)
            for K in range(0, 4):
                assert oracle.ed_banded(x, y, K) == min(d, K + 1)


def test_banded_equals_capped_full_dp_random_pairs():
    rng = np.random.default_rng(0)
    for _ in range(300):
        lx, ly = rng.integers(0, 40, size=2)
        x = rng.choice(list(b"ACGT"), size=lx).astype(np.uint8).tobytes()
        y = rng.choice(list(b"ACGT"), size=ly).astype(np.uint8).tobytes()
        full = oracle.ed_full(x, y)
        # metric facts: length difference <= ED <= max length, symmetry
        assert abs(lx - ly) <= full <= max(lx, ly)
        assert full == oracle.ed_full(y, x)
        for K in (0, 1, 3, 7, 20, 50):
            assert oracle.ed_banded(x, y, K) == min(full, K + 1)


# ---------------------------------------------------------------------------
# Algorithm 1 invariants
# ---------------------------------------------------------------------------

def _rle(seq):
    runs = []
    for c in seq:
        if runs and runs[-1][0] == c:
            runs[-1][1] += 1
        else:
            runs.append([c, 1])
    return runs


def test_cutoff_dp_equals_banded_dp_and_bruteforce():
    # Ukkonen's cutoff only stops the band DP early: min(ED, K+1) is unchanged,
    # on random, similar and equal pairs, and the brute-force join is the same.
    rng = np.random.default_rng(21)
    lut = np.frombuffer(b"ACGT", np.uint8)
    for _ in range(300):
        a = lut[rng.integers(0, 4, size=int(rng.integers(0, 120)))].tobytes()
        if rng.random() < 0.5:
            b = bytearray(a)
            for _ in range(int(rng.integers(0, 12))):
                if b and rng.random() < 0.5:
                    del b[int(rng.integers(0, len(b)))]
                else:
                    b.insert(int(rng.integers(0, len(b) + 1)), int(lut[rng.integers(0, 4)]))
            b = bytes(b)
        else:
            b = lut[rng.integers(0, 4, size=int(rng.integers(0, 120)))].tobytes()
        for K in (0, 1, 3, 8, 20, 60):
            assert oracle.ed_banded_cutoff(a, b, K) == oracle.ed_banded(a, b, K), (a, b, K)
    ss = synth.dna_clusters(5, 8, 6, 15, 40, edits_mean=3.0)
    for K in (1, 3, 6):
        assert np.array_equal(oracle.join_bruteforce(ss.data, ss.offsets, K, cutoff=True),
                              oracle.join_bruteforce(ss.data, ss.offsets, K))


def test_cgk_structure_invariants():
    # Alg. 1 emits x[i] for one or more steps before moving to x[i+1], then
    # pads with bottom: the output has length out_len, bottom only as a
    # suffix, and the non-bottom part is x[0]^c0 x[1]^c1 ... with every c >= 1.
    ss = synth.random_strings(11, 60, 0, 50)
    out_len = 150
    emb, we = oracle.embed(ss.data, ss.offsets, ss.alphabet, 3, out_len, seed=9)
    assert emb.shape == (3, ss.n, out_len)
    for l in range(3):
        for i in range(ss.n):
            t = emb[l, i]
            x = [ss.alphabet.index(b) for b in ss.get(i)]
            w = int(we[l, i])
            assert np.all(t[w:] == 4) and np.all(t[:w] < 4)
            if not x:
                assert w == 0
                continue
            tr, xr = _rle(t[:w].tolist()), _rle(x)
            if w < out_len:          # walk finished: every run of x appears, each stretched
                assert len(tr) == len(xr)
                assert all(a[0] == b[0] and a[1] >= b[1] for a, b in zip(tr, xr))
            else:                    # walk cut by out_len: a prefix of x's runs
                assert len(tr) <= len(xr)
                assert all(a[0] == b[0] for a, b in zip(tr, xr))
                assert all(a[1] >= b[1] for a, b in zip(tr[:-1], xr))


def test_cgk_walk_covers_string_and_steps_are_at_least_one():
    # With walk_end < out_len the walk left the string: each input character
    # was emitted for >= 1 step, so walk_end >= |x|, and about 2 steps per char.
    ss = synth.random_strings(12, 200, 50, 60)
    emb, we = oracle.embed(ss.data, ss.offsets, ss.alphabet, 2, 400, seed=3)
    lens = ss.lengths()
    assert np.all(we >= lens[None, :])
    ratio = (we / lens[None, :]).mean()
    assert 1.8 < ratio < 2.2     # geometric(1/2) dwell time, mean 2


def test_identical_strings_identical_embeddings():
    s = b"ACGTTGCAAGT" * 5
    ss = synth.pack([s, b"A" + s, s], b"ACGT")
    emb, we = oracle.embed(ss.data, ss.offsets, ss.alphabet, 4, 200, seed=21)
    assert np.array_equal(emb[:, 0], emb[:, 2]) and np.array_equal(we[:, 0], we[:, 2])


def test_hamming_upper_bounds_edit_distance_when_walks_finish():
    # ED(x, y) <= Ham(f(x), f(y)) whenever both walks end inside the output
    # (footnote of Section 1 with the padding symbol).
    ss = synth.dna_clusters(13, 30, 4, 20, 40, edits_mean=3.0)
    out_len = 3 * int(ss.lengths().max())
    emb, we = oracle.embed(ss.data, ss.offsets, ss.alphabet, 5, out_len, seed=4)
    checked = 0
    for i, j in itertools.combinations(range(ss.n), 2):
        ed = oracle.ed_full(ss.get(i), ss.get(j))
        for l in range(5):
            if we[l, i] < out_len and we[l, j] < out_len:
                ham = int(np.count_nonzero(emb[l, i] != emb[l, j]))
                assert ed <= ham
                checked += 1
    assert checked > 1000


# ---------------------------------------------------------------------------
# LSH (Theorem 1 with AND/OR amplification) and Algorithm 3
# ---------------------------------------------------------------------------

def test_bit_sampling_collision_rate_closed_form():
    # For a fixed pair of length-L strings at Hamming distance h, one function
    # of z independent coordinates collides with probability (1 - h/L)^z and
    # at least one of m functions with 1 - (1 - (1-h/L)^z)^m.
    L, h, z, m = 64, 12, 3, 4
    rng = np.random.default_rng(1)
    a = rng.integers(0, 4, size=L).astype(np.uint8)
    b = a.copy()
    flip = rng.choice(L, size=h, replace=False)
    b[flip] = (b[flip] + 1) % 4
    emb = np.stack([a, b])[None]              # r=1, n=2
    we = np.full((1, 2), L, dtype=np.int64)
    trials, hits, any_hits = 0, 0, 0
    for seed in range(3000):
        pos = oracle.positions(seed, 1, m, z, L)
        keys = oracle.sign(emb, we, pos, 4)
        eq = keys[:, 0] == keys[:, 1]
        hits += int(eq.sum())
        trials += m
        any_hits += int(eq.any())
    p = (1 - h / L) ** z
    assert abs(hits / trials - p) < 4 * math.sqrt(p * (1 - p) / trials)
    p_or = 1 - (1 - p) ** m
    assert abs(any_hits / 3000 - p_or) < 4 * math.sqrt(p_or * (1 - p_or) / 3000)


def test_keys_are_injective_mixed_radix():
    # the key decodes back to the z sampled symbols (bottom = alphabet size)
    ss = synth.random_strings(5, 40, 5, 30)
    emb, we = oracle.embed(ss.data, ss.offsets, ss.alphabet, 2, 80, seed=2)
    pos = oracle.positions(2, 2, 3, 7, 80)
    keys = oracle.sign(emb, we, pos, 4)
    for l in range(2):
        for f in range(3):
            for i in range(ss.n):
                k = int(keys[l * 3 + f, i])
                for q in range(7):
                    c = k % 5
                    k //= 5
                    p = int(pos[l, f, q])
                    want = emb[l, i, p] if p < we[l, i] else 4
                    assert c == want
                assert k == 0


def test_fewer_samples_give_the_wider_key_modulo_and_nested_buckets():
    # Positions are drawn per (embedding, function, sample) from a counter (reading 2),
    # so parameter sets that differ only in z (or use fewer embeddings / functions)
    # sample the same steps for their common (l, f, q). The key of the first z samples
    # is then the key of z' > z samples modulo (|alphabet|+1)^z, and equal keys at z'
    # imply equal keys at z: a batch of joins relies on both facts to share walks and
    # buckets.
    ss = synth.dna_clusters(7, 10, 6, 20, 60, edits_mean=3.0)
    out_len = 3 * int(ss.lengths().max())
    emb, we = oracle.embed(ss.data, ss.offsets, ss.alphabet, 3, out_len, seed=11)
    wide = oracle.sign(emb, we, oracle.positions(11, 3, 5, 9, out_len), 4)        # r=3, m=5, z=9
    for r, m, z in [(3, 5, 6), (2, 5, 9), (3, 2, 4), (1, 1, 1)]:
        pos = oracle.positions(11, r, m, z, out_len)
        keys = oracle.sign(emb[:r], we[:r], pos, 4)
        for l in range(r):
            for f in range(m):
                got = keys[l * m + f]
                want = wide[l * 5 + f] % np.uint64(5 ** z)
                assert np.array_equal(got, want), (r, m, z, l, f)
                # nested buckets: equal wide keys imply equal narrow ones
                w = wide[l * 5 + f]
                same_w = w[:, None] == w[None, :]
                same_n = got[:, None] == got[None, :]
                assert not np.any(same_w & ~same_n)


def test_alg3_candidates_equal_pairwise_definition():
    # Alg. 3's sliding window with eviction equals the set
    # {(i, j): i < j, ||s_i| - |s_j|| <= K, some table has equal keys}.
    for seed, K in [(1, 2), (2, 5), (3, 0), (4, 30)]:
        ss = synth.dna_clusters(seed, 12, 5, 10, 30, edits_mean=2.0)
        out_len = 3 * int(ss.lengths().max())
        emb, we = oracle.embed(ss.data, ss.offsets, ss.alphabet, 3, out_len, seed=seed)
        pos = oracle.positions(seed, 3, 4, 3, out_len)
        keys = oracle.sign(emb, we, pos, 4)
        got = set(_pairs(oracle.candidates(ss.data, ss.offsets, keys, K)))
        lens = ss.lengths()
        want = set()
        for i, j in itertools.combinations(range(ss.n), 2):
            if abs(int(lens[i]) - int(lens[j])) <= K and np.any(keys[:, i] == keys[:, j]):
                want.add((i, j))
        assert got == want


def test_join_precision_and_recall_small_dna():
    ss = synth.small_dna(scale=0.2)      # 20 clusters of 10
    p = synth.SMALL_DNA_PARAMS
    res = oracle.join(ss.data, ss.offsets, ss.alphabet, K=p["K"], r=p["r"], m=p["m"],
                      z=p["z"], seed=p["seed"])
    truth = set(_pairs(oracle.join_bruteforce(ss.data, ss.offsets, p["K"])))
    got = set(_pairs(res.pairs))
    assert got <= truth                  # 100% precision
    assert len(truth) > 50
    assert len(got) / len(truth) > 0.85  # recall in the paper's reported range
    # every candidate that passed verification is a true pair and vice versa
    cand = set(_pairs(res.candidates))
    assert got == cand & truth


def test_streamed_keys_equal_signatures_of_materialised_embeddings():
    # The streamed form (walk one string over [0, L), sign it, drop the walk)
    # must give the keys of Alg. 1's full embedding signed by Section 3.2's AND
    # functions, whatever range of strings it is asked for; strings whose walks
    # do not finish by L (long ones) and empty strings included.
    rng = np.random.default_rng(31)
    for alphabet, L in [(b"ACGT", 60), (synth.TEXT, 150)]:
        lut = np.frombuffer(alphabet, np.uint8)
        strs = [lut[rng.integers(0, len(alphabet), size=int(rng.integers(0, 140)))].tobytes()
                for _ in range(90)]
        ss = synth.pack(strs, alphabet)
        out_len = max(3 * int(ss.lengths().max()), L)
        emb, we = oracle.embed(ss.data, ss.offsets, alphabet, 3, out_len, seed=4)
        want = oracle.sign(emb, we, oracle.positions(4, 3, 5, 6, L), len(alphabet))
        got = np.concatenate([oracle.keys(ss.data, ss.offsets, alphabet, 3, 5, 6, L, 4, lo, hi)
                              for lo, hi in [(0, 17), (17, 18), (18, 90)]], axis=1)
        assert np.array_equal(got, want)


def test_cutoff_verify_equals_banded_verify():
    ss = synth.dna_clusters(9, 10, 8, 20, 160, edits_mean=6.0)
    rng = np.random.default_rng(5)
    pairs = np.array(sorted({(int(min(a, b)) << 32) | int(max(a, b))
                             for a, b in rng.integers(0, ss.n, size=(400, 2)) if a != b}), dtype=np.uint64)
    for K in (0, 2, 6, 15, 40):
        v = oracle.verify(ss.data, ss.offsets, pairs, K)
        assert np.array_equal(oracle.verify_cutoff(ss.data, ss.offsets, pairs, K), v)
    assert v.sum() > 10
