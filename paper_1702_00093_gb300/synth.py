"""Seeded synthetic string sets shaped like the paper's workloads.

This module only draws inputs. It holds none of the join's arithmetic (no
embedding, hashing or edit distance), so both the CUDA path and the CPU oracle
can be fed from it without sharing any of the method's code.

Every generator returns a ``StringSet``: a packed ``uint8`` byte buffer, an
``int64`` offsets array of length n+1, the alphabet (raw bytes) and, where the
set is built from clusters, the cluster id of every string (used only to
enumerate the planted near-duplicate pairs for recall).

The shapes follow the datasets of Section 6.1 / Table 3 (UNIREF, TREC, the
human-genome reads), which are not available here; the synthetic recipes
stand in for them:

* ``dna_clusters``: uniform {A,C,G,T} cluster bases with members carrying
  Poisson-many random edits (GEN-like reads).
* ``protein_like``: 25 letters with Zipf(1) frequencies, log-normal lengths,
  20% near-duplicates (UNIREF-like).
* ``text_like``: 37 symbols (a-z, 0-9, space) with skewed unigram
  frequencies, uniform lengths, clusters of 2..20 near-duplicates (TREC-like).

Edits: an edit count is drawn per member; each edit picks a uniform position
of the source string and one of {substitution, deletion, insertion} with
equal probability. A substitution changes the symbol to a different one
(uniform among the others), an insertion puts a symbol drawn from the
alphabet's frequency distribution before the chosen position.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

DNA = b"ACGT"
PROTEIN = b"ACDEFGHIKLMNPQRSTVWYBXZUO"  # 25 letters
TEXT = b"etaoinshrdlcumwfgypbvkjxqz0123456789 "  # 37 symbols, letters in frequency rank order


@dataclass
class StringSet:
    data: np.ndarray          # uint8 packed bytes
    offsets: np.ndarray       # int64, n+1
    alphabet: bytes
    cluster: np.ndarray | None = None   # int64 cluster id per string (or None)
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0] - 1)

    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets)

    def get(self, i: int) -> bytes:
        return bytes(self.data[self.offsets[i]:self.offsets[i + 1]])

    def strings(self) -> list[bytes]:
        return [self.get(i) for i in range(self.n)]

    def subset(self, idx) -> "StringSet":
        idx = np.asarray(idx, dtype=np.int64)
        return pack([self.get(int(i)) for i in idx], self.alphabet,
                    None if self.cluster is None else self.cluster[idx])


def pack(strings, alphabet: bytes, cluster=None) -> StringSet:
    """Pack a list of byte strings into (data, offsets)."""
    lens = np.fromiter((len(s) for s in strings), dtype=np.int64, count=len(strings))
    offsets = np.zeros(len(strings) + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    data = np.frombuffer(b"".join(strings), dtype=np.uint8).copy() if len(strings) else np.zeros(0, np.uint8)
    cl = None if cluster is None else np.asarray(cluster, dtype=np.int64)
    return StringSet(data, offsets, bytes(alphabet), cl)


def _codes_to_set(code_list, alphabet: bytes, cluster, perm) -> StringSet:
    lut = np.frombuffer(alphabet, dtype=np.uint8)
    code_list = [code_list[i] for i in perm]
    lens = np.fromiter((c.shape[0] for c in code_list), dtype=np.int64, count=len(code_list))
    offsets = np.zeros(len(code_list) + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    data = lut[np.concatenate(code_list)] if code_list else np.zeros(0, np.uint8)
    cl = None if cluster is None else np.asarray(cluster, dtype=np.int64)[perm]
    return StringSet(data.astype(np.uint8), offsets, bytes(alphabet), cl)


def mutate(rng: np.random.Generator, s: np.ndarray, n_edits: int, sigma: int,
           freqs: np.ndarray | None = None) -> np.ndarray:
    """Apply ``n_edits`` random edits (sub/del/ins, equally likely) to code array ``s``."""
    L = s.shape[0]
    if n_edits <= 0 or L == 0:
        return s.copy()
    pos = rng.integers(0, L, size=n_edits)
    typ = rng.integers(0, 3, size=n_edits)
    vals = s.copy()
    keep = np.ones(L, dtype=bool)
    sub = pos[typ == 0]
    if sub.size:
        vals[sub] = (vals[sub] + rng.integers(1, sigma, size=sub.size)) % sigma
    dele = pos[typ == 1]
    if dele.size:
        keep[dele] = False
    ins = np.sort(pos[typ == 2])
    if ins.size:
        if freqs is None:
            ich = rng.integers(0, sigma, size=ins.size)
        else:
            ich = rng.choice(sigma, size=ins.size, p=freqs)
        vals = np.insert(vals, ins, ich.astype(vals.dtype))
        keep = np.insert(keep, ins, True)
    return vals[keep]


def random_strings(seed: int, n: int, len_lo: int, len_hi: int, alphabet: bytes = DNA) -> StringSet:
    """Independent uniform strings, lengths uniform in [len_lo, len_hi]."""
    rng = np.random.default_rng(seed)
    sigma = len(alphabet)
    lens = rng.integers(len_lo, len_hi + 1, size=n)
    codes = [rng.integers(0, sigma, size=int(l)).astype(np.uint8) for l in lens]
    return _codes_to_set(codes, alphabet, np.arange(n), np.arange(n))


def dna_clusters(seed: int, n_clusters: int, per_cluster: int, len_lo: int, len_hi: int,
                 edits_mean: float | None = None, rate_lo: float | None = None,
                 rate_hi: float | None = None) -> StringSet:
    """Uniform {A,C,G,T} cluster bases, each member = base + Poisson edits.

    Either a fixed Poisson mean ``edits_mean`` per member, or a per-member
    rate drawn uniformly from [rate_lo, rate_hi] with Poisson(rate * len)
    edits. The base itself is not part of the set. Order is shuffled.
    """
    rng = np.random.default_rng(seed)
    sigma = 4
    codes, cl = [], []
    base_lens = rng.integers(len_lo, len_hi + 1, size=n_clusters)
    for c in range(n_clusters):
        base = rng.integers(0, sigma, size=int(base_lens[c])).astype(np.uint8)
        for _ in range(per_cluster):
            if edits_mean is not None:
                k = int(rng.poisson(edits_mean))
            else:
                rate = rng.uniform(rate_lo, rate_hi)
                k = int(rng.poisson(rate * base.shape[0]))
            codes.append(mutate(rng, base, k, sigma))
            cl.append(c)
    perm = rng.permutation(len(codes))
    return _codes_to_set(codes, DNA, cl, perm)


def zipf_freqs(k: int, s: float = 1.0) -> np.ndarray:
    w = 1.0 / np.arange(1, k + 1, dtype=np.float64) ** s
    return w / w.sum()


def protein_like(seed: int, n: int, median: float = 400.0, sigma_ln: float = 0.46,
                 lo: int = 100, hi: int = 2000, dup_frac: float = 0.2,
                 dup_rate: float = 0.05) -> StringSet:
    """25 letters, Zipf(1) frequencies, log-normal lengths, 20% near-duplicates."""
    rng = np.random.default_rng(seed)
    sigma = len(PROTEIN)
    freqs = zipf_freqs(sigma, 1.0)
    n_dup = int(round(n * dup_frac))
    n_orig = n - n_dup
    lens = np.clip(np.round(rng.lognormal(np.log(median), sigma_ln, size=n_orig)), lo, hi).astype(np.int64)
    allc = rng.choice(sigma, size=int(lens.sum()), p=freqs).astype(np.uint8)
    codes = np.split(allc, np.cumsum(lens)[:-1]) if n_orig else []
    cl = list(range(n_orig))
    src = rng.integers(0, max(n_orig, 1), size=n_dup)
    for s in src:
        base = codes[int(s)]
        k = int(rng.poisson(dup_rate * base.shape[0]))
        codes.append(mutate(rng, base, k, sigma, freqs))
        cl.append(int(s))
    perm = rng.permutation(len(codes))
    return _codes_to_set(codes, PROTEIN, cl, perm)


def text_freqs() -> np.ndarray:
    """Space 0.18, ten digits 0.02 in total, letters Zipf(1) over the rank order of ``TEXT``."""
    f = np.zeros(37)
    f[:26] = zipf_freqs(26, 1.0) * 0.80
    f[26:36] = 0.002
    f[36] = 0.18
    return f / f.sum()


def text_like(seed: int, n: int, len_lo: int = 800, len_hi: int = 3000,
              cl_lo: int = 2, cl_hi: int = 20, rate_lo: float = 0.02,
              rate_hi: float = 0.20) -> StringSet:
    """37 symbols, skewed unigram frequencies, clusters of 2..20 near-duplicates."""
    rng = np.random.default_rng(seed)
    sigma = len(TEXT)
    freqs = text_freqs()
    codes, cl = [], []
    c = 0
    while len(codes) < n:
        size = int(rng.integers(cl_lo, cl_hi + 1))
        L = int(rng.integers(len_lo, len_hi + 1))
        base = rng.choice(sigma, size=L, p=freqs).astype(np.uint8)
        for _ in range(size):
            if len(codes) >= n:
                break
            rate = rng.uniform(rate_lo, rate_hi)
            codes.append(mutate(rng, base, int(rng.poisson(rate * L)), sigma, freqs))
            cl.append(c)
        c += 1
    perm = rng.permutation(len(codes))
    return _codes_to_set(codes, TEXT, cl, perm)


# ---------------------------------------------------------------------------
# Named workloads (sizes from the headline configurations)
# ---------------------------------------------------------------------------

def paper_z_rule(N: int, K: int, base_bits: int | None = None) -> int:
    """Positions per LSH function from the paper's rule (Section 4, 'Choices of
    parameters'; Section 6.4 uses 15 in place of log2 N): log2 N - floor(log2 x)
    with x% = K/N."""
    import math
    x = 100.0 * K / N
    top = base_bits if base_bits is not None else math.log2(N)
    return int(round(top - math.floor(math.log2(x))))


def small_dna(scale: float = 1.0) -> StringSet:
    """n=1000 over {A,C,G,T}: 100 clusters of 10, base length U[90,110], Poisson(4) edits."""
    nc = max(1, int(round(100 * scale)))
    return dna_clusters(1001, nc, 10, 90, 110, edits_mean=4.0)


SMALL_DNA_PARAMS = dict(K=6, r=3, m=10, z=12, seed=1)   # L = out_len = 3N


def long_dna(n_clusters: int = 2000, seed: int = 1002) -> StringSet:
    """n=20000 over {A,C,G,T}: 2000 clusters of 10, base length U[4500,5500],
    member edit rate U[1%,8%] of length (Poisson count)."""
    return dna_clusters(seed, n_clusters, 10, 4500, 5500, rate_lo=0.01, rate_hi=0.08)


def long_dna_params(K: int) -> dict:
    """r=7, m=20 functions, z from the paper's Section 6.4 rule with 15 bits and the
    5000 average length, L = avg length."""
    return dict(K=K, r=7, m=20, z=paper_z_rule(5000, K, base_bits=15), L=5000, seed=1)


def protein_workload(n: int = 200000) -> StringSet:
    return protein_like(1003, n)


def protein_params(K: int) -> dict:
    """Protein-like workload: K = 10% / 15% of the median length 400 (40, 60);
    r=7, m=7 (one table per embedding), z=8, L = twice the average length."""
    return dict(K=K, r=7, m=7, z=8, L=890, seed=1)


PROTEIN_KS = (40, 60)


def text_workload(n: int = 350000) -> StringSet:
    return text_like(1004, n)


def text_params(K: int) -> dict:
    """Text-like workload: r=7, m=7, z = 10 / 9 / 9 for K = 100 / 200 / 300,
    L = twice the average length."""
    return dict(K=K, r=7, m=7, z={100: 10, 200: 9, 300: 9}.get(K, 9), L=3800, seed=1)


TEXT_KS = (100, 200, 300)


# ---------------------------------------------------------------------------
# Serving: a resident index and a stream of search queries
# ---------------------------------------------------------------------------

def serving_index(n: int = 1_000_000, seed: int = 1005, len_lo: int = 900, len_hi: int = 1100,
                  dup_frac: float = 0.10, rate_lo: float = 0.01, rate_hi: float = 0.05) -> StringSet:
    """Uniform {A,C,G,T} strings of length U[len_lo, len_hi]; a fraction are planted
    near-duplicates (Poisson(rate * len) edits, rate U[rate_lo, rate_hi]) of others.
    Order is shuffled; cluster = the original's position for the planted ones."""
    rng = np.random.default_rng(seed)
    n_dup = int(round(n * dup_frac))
    n_orig = n - n_dup
    lens_o = rng.integers(len_lo, len_hi + 1, size=n_orig).astype(np.int64)
    offs_o = np.zeros(n_orig + 1, dtype=np.int64)
    np.cumsum(lens_o, out=offs_o[1:])
    codes_o = rng.integers(0, 4, size=int(offs_o[-1]), dtype=np.uint8)
    src = rng.integers(0, max(n_orig, 1), size=n_dup)
    dups = [mutate(rng, codes_o[offs_o[s]:offs_o[s + 1]], int(rng.poisson(rng.uniform(rate_lo, rate_hi) *
                                                                             (offs_o[s + 1] - offs_o[s]))), 4)
            for s in src]
    lens = np.concatenate([lens_o, np.fromiter((d.shape[0] for d in dups), dtype=np.int64, count=n_dup)])
    perm = rng.permutation(n)
    offsets = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens[perm], out=offsets[1:])
    data = np.empty(int(offsets[-1]), dtype=np.uint8)
    lut = np.frombuffer(DNA, dtype=np.uint8)
    for k in range(n):
        i = int(perm[k])
        data[offsets[k]:offsets[k + 1]] = codes_o[offs_o[i]:offs_o[i + 1]] if i < n_orig else dups[i - n_orig]
    data = lut[data]
    cl = np.concatenate([np.arange(n_orig, dtype=np.int64), src.astype(np.int64)])[perm]
    return StringSet(data, offsets, DNA, cl)


def serving_queries(index: StringSet, nq: int, seed: int = 1006, mutated_frac: float = 0.5,
                    len_lo: int = 200, len_hi: int = 5000, k_lo: float = 0.01, k_hi: float = 0.10):
    """Search queries: a fraction are index strings with Poisson(rate * len) edits
    (rate U[1%,10%]), the rest fresh uniform strings of length U[len_lo, len_hi];
    each query's K is U[k_lo, k_hi] of its own length. Returns (list of bytes, K int32)."""
    rng = np.random.default_rng(seed)
    lut = np.frombuffer(index.alphabet, np.uint8)
    rev = np.zeros(256, np.uint8)
    rev[lut] = np.arange(len(lut), dtype=np.uint8)
    qs, ks = [], []
    for _ in range(nq):
        if rng.random() < mutated_frac:
            i = int(rng.integers(0, index.n))
            base = rev[index.data[index.offsets[i]:index.offsets[i + 1]]]
            q = mutate(rng, base, int(rng.poisson(rng.uniform(0.01, 0.10) * base.shape[0])), 4)
        else:
            q = rng.integers(0, 4, size=int(rng.integers(len_lo, len_hi + 1)), dtype=np.uint8)
        qs.append(lut[q].tobytes())
        ks.append(int(round(rng.uniform(k_lo, k_hi) * len(q))))
    return qs, np.array(ks, dtype=np.int32)


SERVING_PARAMS = dict(r=7, m=7, z=8, L=1000, seed=1)
