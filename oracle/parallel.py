"""Process-parallel drivers of the CPU oracle -- TEST INFRASTRUCTURE ONLY.

The oracle itself stays plain single-threaded C (``oracle.c``). These helpers
only split its work across processes so that full-size workloads can be
checked (and the oracle's verification timed on every host core): strings
are split into ranges for the walks and signatures, candidate pairs into
chunks for the verification. Nothing here adds arithmetic of the method;
every result is a concatenation of the single-threaded oracle's results.

Pools use the ``spawn`` start method, so they are safe in a process that has
already used CUDA. Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use this module.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from multiprocessing import shared_memory

import numpy as np


def cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def _pool(procs: int):
    return mp.get_context("spawn").Pool(procs)


def _ranges(offsets: np.ndarray, parts: int) -> list[tuple[int, int]]:
    """Split strings [0, n) into at most `parts` ranges of about equal bytes."""
    n = offsets.shape[0] - 1
    if n <= 0:
        return []
    total = int(offsets[-1])
    cuts = [0]
    for k in range(1, parts):
        c = int(np.searchsorted(offsets, total * k // parts, side="left"))
        c = min(max(c, cuts[-1]), n)
        cuts.append(c)
    cuts.append(n)
    return [(a, b) for a, b in zip(cuts[:-1], cuts[1:]) if b > a]


def _keys_chunk(args):
    data, offsets, alphabet, r, m, z, L, seed = args
    import oracle
    return oracle.keys(data, offsets, alphabet, r, m, z, L, seed)


def keys(data, offsets, alphabet: bytes, r: int, m: int, z: int, L: int, seed: int,
         procs: int | None = None) -> np.ndarray:
    """oracle.keys over all strings ([r*m][n] uint64), string ranges on `procs` processes."""
    data = np.ascontiguousarray(data, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    procs = procs or cores()
    rng = _ranges(offsets, 4 * procs)
    args = []
    for a, b in rng:
        lo, hi = int(offsets[a]), int(offsets[b])
        args.append((data[lo:hi].copy(), offsets[a:b + 1] - lo, bytes(alphabet), r, m, z, L, seed))
    if not args:
        return np.zeros((r * m, 0), dtype=np.uint64)
    if procs == 1:
        parts = [_keys_chunk(x) for x in args]
    else:
        with _pool(procs) as pool:
            parts = pool.map(_keys_chunk, args)
    return np.concatenate(parts, axis=1)


def _verify_chunk(args):
    dname, dlen, oname, olen, pairs, K, cutoff = args
    import oracle
    ds = shared_memory.SharedMemory(name=dname)
    os_ = shared_memory.SharedMemory(name=oname)
    try:
        data = np.ndarray((dlen,), dtype=np.uint8, buffer=ds.buf)
        offs = np.ndarray((olen,), dtype=np.int64, buffer=os_.buf)
        f = (oracle.verify_cutoff if cutoff else oracle.verify)(data, offs, pairs, K)
        out = f.copy()
        del data, offs, f
    finally:
        ds.close()
        os_.close()
    return out


class _Shared:
    """The strings in shared memory for the pool's workers."""

    def __init__(self, data: np.ndarray, offsets: np.ndarray):
        data = np.ascontiguousarray(data, dtype=np.uint8)
        if data.size == 0:
            data = np.zeros(1, np.uint8)
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        self.d = shared_memory.SharedMemory(create=True, size=data.nbytes)
        self.o = shared_memory.SharedMemory(create=True, size=offsets.nbytes)
        np.ndarray(data.shape, np.uint8, buffer=self.d.buf)[:] = data
        np.ndarray(offsets.shape, np.int64, buffer=self.o.buf)[:] = offsets
        self.dlen, self.olen = data.shape[0], offsets.shape[0]

    def close(self):
        for s in (self.d, self.o):
            s.close()
            s.unlink()


def verify(data, offsets, pairs: np.ndarray, K: int, procs: int | None = None, cutoff: bool = True,
           pool=None) -> np.ndarray:
    """oracle.verify (or verify_cutoff, the same flags) over chunks of `pairs` on
    `procs` processes: uint8 flags, 1 iff ED(pair) <= K."""
    pairs = np.ascontiguousarray(pairs, dtype=np.uint64)
    if pairs.shape[0] == 0:
        return np.zeros(0, np.uint8)
    procs = procs or cores()
    chunk = max(1, -(-pairs.shape[0] // (8 * procs)))
    sh = _Shared(data, offsets)
    try:
        args = [(sh.d.name, sh.dlen, sh.o.name, sh.olen, pairs[k:k + chunk], K, cutoff)
                for k in range(0, pairs.shape[0], chunk)]
        if pool is not None:
            parts = pool.map(_verify_chunk, args)
        elif procs == 1:
            parts = [_verify_chunk(a) for a in args]
        else:
            with _pool(procs) as p:
                parts = p.map(_verify_chunk, args)
    finally:
        sh.close()
    return np.concatenate(parts)


def join(data, offsets, alphabet: bytes, K: int, r: int, m: int, z: int, seed: int, L: int,
         procs: int | None = None):
    """EmbedJoin (Alg. 3 with Alg. 2) composed from the oracle's pieces: keys of
    every string (parallel over strings), Alg. 3's candidates (single process),
    verification (parallel over candidates). Returns (sorted output pairs,
    number of candidates): the same as oracle.join with L (and out_len >= L)."""
    import oracle
    k = keys(data, offsets, alphabet, r, m, z, L, seed, procs)
    cand = oracle.candidates(data, offsets, k, K)
    flags = verify(data, offsets, cand, K, procs)
    return cand[flags == 1], int(cand.shape[0])


def partners(keys_: np.ndarray, lengths: np.ndarray, K: int, i: int) -> np.ndarray:
    """Candidates of string i by the definition of Alg. 3's candidate set: every
    j != i that shares a key with i in some table and passes ||s_i|-|s_j|| <= K."""
    hit = np.any(keys_ == keys_[:, i:i + 1], axis=0)
    hit &= np.abs(lengths - lengths[i]) <= K
    hit[i] = False
    return np.nonzero(hit)[0]


def expected_pairs_of(data, offsets, keys_: np.ndarray, K: int, ids, procs: int | None = None,
                      pool=None) -> np.ndarray:
    """The join's output pairs that involve any string in `ids` (sorted unique
    (i<<32)|j): candidates of each id by the definition, verified by the oracle."""
    lengths = np.diff(np.asarray(offsets, dtype=np.int64))
    allp = set()
    for i in ids:
        for j in partners(keys_, lengths, K, int(i)):
            a, b = (int(i), int(j)) if i < j else (int(j), int(i))
            allp.add((a << 32) | b)
    cand = np.array(sorted(allp), dtype=np.uint64)
    flags = verify(data, offsets, cand, K, procs, pool=pool)
    return cand[flags == 1]


def pairs_of(pairs: np.ndarray, ids) -> np.ndarray:
    """The pairs of a sorted pair list that involve any string in `ids`."""
    pairs = np.asarray(pairs, dtype=np.uint64)
    ids = np.asarray(list(ids), dtype=np.uint64)
    a, b = pairs >> np.uint64(32), pairs & np.uint64(0xFFFFFFFF)
    return pairs[np.isin(a, ids) | np.isin(b, ids)]
