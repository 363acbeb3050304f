"""CPU oracle for the EmbedJoin hot path -- TEST INFRASTRUCTURE ONLY.

A thin ctypes wrapper over ``oracle.c`` (plain single-threaded C). Only the
tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg use it;
the CUDA product path never imports it. See ``oracle.c`` for the readings of
the paper that it fixes.

Parity status per function:
  splitmix64 / walk_bit / position : pinned (published SplitMix64 outputs,
                                     statistical uniformity, closed-form LSH
                                     collision rate)
  embed (Alg. 1)                   : pinned (running example, Tables 3-4;
                                     invariants; ED <= Ham)
  sign (bit sampling + AND)        : pinned (running example, Table 4(b))
  candidates (Alg. 3)              : pinned (running example; brute-force
                                     all-pairs signature comparison)
  ed_banded / ed_full / verify     : pinned (worked example of Section 1;
                                     edit-neighbourhood enumeration; textbook
                                     values)
  join                             : pinned (running example output; worked
                                     example; precision against brute force)
  join(key_P) (<u,v> mod P keys)   : pinned (one sample per function reduces to
                                     the exact key; candidates contain the exact
                                     key's; distinct signatures collide at 1/P)
  join_grouped (Section 4.1)       : pinned (one group is EmbedJoin; every pair
                                     within K in length shares a group)
  join_plus (Alg. 4 and 5)         : pinned (equal to join when one substring and
                                     T = 1; candidates equal to the set definition
                                     by brute force; P[>= T matched signatures]
                                     equal to the binomial p_T of Section 5)
  keys (streamed walk + signatures) : pinned equal to sign(embed(...))
  verify_cutoff                    : pinned equal to verify (banded DP)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (plain C11, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [("r", C.c_uint32), ("m", C.c_uint32), ("z", C.c_uint32), ("L", C.c_uint32),
                ("out_len", C.c_int64), ("K", C.c_int32), ("seed", C.c_uint64),
                ("alphabet", C.c_void_p), ("alpha", C.c_uint32),
                ("pi_inject", C.c_void_p), ("inject_steps", C.c_int64),
                ("pos_inject", C.c_void_p)]


class _Stats(C.Structure):
    _fields_ = [("n_candidates", C.c_int64), ("n_out", C.c_int64), ("out_len", C.c_int64),
                ("L", C.c_uint32), ("t_embed", C.c_double), ("t_sign", C.c_double),
                ("t_candidates", C.c_double), ("t_verify", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp, i64, u64, u32, i32 = C.c_void_p, C.c_int64, C.c_uint64, C.c_uint32, C.c_int32
            L.or_splitmix64.restype = u64
            L.or_splitmix64.argtypes = [u64]
            L.or_walk_bit.restype = C.c_int
            L.or_walk_bit.argtypes = [u64, u32, u64, C.c_uint8]
            L.or_position.restype = u32
            L.or_position.argtypes = [u64, u32, u32, u32, u32]
            L.or_embed_all.restype = C.c_int
            L.or_embed_all.argtypes = [vp, vp, i64, vp, u32, u32, i64, u64, vp, i64, vp, vp]
            L.or_positions_all.restype = None
            L.or_positions_all.argtypes = [u64, u32, u32, u32, u32, vp]
            L.or_sign_all.restype = None
            L.or_sign_all.argtypes = [vp, vp, i64, u32, u32, u32, i64, vp, u32, vp]
            L.or_candidates_alg3.restype = i64
            L.or_candidates_alg3.argtypes = [vp, vp, i64, vp, i64, i32, vp, i64]
            L.or_ed_banded.restype = i32
            L.or_ed_banded.argtypes = [vp, i64, vp, i64, i32]
            L.or_ed_full.restype = i64
            L.or_ed_full.argtypes = [vp, i64, vp, i64]
            L.or_verify.restype = None
            L.or_verify.argtypes = [vp, vp, vp, i64, i32, vp]
            L.or_verify_cutoff.restype = None
            L.or_verify_cutoff.argtypes = [vp, vp, vp, i64, i32, vp]
            L.or_keys_range.restype = C.c_int
            L.or_keys_range.argtypes = [vp, vp, i64, i64, vp, u32, u32, u32, u32, u32, u64, vp, vp]
            L.or_join_bruteforce.restype = i64
            L.or_join_bruteforce.argtypes = [vp, vp, i64, i32, vp, i64]
            L.or_join_bruteforce_cutoff.restype = i64
            L.or_join_bruteforce_cutoff.argtypes = [vp, vp, i64, i32, vp, i64]
            L.or_ed_banded_cutoff.restype = i32
            L.or_ed_banded_cutoff.argtypes = [vp, i64, vp, i64, i32]
            L.or_join.restype = C.c_int
            L.or_join.argtypes = [vp, vp, i64, C.POINTER(_Params), vp, i64, vp, i64,
                                  C.POINTER(_Stats)]
            L.or_join_ext.restype = C.c_int
            L.or_join_ext.argtypes = [vp, vp, i64, C.POINTER(_Params), u64, vp, i64, vp, i64, C.POINTER(_Stats)]
            L.or_join_grouped.restype = C.c_int
            L.or_join_grouped.argtypes = [vp, vp, i64, C.POINTER(_Params), u64, vp, i64,
                                          C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
            L.or_group_count.restype = i64
            L.or_group_count.argtypes = [i64, i32]
            L.or_in_group.restype = C.c_int
            L.or_in_group.argtypes = [i64, i64, i32]
            L.or_sign_all_modp.restype = None
            L.or_sign_all_modp.argtypes = [vp, vp, i64, u32, u32, u32, i64, vp, u32, u64, u64, vp]
            L.or_hash_coefficient.restype = u32
            L.or_hash_coefficient.argtypes = [u64, u32, u32, u32, u64]
            L.or_join_plus.restype = C.c_int
            L.or_join_plus.argtypes = [vp, vp, i64, C.POINTER(_Params), i32, i32, vp, i64, vp, i64,
                                       C.POINTER(_Stats), C.POINTER(C.c_int64)]
            L.or_plus_substrings.restype = i32
            L.or_plus_substrings.argtypes = [i32, i32]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p) if a is not None and a.size else None


def _u8(b) -> np.ndarray:
    if isinstance(b, (bytes, bytearray)):
        return np.frombuffer(bytes(b), dtype=np.uint8).copy()
    return np.ascontiguousarray(b, dtype=np.uint8)


def _strings(data, offsets):
    data = np.ascontiguousarray(data, dtype=np.uint8)
    if data.size == 0:
        data = np.zeros(1, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    return data, offsets


# ---------------------------------------------------------------------------
# Random bits
# ---------------------------------------------------------------------------

def splitmix64(x: int) -> int:
    return int(lib().or_splitmix64(x & 0xFFFFFFFFFFFFFFFF))


def walk_bit(seed: int, l: int, j: int, sigma_byte: int) -> int:
    return int(lib().or_walk_bit(seed, l, j, sigma_byte))


def position(seed: int, l: int, f: int, q: int, L: int) -> int:
    return int(lib().or_position(seed, l, f, q, L))


def positions(seed: int, r: int, m: int, z: int, L: int) -> np.ndarray:
    out = np.zeros((r, m, z), dtype=np.uint32)
    lib().or_positions_all(seed, r, m, z, L, _p(out))
    return out


# ---------------------------------------------------------------------------
# Algorithm 1 (CGK embedding) and bit-sampling signatures
# ---------------------------------------------------------------------------

def embed(data, offsets, alphabet: bytes, r: int, out_len: int, seed: int,
          pi_inject: np.ndarray | None = None):
    """Returns (emb uint8 [r][n][out_len] codes, bottom = |alphabet|; walk_end int64 [r][n])."""
    data, offsets = _strings(data, offsets)
    n = offsets.shape[0] - 1
    alpha = len(alphabet)
    ab = _u8(alphabet)
    emb = np.zeros((r, n, out_len), dtype=np.uint8)
    we = np.zeros((r, n), dtype=np.int64)
    inj_steps = 0
    pi = None
    if pi_inject is not None:
        pi = np.ascontiguousarray(pi_inject, dtype=np.uint8)
        assert pi.shape[0] == r and pi.shape[2] == alpha
        inj_steps = pi.shape[1]
    rc = lib().or_embed_all(_p(data), _p(offsets), n, _p(ab), alpha, r, out_len, seed,
                            _p(pi), inj_steps, _p(emb), _p(we))
    if rc != 0:
        raise ValueError(f"oracle embed failed: {rc}")
    return emb, we


def sign(emb: np.ndarray, walk_end: np.ndarray, pos: np.ndarray, alpha: int) -> np.ndarray:
    """keys uint64 [r*m][n] from embeddings [r][n][out_len] and positions [r][m][z]."""
    emb = np.ascontiguousarray(emb, dtype=np.uint8)
    walk_end = np.ascontiguousarray(walk_end, dtype=np.int64)
    pos = np.ascontiguousarray(pos, dtype=np.uint32)
    r, n, out_len = emb.shape
    _, m, z = pos.shape
    keys = np.zeros((r * m, n), dtype=np.uint64)
    lib().or_sign_all(_p(emb), _p(walk_end), n, r, m, z, out_len, _p(pos), alpha, _p(keys))
    return keys


def keys(data, offsets, alphabet: bytes, r: int, m: int, z: int, L: int, seed: int,
         lo: int = 0, hi: int | None = None) -> np.ndarray:
    """Signature keys uint64 [r*m][hi-lo] of strings lo..hi-1, walked and signed
    one string at a time (the same keys as sign(embed(...)) over [0, L))."""
    data, offsets = _strings(data, offsets)
    n = offsets.shape[0] - 1
    hi = n if hi is None else hi
    ab = _u8(alphabet)
    pos = positions(seed, r, m, z, L)
    out = np.zeros((r * m, max(hi - lo, 0)), dtype=np.uint64)
    if hi > lo:
        rc = lib().or_keys_range(_p(data), _p(offsets), lo, hi, _p(ab), len(alphabet), r, m, z, L, seed,
                                 _p(pos), _p(out))
        if rc != 0:
            raise ValueError(f"oracle keys failed: {rc}")
    return out


def candidates(data, offsets, keys: np.ndarray, K: int) -> np.ndarray:
    """Algorithm 3's candidate set (sorted unique uint64 pairs)."""
    data, offsets = _strings(data, offsets)
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    T, n = keys.shape
    cnt = lib().or_candidates_alg3(_p(data), _p(offsets), n, _p(keys), T, K, None, 0)
    if cnt < 0:
        raise RuntimeError(f"oracle candidates failed: {cnt}")
    out = np.zeros(max(cnt, 1), dtype=np.uint64)
    lib().or_candidates_alg3(_p(data), _p(offsets), n, _p(keys), T, K, _p(out), cnt)
    return out[:cnt]


# ---------------------------------------------------------------------------
# Edit distance (Section 3.3) and verification
# ---------------------------------------------------------------------------

def ed_banded(x: bytes, y: bytes, K: int) -> int:
    """min(ED(x, y), K+1) by Ukkonen's banded DP."""
    xa, ya = _u8(x), _u8(y)
    return int(lib().or_ed_banded(_p(xa), len(x), _p(ya), len(y), K))


def ed_banded_cutoff(x: bytes, y: bytes, K: int) -> int:
    """min(ED(x, y), K+1) by the banded DP stopped at Ukkonen's cutoff."""
    xa, ya = _u8(x), _u8(y)
    return int(lib().or_ed_banded_cutoff(_p(xa), len(x), _p(ya), len(y), K))


def ed_full(x: bytes, y: bytes) -> int:
    xa, ya = _u8(x), _u8(y)
    return int(lib().or_ed_full(_p(xa), len(x), _p(ya), len(y)))


def verify(data, offsets, pairs: np.ndarray, K: int) -> np.ndarray:
    """uint8 flags: 1 iff ED(pair) <= K."""
    data, offsets = _strings(data, offsets)
    pairs = np.ascontiguousarray(pairs, dtype=np.uint64)
    flags = np.zeros(max(pairs.shape[0], 1), dtype=np.uint8)
    lib().or_verify(_p(data), _p(offsets), _p(pairs), pairs.shape[0], K, _p(flags))
    return flags[:pairs.shape[0]]


def verify_cutoff(data, offsets, pairs: np.ndarray, K: int) -> np.ndarray:
    """verify() with the DP stopped at Ukkonen's cutoff (same flags)."""
    data, offsets = _strings(data, offsets)
    pairs = np.ascontiguousarray(pairs, dtype=np.uint64)
    flags = np.zeros(max(pairs.shape[0], 1), dtype=np.uint8)
    lib().or_verify_cutoff(_p(data), _p(offsets), _p(pairs), pairs.shape[0], K, _p(flags))
    return flags[:pairs.shape[0]]


def join_bruteforce(data, offsets, K: int, cutoff: bool = False) -> np.ndarray:
    """Every pair i<j with ED <= K (the definition, Section 1), sorted; cutoff
    stops each pair's DP at Ukkonen's cutoff (same result, for larger samples)."""
    data, offsets = _strings(data, offsets)
    n = offsets.shape[0] - 1
    if cutoff:
        cap = max(n * (n - 1) // 2, 1)
        out = np.zeros(cap, dtype=np.uint64)
        cnt = lib().or_join_bruteforce_cutoff(_p(data), _p(offsets), n, K, _p(out), cap)
        return out[:cnt]
    cnt = lib().or_join_bruteforce(_p(data), _p(offsets), n, K, None, 0)
    out = np.zeros(max(cnt, 1), dtype=np.uint64)
    lib().or_join_bruteforce(_p(data), _p(offsets), n, K, _p(out), cnt)
    return out[:cnt]


class JoinResult:
    def __init__(self, pairs, candidates, stats):
        self.pairs = pairs
        self.candidates = candidates
        self.n_candidates = int(stats.n_candidates)
        self.out_len = int(stats.out_len)
        self.L = int(stats.L)
        self.t_embed = stats.t_embed
        self.t_sign = stats.t_sign
        self.t_candidates = stats.t_candidates
        self.t_verify = stats.t_verify


def join(data, offsets, alphabet: bytes, K: int, r: int, m: int, z: int, seed: int,
         L: int = 0, out_len: int = 0, pi_inject=None, pos_inject=None,
         keep_candidates: bool = True, key_P: int = 0) -> JoinResult:
    """EmbedJoin (Alg. 3 with Alg. 2) end to end. key_P > 0 buckets by the
    two-level hash <u, v> mod key_P of Section 4 instead of the exact key."""
    data, offsets = _strings(data, offsets)
    n = offsets.shape[0] - 1
    ab = _u8(alphabet)
    pi = None if pi_inject is None else np.ascontiguousarray(pi_inject, dtype=np.uint8)
    pos = None if pos_inject is None else np.ascontiguousarray(pos_inject, dtype=np.uint32)
    prm = _Params(r, m, z, L, out_len, K, seed, _p(ab), len(alphabet), _p(pi),
                  0 if pi is None else pi.shape[1], _p(pos))
    cap = 1 << 16
    while True:
        out = np.zeros(cap, dtype=np.uint64)
        cand = np.zeros(cap if keep_candidates else 1, dtype=np.uint64)
        st = _Stats()
        rc = lib().or_join_ext(_p(data), _p(offsets), n, C.byref(prm), key_P, _p(out), cap,
                               _p(cand) if keep_candidates else None, cap if keep_candidates else 0,
                               C.byref(st))
        if rc != 0:
            raise ValueError(f"oracle join failed: {rc}")
        if st.n_out <= cap and (not keep_candidates or st.n_candidates <= cap):
            return JoinResult(out[:st.n_out].copy(),
                              cand[:st.n_candidates].copy() if keep_candidates else None, st)
        cap = max(int(st.n_out), int(st.n_candidates)) + 1


# ---------------------------------------------------------------------------
# EmbedJoin+ (Algorithms 4 and 5)
# ---------------------------------------------------------------------------

def plus_substrings(K: int, delta: int) -> int:
    """ceil(K / delta), at least 1: the substrings (suffixes) embedded per string."""
    return int(lib().or_plus_substrings(K, delta))


def join_plus(data, offsets, alphabet: bytes, K: int, r: int, m: int, z: int, seed: int, delta: int,
              T: int | None = None, L: int = 0, out_len: int = 0, pi_inject=None, pos_inject=None,
              keep_candidates: bool = True) -> JoinResult:
    """EmbedJoin+ end to end. T defaults to Section 5's rule: 2 when there is
    more than one substring per string, else 1."""
    data, offsets = _strings(data, offsets)
    n = offsets.shape[0] - 1
    if T is None:
        T = 2 if plus_substrings(K, delta) > 1 else 1
    ab = _u8(alphabet)
    pi = None if pi_inject is None else np.ascontiguousarray(pi_inject, dtype=np.uint8)
    pos = None if pos_inject is None else np.ascontiguousarray(pos_inject, dtype=np.uint32)
    prm = _Params(r, m, z, L, out_len, K, seed, _p(ab), len(alphabet), _p(pi),
                  0 if pi is None else pi.shape[1], _p(pos))
    cap = 1 << 16
    while True:
        out = np.zeros(cap, dtype=np.uint64)
        cand = np.zeros(cap if keep_candidates else 1, dtype=np.uint64)
        st = _Stats()
        nt = C.c_int64(0)
        rc = lib().or_join_plus(_p(data), _p(offsets), n, C.byref(prm), delta, T, _p(out), cap,
                                _p(cand) if keep_candidates else None, cap if keep_candidates else 0,
                                C.byref(st), C.byref(nt))
        if rc != 0:
            raise ValueError(f"oracle join_plus failed: {rc}")
        if st.n_out <= cap and (not keep_candidates or st.n_candidates <= cap):
            res = JoinResult(out[:st.n_out].copy(),
                             cand[:st.n_candidates].copy() if keep_candidates else None, st)
            res.n_tuples = int(nt.value)
            res.T = T
            return res
        cap = max(int(st.n_out), int(st.n_candidates)) + 1


# ---------------------------------------------------------------------------
# Two-level hashing and grouping (Section 4)
# ---------------------------------------------------------------------------

def hash_coefficient(seed: int, l: int, f: int, q: int, P: int) -> int:
    return int(lib().or_hash_coefficient(seed, l, f, q, P))


def sign_modp(emb: np.ndarray, walk_end: np.ndarray, pos: np.ndarray, alpha: int, seed: int, P: int) -> np.ndarray:
    """Hashed keys uint64 [r*m][n]: <u, v> mod P of every signature."""
    emb = np.ascontiguousarray(emb, dtype=np.uint8)
    walk_end = np.ascontiguousarray(walk_end, dtype=np.int64)
    pos = np.ascontiguousarray(pos, dtype=np.uint32)
    r, n, out_len = emb.shape
    _, m, z = pos.shape
    keys = np.zeros((r * m, n), dtype=np.uint64)
    lib().or_sign_all_modp(_p(emb), _p(walk_end), n, r, m, z, out_len, _p(pos), alpha, seed, P, _p(keys))
    return keys


def group_count(N: int, K: int) -> int:
    return int(lib().or_group_count(N, K))


def in_group(length: int, g: int, K: int) -> bool:
    return bool(lib().or_in_group(length, g, K))


def join_grouped(data, offsets, alphabet: bytes, K: int, r: int, m: int, z: int, seed: int, L: int = 0,
                 key_P: int = 0):
    """EmbedJoin with grouping (Section 4.1): (sorted output pairs, candidates
    verified over all groups)."""
    data, offsets = _strings(data, offsets)
    n = offsets.shape[0] - 1
    ab = _u8(alphabet)
    prm = _Params(r, m, z, L, 0, K, seed, _p(ab), len(alphabet), None, 0, None)
    cap = 1 << 16
    while True:
        out = np.zeros(cap, dtype=np.uint64)
        no, nc = C.c_int64(0), C.c_int64(0)
        rc = lib().or_join_grouped(_p(data), _p(offsets), n, C.byref(prm), key_P, _p(out), cap, C.byref(no),
                                   C.byref(nc))
        if rc != 0:
            raise ValueError(f"oracle join_grouped failed: {rc}")
        if no.value <= cap:
            return out[:no.value].copy(), int(nc.value)
        cap = int(no.value)
