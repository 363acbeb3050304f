"""Python binding of the EmbedJoin C-ABI library (argument marshalling only).

Every step of the join runs in the CUDA kernels of ``libembedjoin.so``; this
module only passes pointers, sizes and streams. Arrays may be torch tensors
(device or host) or numpy arrays (host). PyTorch is used for device memory and
streams. Loading fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libembedjoin.so")

EJ_OK = 0
EJ_ERR_INVALID_ARG = 1
EJ_ERR_OOM = 2
EJ_ERR_CAPACITY = 3
EJ_ERR_CUDA = 4
EJ_ERR_TIMEOUT = 5
EJ_ERR_UNSUPPORTED = 6
EJ_ERR_TOO_LARGE = 7
NOALLOC_SCRATCH_BYTES = 64 << 20

EXPORTED = ["ej_create", "ej_destroy", "ej_status_string", "ej_last_error", "ej_set_timing",
            "ej_plan", "ej_embed", "ej_sign", "ej_lsh_candidates", "ej_verify", "ej_join",
            "ej_set_test_tables", "ej_set_verify_config", "ej_embed_sign", "ej_verify_noalloc",
            "ej_set_schedule", "ej_set_loop_bound", "ej_measure_int_peak", "ej_join_plus",
            "ej_set_key_hash", "ej_join_grouped", "ej_set_autotune", "ej_autotune_table", "ej_batch_create", "ej_batch_run", "ej_batch_result", "ej_batch_kernel_count",
            "ej_batch_verify_ms",
            "ej_batch_destroy", "ej_index_create", "ej_index_size", "ej_index_search", "ej_index_destroy",
            "ej_server_create", "ej_server_submit", "ej_server_poll", "ej_server_release", "ej_server_get_stats",
            "ej_server_reset_stats", "ej_server_destroy"]


class EJError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class ServerConfig(C.Structure):
    _fields_ = [("max_batch", C.c_int32), ("inflight", C.c_int32), ("max_batch_bytes", C.c_int64),
                ("hbm_reserve", C.c_uint64), ("hbm_budget", C.c_uint64)]


class SearchResult(C.Structure):
    _fields_ = [("id", C.c_int64), ("status", C.c_int32), ("n_matches", C.c_int32),
                ("matches", C.POINTER(C.c_uint32)), ("latency_ms", C.c_double), ("queue_ms", C.c_double)]


class ServerStats(C.Structure):
    _fields_ = [("completed", C.c_int64), ("batches", C.c_int64), ("retries", C.c_int64), ("deferred", C.c_int64),
                ("mean_batch", C.c_double), ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("mean_ms", C.c_double),
                ("queries_per_s", C.c_double), ("device_bytes", C.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class _Schedule(C.Structure):
    _fields_ = [("mode", C.c_int32), ("slots_per_warp", C.c_int32), ("warps_per_subpartition", C.c_int32),
                ("order", C.c_int32), ("buckets", C.c_int32), ("chain", C.c_int32)]


class TuneEntry(C.Structure):
    _fields_ = [("length_class", C.c_int32), ("K", C.c_int32), ("walk_threads", C.c_int32),
                ("lanes_per_pair", C.c_int32), ("words_per_lane", C.c_int32), ("configs_tried", C.c_int32),
                ("schedule", _Schedule), ("walk_ms", C.c_float), ("back_ms", C.c_float)]

    def as_dict(self) -> dict:
        sc = self.schedule
        return {"length_class": self.length_class, "mean_length_range": [1 << self.length_class,
                                                                          (2 << self.length_class) - 1],
                "K": self.K, "walk_threads_per_block": self.walk_threads,
                "verifier": {0: "automatic", 1: "persistent", 2: "grid-strided", 3: "shared-string"}.get(sc.mode),
                "slots_per_warp": sc.slots_per_warp, "warps_per_subpartition": sc.warps_per_subpartition,
                "order": sc.order, "lanes_per_pair": self.lanes_per_pair, "words_per_lane": self.words_per_lane,
                "configs_tried": self.configs_tried, "walk_ms": self.walk_ms, "back_ms": self.back_ms}


class _Params(C.Structure):
    _fields_ = [("r", C.c_uint32), ("m", C.c_uint32), ("z", C.c_uint32), ("L", C.c_uint32),
                ("out_len", C.c_uint32), ("K", C.c_int32), ("seed", C.c_uint64),
                ("alphabet", C.c_void_p), ("alphabet_size", C.c_uint32)]


class _Strings(C.Structure):
    _fields_ = [("bytes", C.c_void_p), ("offsets", C.c_void_p), ("n", C.c_int64)]


class PlanInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("max_len", C.c_int64), ("total_bytes", C.c_int64),
                ("out_len", C.c_uint32), ("L", C.c_uint32), ("planes", C.c_uint32),
                ("blocks32", C.c_uint32), ("embedding_bytes", C.c_uint64),
                ("walk_end_count", C.c_uint64), ("key_count", C.c_uint64)]


class JoinStats(C.Structure):
    _fields_ = [("n_raw_pairs", C.c_int64), ("n_candidates", C.c_int64), ("n_out", C.c_int64),
                ("max_bucket", C.c_int64), ("ms_prepare", C.c_float), ("ms_embed_sign", C.c_float),
                ("ms_candidates", C.c_float), ("ms_verify", C.c_float), ("ms_total", C.c_float),
                ("band_cells", C.c_uint64), ("verify_word_columns", C.c_uint64),
                ("kernel_launches", C.c_int64), ("ms_pack", C.c_float), ("ms_buckets", C.c_float),
                ("ms_dedup", C.c_float), ("ms_reserved", C.c_float)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """Load libembedjoin.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libembedjoin.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
        L.ej_create.argtypes = [C.POINTER(vp), C.c_int]
        L.ej_create.restype = C.c_int
        L.ej_destroy.argtypes = [vp]
        L.ej_destroy.restype = None
        L.ej_status_string.argtypes = [C.c_int]
        L.ej_status_string.restype = C.c_char_p
        L.ej_last_error.argtypes = [vp]
        L.ej_last_error.restype = C.c_char_p
        L.ej_set_timing.argtypes = [vp, C.c_int]
        L.ej_set_timing.restype = C.c_int
        L.ej_plan.argtypes = [vp, C.POINTER(_Strings), C.POINTER(_Params), C.POINTER(PlanInfo), vp]
        L.ej_plan.restype = C.c_int
        L.ej_embed.argtypes = [vp, C.POINTER(_Strings), C.POINTER(_Params), vp, vp, vp]
        L.ej_embed.restype = C.c_int
        L.ej_sign.argtypes = [vp, C.POINTER(_Strings), C.POINTER(_Params), vp, vp, vp, vp]
        L.ej_sign.restype = C.c_int
        L.ej_lsh_candidates.argtypes = [vp, C.POINTER(_Strings), C.POINTER(_Params), vp, vp, i64,
                                        C.POINTER(i64), C.POINTER(i64), vp]
        L.ej_lsh_candidates.restype = C.c_int
        L.ej_verify.argtypes = [vp, C.POINTER(_Strings), C.POINTER(_Params), vp, i64, vp,
                                C.POINTER(i64), vp]
        L.ej_verify.restype = C.c_int
        L.ej_join.argtypes = [vp, C.POINTER(_Strings), C.POINTER(_Params), vp, i64, C.POINTER(i64),
                              C.POINTER(JoinStats), vp]
        L.ej_join.restype = C.c_int
        L.ej_set_test_tables.argtypes = [vp, vp, C.c_uint32, C.c_uint32, C.c_uint32, vp,
                                         C.c_uint32, C.c_uint32]
        L.ej_set_test_tables.restype = C.c_int
        L.ej_verify_noalloc.argtypes = [C.POINTER(_Strings), C.POINTER(_Params), vp, i64, vp,
                                        C.POINTER(i64), vp]
        L.ej_verify_noalloc.restype = C.c_int
        L.ej_embed_sign.argtypes = [vp, C.POINTER(_Strings), C.POINTER(_Params), vp, vp]
        L.ej_embed_sign.restype = C.c_int
        L.ej_set_verify_config.argtypes = [vp, C.c_int, C.c_int, C.c_int]
        L.ej_set_verify_config.restype = C.c_int
        L.ej_set_autotune.argtypes = [vp, C.c_int]
        L.ej_set_autotune.restype = C.c_int
        L.ej_autotune_table.argtypes = [vp, vp, C.c_int32, C.POINTER(C.c_int32)]
        L.ej_autotune_table.restype = C.c_int
        L.ej_set_key_hash.argtypes = [vp, C.c_uint64]
        L.ej_set_key_hash.restype = C.c_int
        L.ej_join_grouped.argtypes = [vp, vp, vp, vp, C.c_int64, C.POINTER(C.c_int64), vp, vp]
        L.ej_join_grouped.restype = C.c_int
        L.ej_join_plus.argtypes = [vp, vp, vp, C.c_int32, C.c_int32, vp, C.c_int64, C.POINTER(C.c_int64), vp, vp]
        L.ej_join_plus.restype = C.c_int
        L.ej_set_loop_bound.argtypes = [vp, C.c_int64]
        L.ej_set_loop_bound.restype = C.c_int
        L.ej_measure_int_peak.argtypes = [C.c_int, C.c_int32, C.c_int32, C.POINTER(C.c_double),
                                          C.POINTER(C.c_double)]
        L.ej_measure_int_peak.restype = C.c_int
        L.ej_set_schedule.argtypes = [vp, C.POINTER(_Schedule)]
        L.ej_set_schedule.restype = C.c_int
        L.ej_batch_create.argtypes = [vp, C.POINTER(_Strings), C.POINTER(_Params), C.c_int32, C.c_int32,
                                      C.POINTER(vp), vp]
        L.ej_batch_create.restype = C.c_int
        L.ej_batch_run.argtypes = [vp, vp]
        L.ej_batch_run.restype = C.c_int
        L.ej_batch_result.argtypes = [vp, C.c_int32, vp, i64, C.POINTER(i64), C.POINTER(JoinStats), vp]
        L.ej_batch_result.restype = C.c_int
        L.ej_batch_verify_ms.argtypes = [vp, C.POINTER(C.c_float)]
        L.ej_batch_verify_ms.restype = C.c_int
        L.ej_batch_kernel_count.argtypes = [vp]
        L.ej_batch_kernel_count.restype = i64
        L.ej_batch_destroy.argtypes = [vp]
        L.ej_batch_destroy.restype = None
        L.ej_index_create.argtypes = [vp, C.POINTER(_Strings), C.POINTER(_Params), C.POINTER(vp), vp]
        L.ej_index_create.restype = C.c_int
        L.ej_index_size.argtypes = [vp]
        L.ej_index_size.restype = i64
        L.ej_index_search.argtypes = [vp, vp, C.POINTER(_Strings), vp, vp, i64, C.POINTER(i64), vp]
        L.ej_index_search.restype = C.c_int
        L.ej_index_destroy.argtypes = [vp]
        L.ej_index_destroy.restype = None
        L.ej_server_create.argtypes = [vp, C.POINTER(ServerConfig), C.POINTER(vp)]
        L.ej_server_create.restype = C.c_int
        L.ej_server_submit.argtypes = [vp, vp, C.c_int32, C.c_int32]
        L.ej_server_submit.restype = i64
        L.ej_server_poll.argtypes = [vp, C.POINTER(SearchResult), C.c_int32, C.POINTER(C.c_int32), C.c_int32]
        L.ej_server_poll.restype = C.c_int
        L.ej_server_release.argtypes = [vp, i64]
        L.ej_server_release.restype = C.c_int
        L.ej_server_get_stats.argtypes = [vp, C.POINTER(ServerStats)]
        L.ej_server_get_stats.restype = C.c_int
        L.ej_server_reset_stats.argtypes = [vp]
        L.ej_server_reset_stats.restype = C.c_int
        L.ej_server_destroy.argtypes = [vp]
        L.ej_server_destroy.restype = None
        _lib = L
    return _lib


def _ptr(a) -> int | None:
    """Raw address of a torch tensor or numpy array (must be contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data if a.size else None
    assert a.is_contiguous()
    return a.data_ptr() if a.numel() else None


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


@dataclass
class Params:
    """Method parameters: r embeddings, m LSH functions of z positions each,
    sampling range L (0 = out_len), out_len (0 = 3N), threshold K, seed."""
    K: int
    r: int
    m: int
    z: int
    seed: int = 1
    L: int = 0
    out_len: int = 0
    alphabet: bytes = b"ACGT"

    def _c(self):
        buf = C.create_string_buffer(bytes(self.alphabet), len(self.alphabet))
        p = _Params(self.r, self.m, self.z, self.L, self.out_len, self.K, self.seed & (2**64 - 1),
                    C.cast(buf, C.c_void_p), len(self.alphabet))
        return p, buf


class Strings:
    """Packed strings: uint8 bytes + int64 offsets (n+1), torch tensors or numpy."""

    def __init__(self, data, offsets):
        self.data = data
        self.offsets = offsets
        self.n = int(offsets.shape[0]) - 1

    def _c(self):
        return _Strings(_ptr(self.data), _ptr(self.offsets), self.n)

    @staticmethod
    def from_set(ss, device=None):
        """From a ``synth.StringSet``; device=None keeps host numpy arrays."""
        if device is None:
            return Strings(ss.data, ss.offsets)
        import torch
        d = torch.from_numpy(ss.data if ss.data.size else np.zeros(1, np.uint8)).to(device)
        o = torch.from_numpy(ss.offsets).to(device)
        return Strings(d, o)


class Context:
    """An ej_ctx bound to one CUDA device (owns scratch memory)."""

    def __init__(self, device: int = 0):
        self._h = C.c_void_p()
        st = lib().ej_create(C.byref(self._h), device)
        if st != EJ_OK:
            raise EJError(st, f"ej_create failed: {lib().ej_status_string(st).decode()}")
        self.device = device

    def close(self):
        if self._h:
            lib().ej_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, what: str):
        if st != EJ_OK:
            detail = lib().ej_last_error(self._h).decode()
            raise EJError(st, f"{what}: {lib().ej_status_string(st).decode()}: {detail}")

    def set_verify_config(self, lanes_per_pair: int = 0, words_per_lane: int = 0, warps: int = 0):
        """Verifier tiling (G lanes per pair, V words per lane); zeros = automatic."""
        self._check(lib().ej_set_verify_config(self._h, lanes_per_pair, words_per_lane, warps),
                    "ej_set_verify_config")

    def set_schedule(self, mode: int = 0, slots_per_warp: int = 0, warps_per_subpartition: int = 0,
                     order: int = 0, buckets: int = 0, chain: int = 0):
        """ej_join's back-half schedule (ej_schedule); zeros = defaults. See the header."""
        sc = _Schedule(mode, slots_per_warp, warps_per_subpartition, order, buckets, chain)
        self._check(lib().ej_set_schedule(self._h, C.byref(sc)), "ej_set_schedule")

    def set_loop_bound(self, passes: int = 0):
        """Loop passes per warp of the persistent verifier before it gives up
        (EJ_ERR_TIMEOUT); 0 = the default bound."""
        self._check(lib().ej_set_loop_bound(self._h, passes), "ej_set_loop_bound")

    def set_timing(self, on: bool = True):
        self._check(lib().ej_set_timing(self._h, 1 if on else 0), "ej_set_timing")

    def plan(self, s: Strings, p: Params, stream=None) -> PlanInfo:
        info = PlanInfo()
        cs, (cp, _keep) = s._c(), p._c()
        self._check(lib().ej_plan(self._h, C.byref(cs), C.byref(cp), C.byref(info), _stream(stream)),
                    "ej_plan")
        return info

    def embed(self, s: Strings, p: Params, emb, walk_end, stream=None):
        cs, (cp, _keep) = s._c(), p._c()
        self._check(lib().ej_embed(self._h, C.byref(cs), C.byref(cp), _ptr(emb), _ptr(walk_end),
                                   _stream(stream)), "ej_embed")

    def sign(self, s: Strings, p: Params, emb, walk_end, keys, stream=None):
        cs, (cp, _keep) = s._c(), p._c()
        self._check(lib().ej_sign(self._h, C.byref(cs), C.byref(cp), _ptr(emb), _ptr(walk_end),
                                  _ptr(keys), _stream(stream)), "ej_sign")

    def embed_sign(self, s: Strings, p: Params, keys, stream=None):
        """Keys [r*m][n] without materialising the embedding (fused walk)."""
        cs, (cp, _keep) = s._c(), p._c()
        self._check(lib().ej_embed_sign(self._h, C.byref(cs), C.byref(cp), _ptr(keys), _stream(stream)),
                    "ej_embed_sign")

    def lsh_candidates(self, s: Strings, p: Params, keys, pairs, stream=None) -> tuple[int, int]:
        """Returns (count, max_bucket). Raises EJError(EJ_ERR_CAPACITY) with
        .needed set when `pairs` is too small."""
        cs, (cp, _keep) = s._c(), p._c()
        n = C.c_int64(0)
        mb = C.c_int64(0)
        cap = 0 if pairs is None else int(pairs.shape[0])
        st = lib().ej_lsh_candidates(self._h, C.byref(cs), C.byref(cp), _ptr(keys), _ptr(pairs), cap,
                                     C.byref(n), C.byref(mb), _stream(stream))
        if st == EJ_ERR_CAPACITY:
            e = EJError(st, "ej_lsh_candidates: capacity")
            e.needed = n.value
            raise e
        self._check(st, "ej_lsh_candidates")
        return n.value, mb.value

    def verify(self, s: Strings, p: Params, pairs, out, stream=None) -> int:
        cs, (cp, _keep) = s._c(), p._c()
        n = C.c_int64(0)
        self._check(lib().ej_verify(self._h, C.byref(cs), C.byref(cp), _ptr(pairs), int(pairs.shape[0]),
                                    _ptr(out), C.byref(n), _stream(stream)), "ej_verify")
        return n.value

    def batch(self, s: Strings, params: list, autotune: bool = False, stream=None, eager: bool = False) -> "Batch":
        """ej_batch_create: all joins of `params` over device strings `s` as one CUDA
        graph (see Batch), or issued anew by every run when `eager`. `stream` must
        not be the legacy default stream."""
        return Batch(self, s, params, autotune, stream, eager)

    def join_into(self, s: Strings, p: Params, out, stream=None) -> tuple[int, JoinStats]:
        """ej_join into a caller buffer. Raises EJError with .needed on overflow."""
        cs, (cp, _keep) = s._c(), p._c()
        n = C.c_int64(0)
        stats = JoinStats()
        cap = 0 if out is None else int(out.shape[0])
        st = lib().ej_join(self._h, C.byref(cs), C.byref(cp), _ptr(out), cap, C.byref(n),
                           C.byref(stats), _stream(stream))
        if st == EJ_ERR_CAPACITY:
            e = EJError(st, "ej_join: capacity")
            e.needed = n.value
            raise e
        self._check(st, "ej_join")
        return n.value, stats

    def join(self, s: Strings, p: Params, device=None, capacity: int = 1 << 16, stream=None):
        """Convenience: returns (pairs, stats) with pairs a uint64 tensor on `device`
        (or a numpy array if device is None), growing the buffer on overflow."""
        while True:
            if device is None:
                out = np.zeros(max(capacity, 1), dtype=np.uint64)
            else:
                import torch
                out = torch.empty(max(capacity, 1), dtype=torch.int64, device=device)
            try:
                n, stats = self.join_into(s, p, out, stream)
                return out[:n], stats
            except EJError as e:
                if e.status != EJ_ERR_CAPACITY:
                    raise
                capacity = e.needed

    def join_plus_into(self, s: Strings, p: Params, delta: int, T: int, out, stream=None) -> tuple[int, JoinStats]:
        """ej_join_plus into a caller buffer. Raises EJError with .needed on overflow."""
        cs, (cp, _keep) = s._c(), p._c()
        n = C.c_int64(0)
        stats = JoinStats()
        cap = 0 if out is None else int(out.shape[0])
        st = lib().ej_join_plus(self._h, C.byref(cs), C.byref(cp), delta, T, _ptr(out), cap, C.byref(n),
                                C.byref(stats), _stream(stream))
        if st == EJ_ERR_CAPACITY:
            e = EJError(st, "ej_join_plus: capacity")
            e.needed = n.value
            raise e
        self._check(st, "ej_join_plus")
        return n.value, stats

    def join_plus(self, s: Strings, p: Params, delta: int, T: int | None = None, device=None,
                  capacity: int = 1 << 16, stream=None):
        """EmbedJoin+ (Section 5): (pairs, stats) as join(); T defaults to 2 when
        ceil(K/delta) > 1, else 1."""
        if T is None:
            T = 2 if max(1, -(-p.K // delta)) > 1 else 1
        while True:
            if device is None:
                out = np.zeros(max(capacity, 1), dtype=np.uint64)
            else:
                import torch
                out = torch.empty(max(capacity, 1), dtype=torch.int64, device=device)
            try:
                n, stats = self.join_plus_into(s, p, delta, T, out, stream)
                return out[:n], stats
            except EJError as e:
                if e.status != EJ_ERR_CAPACITY:
                    raise
                capacity = e.needed

    def set_autotune(self, enable: int = 1):
        """Autotuner on (1) / off (0) / off and table cleared (-1); see the header."""
        self._check(lib().ej_set_autotune(self._h, enable), "ej_set_autotune")

    def autotune_table(self) -> list:
        n = C.c_int32(0)
        self._check(lib().ej_autotune_table(self._h, None, 0, C.byref(n)), "ej_autotune_table")
        arr = (TuneEntry * max(n.value, 1))()
        self._check(lib().ej_autotune_table(self._h, arr, n.value, C.byref(n)), "ej_autotune_table")
        return [arr[i].as_dict() for i in range(n.value)]

    def set_key_hash(self, P: int = 0):
        """Bucket keys by the two-level hash <u, v> mod P of Section 4 (0 = exact keys)."""
        self._check(lib().ej_set_key_hash(self._h, P), "ej_set_key_hash")

    def join_grouped(self, s: Strings, p: Params, device=None, capacity: int = 1 << 16, stream=None):
        """EmbedJoin with grouping by length (Section 4.1): (pairs, stats) as join()."""
        while True:
            if device is None:
                out = np.zeros(max(capacity, 1), dtype=np.uint64)
            else:
                import torch
                out = torch.empty(max(capacity, 1), dtype=torch.int64, device=device)
            cs, (cp, _keep) = s._c(), p._c()
            n = C.c_int64(0)
            stats = JoinStats()
            st = lib().ej_join_grouped(self._h, C.byref(cs), C.byref(cp), _ptr(out), int(out.shape[0]), C.byref(n),
                                       C.byref(stats), _stream(stream))
            if st == EJ_ERR_CAPACITY and n.value > out.shape[0]:
                capacity = n.value
                continue
            self._check(st, "ej_join_grouped")
            return out[:n.value], stats

    def set_test_tables(self, pi=None, positions=None):
        """Inject explicit pi tables [r][steps][alphabet] (0/1) and/or positions
        [r][m][z] (the running example's Tables 2-3). No arguments restores RNG."""
        pi_a = None if pi is None else np.ascontiguousarray(pi, dtype=np.uint8)
        pos_a = None if positions is None else np.ascontiguousarray(positions, dtype=np.uint32)
        r = pi_a.shape[0] if pi_a is not None else (pos_a.shape[0] if pos_a is not None else 0)
        st = lib().ej_set_test_tables(
            self._h, _ptr(pi_a), r, 0 if pi_a is None else pi_a.shape[1],
            0 if pi_a is None else pi_a.shape[2], _ptr(pos_a),
            0 if pos_a is None else pos_a.shape[1], 0 if pos_a is None else pos_a.shape[2])
        self._check(st, "ej_set_test_tables")


def measure_int_peak(device: int = 0, mix: int = 0, iters: int = 4096) -> tuple[float, float]:
    """ej_measure_int_peak: (32-bit integer instructions/s over the GPU, ms of the
    timed launch) for mix 0 (lop3 + add), 1 (lop3) or 2 (add)."""
    ops, ms = C.c_double(0.0), C.c_double(0.0)
    st = lib().ej_measure_int_peak(device, mix, iters, C.byref(ops), C.byref(ms))
    if st != EJ_OK:
        raise EJError(st, f"ej_measure_int_peak: {lib().ej_status_string(st).decode()}")
    return ops.value, ms.value


def verify_noalloc(s: Strings, p: Params, pairs, out, stream=None) -> int:
    """ej_verify_noalloc: verification that allocates nothing (device arrays only).

    For callers whose device memory is reserved by another allocator or who must
    not trigger cudaMalloc/cudaFree on their request path. Returns the number of
    passing pairs written to `out`; raises EJError on failure (EJ_ERR_TOO_LARGE
    when the request does not fit the library's fixed 64 MiB scratch array).
    """
    cs, (cp, _keep) = s._c(), p._c()
    n = C.c_int64(0)
    st = lib().ej_verify_noalloc(C.byref(cs), C.byref(cp), _ptr(pairs), int(pairs.shape[0]), _ptr(out),
                                 C.byref(n), _stream(stream))
    if st != EJ_OK:
        raise EJError(st, f"ej_verify_noalloc: {lib().ej_status_string(st).decode()}")
    return n.value


def decode_embedding(emb_words: np.ndarray, walk_end: np.ndarray, r: int, n: int, out_len: int,
                     planes: int, alphabet_size: int) -> np.ndarray:
    """Bit-sliced ej_embed output -> codes [r][n][out_len] (bottom = alphabet_size).
    Host-side inspection helper (numpy), not part of the join."""
    nb32 = (n + 31) // 32
    w = np.asarray(emb_words, dtype=np.uint32).reshape(r, nb32, out_len, planes)
    bits = ((w[..., None] >> np.arange(32, dtype=np.uint32)) & 1).astype(np.uint8)  # r,B,j,k,t
    codes = np.zeros((r, nb32, 32, out_len), dtype=np.uint8)
    for k in range(planes):
        codes |= (bits[:, :, :, k, :].transpose(0, 1, 3, 2) << k).astype(np.uint8)
    codes = codes.reshape(r, nb32 * 32, out_len)[:, :n]
    steps = np.arange(out_len)[None, None, :]
    codes = np.where(steps >= np.asarray(walk_end)[:, :, None], alphabet_size, codes).astype(np.uint8)
    return codes


EJ_BATCH_AUTOTUNE = 1
EJ_BATCH_EAGER = 2


class Batch:
    """ej_batch: the device path of several joins over the same device strings,
    captured once as a CUDA graph. run() replays it (no host sync); result(i)
    waits and returns join i's sorted pairs, as ej_join would."""

    def __init__(self, ctx: Context, s: Strings, params: list, autotune: bool = False, stream=None,
                 eager: bool = False):
        self._ctx = ctx
        self._h = C.c_void_p()
        self._keep = [s, params]
        cs = s._c()
        cps = [p._c() for p in params]
        arr = (_Params * len(params))(*[cp for cp, _ in cps])
        self._keep.append(cps)
        flags = (EJ_BATCH_AUTOTUNE if autotune else 0) | (EJ_BATCH_EAGER if eager else 0)
        st = lib().ej_batch_create(ctx._h, C.byref(cs), arr, len(params), flags, C.byref(self._h), _stream(stream))
        ctx._check(st, "ej_batch_create")
        self.n = len(params)
        self.kernel_count = int(lib().ej_batch_kernel_count(self._h))

    def run(self, stream=None):
        self._ctx._check(lib().ej_batch_run(self._h, _stream(stream)), "ej_batch_run")

    def verify_ms(self) -> float:
        """Device time of the merged verifier launch in the last run (ms)."""
        ms = C.c_float(0.0)
        self._ctx._check(lib().ej_batch_verify_ms(self._h, C.byref(ms)), "ej_batch_verify_ms")
        return float(ms.value)

    def result_into(self, i: int, out, stream=None) -> tuple[int, JoinStats]:
        n = C.c_int64(0)
        stats = JoinStats()
        cap = 0 if out is None else int(out.shape[0])
        st = lib().ej_batch_result(self._h, i, _ptr(out), cap, C.byref(n), C.byref(stats), _stream(stream))
        if st == EJ_ERR_CAPACITY and n.value > cap:
            e = EJError(st, "ej_batch_result: capacity")
            e.needed = n.value
            raise e
        self._ctx._check(st, "ej_batch_result")
        return n.value, stats

    def result(self, i: int, device=None, capacity: int = 1 << 16, stream=None):
        while True:
            if device is None:
                out = np.zeros(max(capacity, 1), dtype=np.uint64)
            else:
                import torch
                out = torch.empty(max(capacity, 1), dtype=torch.int64, device=device)
            try:
                n, stats = self.result_into(i, out, stream)
                return out[:n], stats
            except EJError as e:
                if getattr(e, "needed", None) is None:
                    raise
                capacity = e.needed

    def close(self):
        if self._h:
            lib().ej_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _host_strings(queries):
    """Host Strings from a list of bytes objects (or a host Strings as is)."""
    if isinstance(queries, Strings):
        return queries
    lens = np.array([len(q) for q in queries], dtype=np.int64)
    offs = np.zeros(len(queries) + 1, dtype=np.int64)
    np.cumsum(lens, out=offs[1:])
    data = np.frombuffer(b"".join(queries), dtype=np.uint8).copy() if offs[-1] else np.zeros(1, np.uint8)
    return Strings(data, offs)


class Index:
    """ej_index: EmbedJoin's tables and buckets of a string set, resident on the GPU."""

    def __init__(self, ctx: Context, s: Strings, p: Params, stream=None):
        self._ctx = ctx
        self._h = C.c_void_p()
        cs, (cp, _keep) = s._c(), p._c()
        ctx._check(lib().ej_index_create(ctx._h, C.byref(cs), C.byref(cp), C.byref(self._h), _stream(stream)),
                   "ej_index_create")
        self.n = int(lib().ej_index_size(self._h))

    def search(self, queries, K, capacity: int = 1 << 16) -> np.ndarray:
        """All (q << 32 | i) with ED(query q, index string i) <= K[q] among the
        EmbedJoin candidates of q, ascending (uint64 numpy array)."""
        hs = _host_strings(queries)
        Ks = np.ascontiguousarray(np.broadcast_to(np.asarray(K, dtype=np.int32), (hs.n,)))
        cs = hs._c()
        while True:
            out = np.zeros(max(capacity, 1), dtype=np.uint64)
            n = C.c_int64(0)
            st = lib().ej_index_search(self._ctx._h, self._h, C.byref(cs), _ptr(Ks), _ptr(out), out.shape[0],
                                       C.byref(n), None)
            if st == EJ_ERR_CAPACITY:
                capacity = n.value
                continue
            self._ctx._check(st, "ej_index_search")
            return out[:n.value].copy()

    def close(self):
        if self._h:
            lib().ej_index_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """ej_server: continuous-batching search service over an Index."""

    def __init__(self, index: Index, max_batch: int = 0, inflight: int = 0, max_batch_bytes: int = 0,
                 hbm_reserve: int = 0, hbm_budget: int = 0):
        self._index = index
        self._h = C.c_void_p()
        cfg = ServerConfig(max_batch, inflight, max_batch_bytes, hbm_reserve, hbm_budget)
        st = lib().ej_server_create(index._h, C.byref(cfg), C.byref(self._h))
        if st != EJ_OK:
            raise EJError(st, "ej_server_create failed")
        self._buf = (SearchResult * 1024)()

    def submit(self, query: bytes, K: int) -> int:
        buf = np.frombuffer(query, dtype=np.uint8) if len(query) else np.zeros(1, np.uint8)
        rid = int(lib().ej_server_submit(self._h, _ptr(buf), len(query), int(K)))
        if rid < 0:
            raise EJError(-rid, "ej_server_submit: invalid query")
        return rid

    def poll(self, max_results: int = 1024, wait_us: int = 1000) -> list:
        """Finished requests: (id, status, matches uint32 array, latency_ms, queue_ms)."""
        n = C.c_int32(0)
        m = min(max_results, len(self._buf))
        st = lib().ej_server_poll(self._h, self._buf, m, C.byref(n), int(wait_us))
        if st != EJ_OK:
            raise EJError(st, "ej_server_poll")
        out = []
        for k in range(n.value):
            r = self._buf[k]
            mt = np.ctypeslib.as_array(r.matches, shape=(r.n_matches,)).copy() if r.n_matches else \
                np.zeros(0, dtype=np.uint32)
            out.append((int(r.id), int(r.status), mt, float(r.latency_ms), float(r.queue_ms)))
            lib().ej_server_release(self._h, r.id)
        return out

    def stats(self) -> dict:
        st = ServerStats()
        lib().ej_server_get_stats(self._h, C.byref(st))
        return st.as_dict()

    def reset_stats(self):
        lib().ej_server_reset_stats(self._h)

    def close(self):
        if self._h:
            lib().ej_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
