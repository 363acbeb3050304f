"""Search against a resident index (ej_index_*) and the continuous-batching
server (ej_server_*): results equal the oracle's (keys by the oracle's CGK walk
and signatures, candidates by signature equality and the length filter, exact
banded edit distance), the server returns exactly what the offline batch search
returns, and a request's result is the same alone and in a mix of concurrent
requests."""
import time

import numpy as np
import pytest

import oracle
from paper_1702_00093_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DEV = "cuda:0"
PRM = dict(r=7, m=7, z=8, L=1000, seed=1)


@pytest.fixture(scope="module")
def ej():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_00093_gb300 import build
    build.build()
    oracle.build()
    from paper_1702_00093_gb300 import embedjoin
    return embedjoin


@pytest.fixture(scope="module")
def ctx(ej):
    c = ej.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def setup(ej, ctx):
    idx_ss = synth.serving_index(3000, seed=91)
    qs, ks = synth.serving_queries(idx_ss, 80, seed=92)
    # a few queries that are index strings themselves (with K large enough to
    # also catch their planted near-duplicates), an empty query, a tiny K
    for i in range(4):
        qs.append(idx_ss.get(int(i * 17)))
        ks = np.append(ks, 60)
    qs.append(b"")
    ks = np.append(ks, 3)
    qs.append(idx_ss.get(5)[:300])
    ks = np.append(ks, 0)
    ks = ks.astype(np.int32)
    index = ej.Index(ctx, ej.Strings.from_set(idx_ss, DEV), ej.Params(K=0, alphabet=idx_ss.alphabet, **PRM))
    return idx_ss, qs, ks, index


def oracle_search(idx_ss, qs, ks):
    """The search the oracle defines: keys of every index string and query by the
    oracle's walk and signatures, candidates = index strings sharing a key in some
    table with the query and within K of its length, then ED <= K exactly."""
    n = idx_ss.n
    allset = synth.pack([idx_ss.get(i) for i in range(n)] + list(qs), idx_ss.alphabet)
    emb, we = oracle.embed(allset.data, allset.offsets, allset.alphabet, PRM["r"], PRM["L"], PRM["seed"])
    pos = oracle.positions(PRM["seed"], PRM["r"], PRM["m"], PRM["z"], PRM["L"])
    keys = oracle.sign(emb, we, pos, len(allset.alphabet))   # [r*m][n + nq]
    lens = allset.lengths()
    want = []
    for q in range(len(qs)):
        hit = np.zeros(n, dtype=bool)
        for t in range(keys.shape[0]):
            hit |= keys[t, :n] == keys[t, n + q]
        cand = np.nonzero(hit & (np.abs(lens[:n] - lens[n + q]) <= ks[q]))[0]
        if cand.size == 0:
            continue
        pairs = np.array([(int(i) << 32) | (n + q) for i in cand], dtype=np.uint64)
        ok = oracle.verify(allset.data, allset.offsets, pairs, int(ks[q])) == 1
        want += [(q << 32) | int(i) for i in cand[ok]]
    return np.array(sorted(want), dtype=np.uint64)


def test_index_search_equals_oracle(ej, setup):
    idx_ss, qs, ks, index = setup
    got = index.search(qs, ks)
    want = oracle_search(idx_ss, qs, ks)
    assert want.size > 10
    assert np.array_equal(got, want)
    # the planted near-duplicates of an exact index string are found
    assert np.any((got >> np.uint64(32)) == np.uint64(80))


def test_server_equals_offline_search(ej, setup):
    idx_ss, qs, ks, index = setup
    offline = index.search(qs, ks)
    per_q = {q: sorted(int(v) & 0xFFFFFFFF for v in offline if int(v) >> 32 == q) for q in range(len(qs))}
    srv = ej.Server(index, max_batch=16, inflight=3)
    try:
        ids = {}
        for rnd in range(2):
            order = np.random.default_rng(rnd).permutation(len(qs))
            for q in order:
                ids[srv.submit(qs[q], int(ks[q]))] = int(q)
                if q % 7 == 0:
                    time.sleep(0.0005)   # arrivals while batches are in flight
            seen = 0
            deadline = time.time() + 60
            while seen < len(qs) and time.time() < deadline:
                for rid, status, matches, lat, queue in srv.poll(256, 2000):
                    assert status == 0
                    assert list(matches) == per_q[ids[rid]]
                    assert lat >= queue >= 0
                    seen += 1
            assert seen == len(qs)
        st = srv.stats()
        assert st["completed"] == 2 * len(qs) and st["batches"] >= 2 and st["p99_ms"] >= st["p50_ms"] > 0
    finally:
        srv.close()


def test_result_alone_equals_result_in_mix(ej, setup):
    idx_ss, qs, ks, index = setup
    probe = [80, 81, 0, 1]     # exact index strings and two mutated ones
    srv = ej.Server(index, max_batch=8, inflight=4)
    try:
        alone = {}
        for q in probe:
            srv.submit(qs[q], int(ks[q]))
            res = []
            while not res:
                res = srv.poll(8, 5000)
            alone[q] = list(res[0][2])
        mixed = {}
        rid_of = {}
        for rep in range(3):
            for q in range(len(qs)):
                rid = srv.submit(qs[q], int(ks[q]))
                if q in probe:
                    rid_of[rid] = q
        got = 0
        deadline = time.time() + 60
        while got < 3 * len(qs) and time.time() < deadline:
            for rid, status, matches, _, _ in srv.poll(256, 2000):
                got += 1
                if rid in rid_of:
                    mixed.setdefault(rid_of[rid], []).append(list(matches))
        assert got == 3 * len(qs)
        for q in probe:
            assert all(m == alone[q] for m in mixed[q]) and len(mixed[q]) == 3
    finally:
        srv.close()


def test_serving_misuse(ej, ctx, setup):
    idx_ss, qs, ks, index = setup
    srv = ej.Server(index, max_batch=4, inflight=1)
    try:
        with pytest.raises(ej.EJError):
            srv.submit(b"ACGTX", 2)          # byte outside the alphabet
        with pytest.raises(ej.EJError):
            srv.submit(b"ACGT", -1)
    finally:
        srv.close()
    with pytest.raises(ej.EJError):
        index.search([b"ACGN"], [1])
    with pytest.raises(ej.EJError):          # an index needs L > 0
        ej.Index(ctx, ej.Strings.from_set(idx_ss, DEV), ej.Params(K=0, r=2, m=2, z=4, seed=1, L=0,
                                                                  alphabet=idx_ss.alphabet))


def test_hbm_budget_admission(ej, setup):
    idx_ss, qs, ks, index = setup
    nq = 24
    offline = index.search(qs[:nq], ks[:nq])
    per_q = {q: sorted(int(v) & 0xFFFFFFFF for v in offline if int(v) >> 32 == q) for q in range(nq)}
    cfg = dict(max_batch=4, inflight=2, max_batch_bytes=16384)
    # the scratch a server of this shape sizes up front
    srv = ej.Server(index, **cfg)
    presized = srv.stats()["device_bytes"]
    srv.close()
    assert presized > 0
    long_q = bytes(np.random.default_rng(5).choice(np.frombuffer(idx_ss.alphabet, np.uint8), 200000))
    # a budget of exactly that: ordinary batches run, a query that would make a
    # slot grow beyond it finishes with EJ_ERR_OOM, and the server carries on
    srv = ej.Server(index, hbm_budget=presized, **cfg)
    try:
        ids = {srv.submit(qs[q], int(ks[q])): q for q in range(nq // 2)}
        big = srv.submit(long_q, 5)
        ids.update({srv.submit(qs[q], int(ks[q])): q for q in range(nq // 2, nq)})
        got = {}
        deadline = time.time() + 60
        while len(got) < nq + 1 and time.time() < deadline:
            for rid, status, matches, _, _ in srv.poll(256, 2000):
                got[rid] = (status, list(matches))
        assert len(got) == nq + 1
        assert got[big][0] == ej.EJ_ERR_OOM
        for rid, q in ids.items():
            assert got[rid] == (0, per_q[q])
        st = srv.stats()
        assert st["device_bytes"] <= presized
    finally:
        srv.close()
    # a budget too small for any scratch: every request fails the same way
    srv = ej.Server(index, hbm_budget=1, **cfg)
    try:
        rid = srv.submit(qs[0], int(ks[0]))
        res = []
        deadline = time.time() + 30
        while not res and time.time() < deadline:
            res = srv.poll(8, 2000)
        assert res and res[0][0] == rid and res[0][1] == ej.EJ_ERR_OOM
    finally:
        srv.close()
