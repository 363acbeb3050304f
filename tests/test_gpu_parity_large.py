"""GPU parity at the sizes where the full workloads run.

Tables of more than 21845 records are bucketed in global memory (not in one
block's shared memory), tables of more than 24576 records are sorted by the
segmented LSD radix sort (not in one block), and the serving index is sorted
the same way. These tests drive every one of those paths at n = 30000 and
compare with the CPU oracle element by element (pairs, candidate counts,
keys), through the C ABI.

At the workloads' full sizes the oracle checks what it can compute in
seconds: the whole long-DNA join (20000 strings, K = 50/150/250, composed from
the oracle's pieces on all host cores); for the protein-like (n = 200000) and
text-like (n = 350000) joins, every signature key of every string, and the
exact output pairs of sampled strings (the candidates of a string by the
definition of Alg. 3's candidate set, verified by the oracle's banded DP).
The GPU side runs the batch form that the benchmark times.
"""
import numpy as np
import pytest

import oracle
from oracle import parallel
from paper_1702_00093_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DEV = "cuda:0"


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
def stream():
    return torch.cuda.Stream()


def _u64(t):
    return t.cpu().numpy().view(np.uint64) if hasattr(t, "cpu") else np.asarray(t, dtype=np.uint64)


N_LARGE = 30000


LARGE = dict(r=2, m=3, seed=9, L=40)
LARGE_KZ = ((2, 8), (3, 7))


@pytest.fixture(scope="module")
def large_set():
    # 3000 clusters of 10 DNA strings of 20-28 symbols (~1.5 edits per member):
    # buckets of a few to hundreds of records, ~2-3M candidates per join
    ss = synth.dna_clusters(30, 3000, 10, 20, 28, edits_mean=1.5)
    ref = {K: oracle.join(ss.data, ss.offsets, b"ACGT", K=K, z=z, **LARGE) for K, z in LARGE_KZ}
    return ss, ref


@pytest.mark.parametrize("buckets", [0, 1, 2])
@pytest.mark.parametrize("mode", [1, 2])
def test_join_global_and_radix_bucket_paths_equal_oracle(ej, ctx, large_set, buckets, mode):
    """n = 30000: hashed buckets in global memory (buckets 0 and 1) and the
    sorted path whose per-table sort is the segmented radix sort (buckets 2),
    with the persistent (mode 1) and grid-strided (mode 2) verifiers."""
    ss, ref = large_set
    assert ss.n == N_LARGE
    s = ej.Strings.from_set(ss, DEV)
    params = ej.Params(K=2, z=8, alphabet=b"ACGT", **LARGE)
    try:
        ctx.set_schedule(mode=mode, buckets=buckets)
        pairs, st = ctx.join(s, params, device=DEV, capacity=1 << 20)
    finally:
        ctx.set_schedule()
    want = ref[2]
    assert want.n_candidates > 100000 and st.max_bucket > 20
    assert st.n_candidates == want.n_candidates
    assert np.array_equal(_u64(pairs), want.pairs)


def test_lsh_candidates_radix_path_equals_oracle(ej, ctx, large_set):
    """The plain per-stage path at n = 30000: fused walk keys, then
    ej_lsh_candidates (length order and per-table sorts by the segmented radix
    sort, windows, pair sort-unique), then ej_verify."""
    ss, ref = large_set
    s = ej.Strings.from_set(ss, DEV)
    params = ej.Params(K=2, z=8, alphabet=b"ACGT", **LARGE)
    keys = torch.zeros(params.r * params.m * ss.n, dtype=torch.int64, device=DEV)
    ctx.embed_sign(s, params, keys)
    want_keys = oracle.keys(ss.data, ss.offsets, b"ACGT", params.r, params.m, params.z, params.L, params.seed)
    assert np.array_equal(_u64(keys).reshape(6, ss.n), want_keys)
    cand_ref = oracle.candidates(ss.data, ss.offsets, want_keys, 2)
    out = torch.empty(cand_ref.shape[0] + 16, dtype=torch.int64, device=DEV)
    n, mb = ctx.lsh_candidates(s, params, keys, out)
    assert n == cand_ref.shape[0] == ref[2].n_candidates
    assert np.array_equal(_u64(out[:n]), cand_ref)
    vout = torch.empty(n, dtype=torch.int64, device=DEV)
    k = ctx.verify(s, params, out[:n], vout)
    assert np.array_equal(_u64(vout[:k]), ref[2].pairs)


@pytest.mark.parametrize("buckets", [0, 2])
def test_batch_large_tables_equals_oracle(ej, ctx, large_set, stream, buckets):
    """A two-join batch at n = 30000 (K = 2 with z = 8, K = 3 with z = 7; same
    seed, L, r, m): shared walks and shared global buckets (buckets 0) or the
    sorted path (buckets 2), replayed as a graph; each join equals the oracle."""
    ss, ref = large_set
    s = ej.Strings.from_set(ss, DEV)
    params = [ej.Params(K=K, z=z, alphabet=b"ACGT", **LARGE) for K, z in LARGE_KZ]
    try:
        ctx.set_schedule(buckets=buckets)
        with torch.cuda.stream(stream):
            b = ctx.batch(s, params, stream=stream)
            for rep in range(2):
                b.run(stream)
                for i, p in enumerate(params):
                    got, st = b.result(i, device=DEV, capacity=1 << 20, stream=stream)
                    want = ref[p.K]
                    assert st.n_candidates == want.n_candidates, (rep, i)
                    assert np.array_equal(_u64(got), want.pairs), (rep, i)
            b.close()
    finally:
        ctx.set_schedule()


def test_index_sorted_by_radix_equals_oracle_search(ej, ctx):
    """A serving index of 30000 strings (its per-table sort is the segmented
    radix sort) searched with mixed queries equals the search the oracle
    defines: keys by the oracle's walk and signatures, candidates by key
    equality and the length filter, then the exact banded DP."""
    prm = dict(r=3, m=4, z=6, L=120, seed=1)
    idx = synth.serving_index(N_LARGE, seed=93, len_lo=50, len_hi=70)
    qs, ks = synth.serving_queries(idx, 60, seed=94, len_lo=20, len_hi=140, k_lo=0.02, k_hi=0.12)
    for i in range(4):
        qs.append(idx.get(int(1000 * i + 7)))
        ks = np.append(ks, 6)
    ks = ks.astype(np.int32)
    index = ej.Index(ctx, ej.Strings.from_set(idx, DEV), ej.Params(K=0, alphabet=b"ACGT", **prm))
    try:
        got = index.search(qs, ks)
    finally:
        index.close()
    allset = synth.pack([idx.get(i) for i in range(idx.n)] + list(qs), b"ACGT")
    keys = oracle.keys(allset.data, allset.offsets, b"ACGT", prm["r"], prm["m"], prm["z"], prm["L"], prm["seed"])
    lens = allset.lengths()
    n = idx.n
    want = []
    for q in range(len(qs)):
        hit = np.any(keys[:, :n] == keys[:, n + q:n + q + 1], axis=0) & (np.abs(lens[:n] - lens[n + q]) <= ks[q])
        cand = np.nonzero(hit)[0]
        if cand.size == 0:
            continue
        pairs = np.array([(int(i) << 32) | (n + q) for i in cand], dtype=np.uint64)
        ok = oracle.verify(allset.data, allset.offsets, pairs, int(ks[q])) == 1
        want += [(q << 32) | int(i) for i in cand[ok]]
    want = np.array(sorted(want), dtype=np.uint64)
    assert want.shape[0] >= 4
    assert np.array_equal(got, want)


# ---------------------------------------------------------------------------
# Full-size workloads, as the benchmark runs them
# ---------------------------------------------------------------------------

def _bench_batch(ej, ctx, ss, params, stream):
    s = ej.Strings.from_set(ss, DEV)
    outs, stats = [], []
    with torch.cuda.stream(stream):
        b = ctx.batch(s, params, stream=stream)
        b.run(stream)
        for i in range(len(params)):
            got, st = b.result(i, device=DEV, capacity=1 << 20, stream=stream)
            outs.append(_u64(got))
            stats.append(st)
        b.close()
    torch.cuda.synchronize()
    return outs, stats


@pytest.mark.slow
def test_long_dna_full_size_batch_equals_oracle(ej, ctx, stream):
    """The long-DNA workload at its full size (n = 20000, K = 50/150/250,
    r = 7, m = 20, z = 15/14/13, L = 5000): every join of the benchmark's batch
    equals the oracle's join (all candidates, all output pairs)."""
    ss = synth.long_dna()
    params = [ej.Params(alphabet=ss.alphabet, **synth.long_dna_params(K)) for K in (50, 150, 250)]
    outs, stats = _bench_batch(ej, ctx, ss, params, stream)
    for p, got, st in zip(params, outs, stats):
        want, nc = parallel.join(ss.data, ss.offsets, ss.alphabet, K=p.K, r=p.r, m=p.m, z=p.z, seed=p.seed, L=p.L)
        assert st.n_candidates == nc, p.K
        assert np.array_equal(got, want), p.K


def _sampled_full_size(ej, ctx, stream, ss, params, n_random=10, n_from_output=6, n_clustered=6):
    outs, stats = _bench_batch(ej, ctx, ss, params, stream)
    lens = ss.lengths()
    rng = np.random.default_rng(7)
    with parallel._pool(parallel.cores()) as pool:
        for p, got, st in zip(params, outs, stats):
            keys = parallel.keys(ss.data, ss.offsets, ss.alphabet, p.r, p.m, p.z, p.L, p.seed)
            # every key of every string, against the fused walk of the GPU
            s = ej.Strings.from_set(ss, DEV)
            gk = torch.zeros(p.r * p.m * ss.n, dtype=torch.int64, device=DEV)
            ctx.embed_sign(s, p, gk)
            assert np.array_equal(_u64(gk).reshape(p.r * p.m, ss.n), keys), p.K
            del gk, s
            ids = set(rng.integers(0, ss.n, size=n_random).tolist())
            if got.shape[0]:
                pick = got[rng.integers(0, got.shape[0], size=n_from_output)]
                ids |= set((pick >> np.uint64(32)).astype(np.int64).tolist())
            if ss.cluster is not None:
                sizes = np.bincount(ss.cluster)
                members = np.nonzero(sizes[ss.cluster] > 1)[0]
                ids |= set(rng.choice(members, size=n_clustered, replace=False).tolist())
            ids = sorted(ids)
            want = parallel.expected_pairs_of(ss.data, ss.offsets, keys, p.K, ids, pool=pool)
            assert np.array_equal(parallel.pairs_of(got, ids), want), p.K
            # precision on a random sample of all output pairs
            if got.shape[0]:
                smp = got[rng.integers(0, got.shape[0], size=min(200, got.shape[0]))]
                assert parallel.verify(ss.data, ss.offsets, smp, p.K, pool=pool).all()
    return outs, stats


@pytest.mark.slow
def test_protein_full_size_batch_sampled_against_oracle(ej, ctx, stream):
    """Protein-like workload at full size (n = 200000, K = 40/60, r = 7, m = 7,
    z = 8, L = 890)."""
    ss = synth.protein_workload()
    params = [ej.Params(alphabet=ss.alphabet, **synth.protein_params(K)) for K in synth.PROTEIN_KS]
    outs, stats = _sampled_full_size(ej, ctx, stream, ss, params)
    assert all(o.shape[0] > 1000 for o in outs)


@pytest.mark.slow
def test_text_full_size_batch_sampled_against_oracle(ej, ctx, stream):
    """Text-like workload at full size (n = 350000, K = 100/200/300, r = 7,
    m = 7, z = 10/9/9, L = 3800)."""
    ss = synth.text_workload()
    params = [ej.Params(alphabet=ss.alphabet, **synth.text_params(K)) for K in synth.TEXT_KS]
    outs, stats = _sampled_full_size(ej, ctx, stream, ss, params)
    assert all(o.shape[0] > 1000 for o in outs)
