"""Batched joins as one CUDA graph (ej_batch_*): every join of the batch returns
exactly what ej_join returns for the same parameters (and the oracle's pair
set), across replays, after the strings are rewritten in place, and with the
autotuner on; misuse is reported, not run."""
import numpy as np
import pytest

import oracle
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
    return t.cpu().numpy().view(np.uint64)


def _params(ej, ss, Ks, kw):
    return [ej.Params(K=K, alphabet=ss.alphabet, **kw(K)) for K in Ks]


def test_batch_equals_join_and_oracle_long_dna(ej, ctx, stream):
    ss = synth.long_dna(n_clusters=4, seed=77)
    s = ej.Strings.from_set(ss, DEV)

    def kw(K):
        p = synth.long_dna_params(K)
        return dict(r=p["r"], m=p["m"], z=p["z"], seed=p["seed"], L=p["L"])

    params = _params(ej, ss, [50, 150, 250], kw)
    with torch.cuda.stream(stream):
        b = ctx.batch(s, params, stream=stream)
        assert b.kernel_count > 3 * 5
        for rep in range(2):
            b.run(stream)
            for i, p in enumerate(params):
                got, st = b.result(i, device=DEV, stream=stream)
                want, st_j = ctx.join(s, p, device=DEV, stream=stream)
                assert np.array_equal(_u64(got), _u64(want))
                assert st.n_candidates == st_j.n_candidates
                if rep == 0:
                    ref = oracle.join(ss.data, ss.offsets, ss.alphabet, K=p.K, r=p.r, m=p.m, z=p.z, seed=p.seed,
                                      L=p.L)
                    assert np.array_equal(_u64(got), ref.pairs)
        b.close()


def test_batch_shares_walks_across_parameter_sets(ej, ctx, stream):
    """Joins whose (r, m, z) another join of the batch covers (same seed and L)
    take their keys from that join's walks: a narrower set by the modulus of the
    wider key, an equal set directly. Each must still return exactly ej_join's
    pairs, and a join with another seed walks on its own."""
    ss = synth.small_dna(0.5)
    s = ej.Strings.from_set(ss, DEV)
    a = ss.alphabet
    params = [ej.Params(K=6, alphabet=a, r=2, m=6, z=9, seed=1),
              ej.Params(K=5, alphabet=a, r=3, m=10, z=12, seed=1),
              ej.Params(K=7, alphabet=a, r=3, m=10, z=12, seed=1),
              ej.Params(K=6, alphabet=a, r=3, m=4, z=12, seed=1),
              ej.Params(K=6, alphabet=a, r=3, m=10, z=11, seed=2)]
    with torch.cuda.stream(stream):
        b = ctx.batch(s, params, stream=stream)
        b.run(stream)
        outs = []
        for i, p in enumerate(params):
            got, st = b.result(i, device=DEV, stream=stream)
            want, st_j = ctx.join(s, p, device=DEV, stream=stream)
            assert np.array_equal(_u64(got), _u64(want)), i
            assert st.n_candidates == st_j.n_candidates
            outs.append(_u64(got))
        b.close()
    ref = oracle.join(ss.data, ss.offsets, a, K=6, r=2, m=6, z=9, seed=1)
    assert np.array_equal(outs[0], ref.pairs)


@pytest.mark.parametrize("chain", [0, 1, 2, 3, 4])
def test_batch_persistent_verifiers_merged_chained_or_overlapping(ej, stream, chain):
    """Joins on the persistent verifier with different K (4, 40, 100, 20; the
    same signatures, so their candidate sets nest): verified by one merged
    launch over the union of their candidates, each pair once at the largest K
    of the joins that list it (chain 4), one merged launch over the joins in
    turn (3), one launch per join in turn (2) or overlapping (1); every join
    returns ej_join's pairs and counts its band cells at its own K."""
    c = ej.Context(0)
    try:
        c.set_schedule(mode=1, chain=chain)
        ss = synth.small_dna(0.5)
        s = ej.Strings.from_set(ss, DEV)
        params = _params(ej, ss, [4, 40, 100, 20], lambda K: dict(r=3, m=10, z=12, seed=1))
        with torch.cuda.stream(stream):
            b = c.batch(s, params, stream=stream)
            for rep in range(2):
                b.run(stream)
                for i, p in enumerate(params):
                    got, st = b.result(i, device=DEV, stream=stream)
                    want, st_j = c.join(s, p, device=DEV, stream=stream)
                    assert np.array_equal(_u64(got), _u64(want)), (chain, i)
                    assert st.n_candidates == st_j.n_candidates
                    assert st.band_cells == st_j.band_cells
            with pytest.raises(ej.EJError):   # timed only without a graph
                b.verify_ms()
            # the same work issued without a graph
            e = c.batch(s, params, stream=stream, eager=True)
            assert e.kernel_count == b.kernel_count
            e.run(stream)
            for i, p in enumerate(params):
                got, _ = e.result(i, device=DEV, stream=stream)
                want, _ = b.result(i, device=DEV, stream=stream)
                assert np.array_equal(_u64(got), _u64(want)), (chain, i)
            if chain in (3, 4):
                assert e.verify_ms() > 0
            elif chain in (1, 2):
                with pytest.raises(ej.EJError):
                    e.verify_ms()
            e.close()
            b.close()
    finally:
        c.close()


@pytest.mark.parametrize("buckets", [0, 1, 2])
def test_batch_bucket_sharing_modes(ej, stream, buckets):
    """Joins with the same seed, L, r, m and z = 15/14/13: with buckets 0 the two
    finer joins take their pairs from the z=13 join's buckets; 1 keeps each
    join's own hashed buckets, 2 sorts. Every join returns ej_join's pairs,
    candidate count and largest bucket."""
    c = ej.Context(0)
    try:
        c.set_schedule(buckets=buckets)
        ss = synth.long_dna(n_clusters=6, seed=78)
        s = ej.Strings.from_set(ss, DEV)

        def kw(K):
            p = synth.long_dna_params(K)
            return dict(r=p["r"], m=p["m"], z=p["z"], seed=p["seed"], L=p["L"])

        params = _params(ej, ss, [250, 50, 150], kw)
        with torch.cuda.stream(stream):
            b = c.batch(s, params, stream=stream)
            for rep in range(2):
                b.run(stream)
                for i, p in enumerate(params):
                    got, st = b.result(i, device=DEV, stream=stream)
                    want, st_j = c.join(s, p, device=DEV, stream=stream)
                    assert np.array_equal(_u64(got), _u64(want)), (buckets, i)
                    assert st.n_candidates == st_j.n_candidates and st.n_raw_pairs == st_j.n_raw_pairs
                    assert st.max_bucket == st_j.max_bucket
            b.close()
    finally:
        c.close()


def test_batch_rerun_after_rewriting_strings(ej, ctx, stream):
    ss = synth.small_dna(0.5)
    s = ej.Strings.from_set(ss, DEV)
    params = _params(ej, ss, [4, 6, 9], lambda K: dict(r=3, m=10, z=12, seed=1))
    with torch.cuda.stream(stream):
        b = ctx.batch(s, params, stream=stream)
        for rnd in range(3):
            if rnd > 0:
                # rewrite the contents in place (same lengths): rotate the alphabet
                lut = torch.zeros(256, dtype=torch.uint8, device=DEV)
                for c in range(4):
                    lut[ss.alphabet[c]] = ss.alphabet[(c + rnd) % 4]
                s.data.copy_(lut[s.data.long()])
            b.run(stream)
            for i, p in enumerate(params):
                got, _ = b.result(i, device=DEV, stream=stream)
                want, _ = ctx.join(s, p, device=DEV, stream=stream)
                assert np.array_equal(_u64(got), _u64(want)), (rnd, i)
        b.close()


def test_batch_large_output_to_device_and_host(ej, ctx, stream):
    """A join with more output pairs than the run sorts on the device (8192):
    ej_batch_result sorts those itself; results into device and host buffers
    equal ej_join's."""
    rng = np.random.default_rng(3)
    base = rng.integers(0, 4, size=300).astype(np.uint8)
    strs = []
    for k in range(160):                      # 160 near-copies: 12720 pairs within K
        x = base.copy()
        x[rng.integers(0, 300)] = rng.integers(0, 4)
        strs.append(np.frombuffer(b"ACGT", np.uint8)[x].tobytes())
    ss = synth.pack(strs, b"ACGT")
    s = ej.Strings.from_set(ss, DEV)
    params = _params(ej, ss, [2, 1], lambda K: dict(r=2, m=4, z=6, seed=3))
    with torch.cuda.stream(stream):
        b = ctx.batch(s, params, stream=stream)
        b.run(stream)
        for i, p in enumerate(params):
            want, _ = ctx.join(s, p, device=DEV, stream=stream)
            got, st = b.result(i, device=DEV, stream=stream)
            assert np.array_equal(_u64(got), _u64(want)), i
            host, _ = b.result(i, device=None, stream=stream)
            assert np.array_equal(host.view(np.uint64), _u64(want)), i
            if i == 0:
                assert st.n_out > 8192
        b.close()


def test_batch_autotune_keeps_results(ej, ctx, stream):
    ss = synth.protein_like(6, 200, median=150, lo=40, hi=500)
    s = ej.Strings.from_set(ss, DEV)
    L = int(2 * ss.lengths().mean())
    params = _params(ej, ss, [10, 25], lambda K: dict(r=4, m=6, z=5, seed=3, L=L))
    with torch.cuda.stream(stream):
        b = ctx.batch(s, params, autotune=True, stream=stream)
        b.run(stream)
        for i, p in enumerate(params):
            got, _ = b.result(i, device=DEV, stream=stream)
            ref = oracle.join(ss.data, ss.offsets, ss.alphabet, K=p.K, r=p.r, m=p.m, z=p.z, seed=p.seed, L=p.L)
            assert np.array_equal(_u64(got), ref.pairs)
        b.close()


def test_batch_misuse_is_reported(ej, ctx, stream):
    ss = synth.small_dna(0.2)
    params = _params(ej, ss, [5], lambda K: dict(r=2, m=4, z=8, seed=1))
    # host strings
    with pytest.raises(ej.EJError):
        ctx.batch(ej.Strings(ss.data, ss.offsets), params, stream=stream)
    # different alphabets in one batch
    s = ej.Strings.from_set(ss, DEV)
    other = ej.Params(K=5, r=2, m=4, z=8, seed=1, alphabet=b"ACGTN")
    with pytest.raises(ej.EJError):
        ctx.batch(s, params + [other], stream=stream)
    # offsets[n] grows beyond the plan: the bytes buffer really holds the extra
    # bytes, the validation kernel zeroes every length and flags it
    data = torch.cat([torch.from_numpy(ss.data).to(DEV), torch.full((4096,), ord("A"), dtype=torch.uint8,
                                                                     device=DEV)])
    offs = torch.from_numpy(ss.offsets.astype(np.int64)).to(DEV)
    s2 = ej.Strings(data, offs)
    with torch.cuda.stream(stream):
        b = ctx.batch(s2, params, stream=stream)
        b.run(stream)
        b.result(0, device=DEV, stream=stream)
        offs[-1] += 1000
        b.run(stream)
        with pytest.raises(ej.EJError) as e:
            b.result(0, device=DEV, stream=stream)
        assert e.value.status == ej.EJ_ERR_INVALID_ARG
        b.close()


@pytest.mark.parametrize("chain", [3, 4])
def test_batch_union_of_overlapping_candidate_sets_equals_oracle(ej, stream, chain):
    """Persistent-verifier joins whose candidate sets overlap only in part (two
    seeds, different z and K): the union launch verifies a pair listed by
    several joins once, at the largest of their K, and each join still gets
    exactly the oracle's pairs."""
    c = ej.Context(0)
    try:
        c.set_schedule(mode=1, chain=chain)
        ss = synth.small_dna(0.5)
        s = ej.Strings.from_set(ss, DEV)
        a = ss.alphabet
        cfg = [(6, 12, 1), (12, 10, 2), (9, 11, 1), (3, 9, 2)]   # (K, z, seed)
        params = [ej.Params(alphabet=a, K=K, r=3, m=8, z=z, seed=sd) for K, z, sd in cfg]
        with torch.cuda.stream(stream):
            b = c.batch(s, params, stream=stream)
            b.run(stream)
            for i, (K, z, sd) in enumerate(cfg):
                got, st = b.result(i, device=DEV, stream=stream)
                ref = oracle.join(ss.data, ss.offsets, a, K=K, r=3, m=8, z=z, seed=sd)
                assert np.array_equal(_u64(got), ref.pairs), (chain, i)
                assert st.n_candidates == ref.n_candidates, (chain, i)
            b.close()
    finally:
        c.close()


def test_batch_moves_huge_buckets_to_global_memory_and_chains_verifiers(ej, ctx, stream):
    """Short protein-like strings whose walks end early share signatures made of
    the bottom symbol: buckets of hundreds of records. The batch's sizing pass
    moves such joins from one block's shared memory to the buckets in global
    memory, and its grid-strided verifiers run one after another; every join
    still equals ej_join and the oracle."""
    ss = synth.protein_like(7, 3000, median=120, lo=20, hi=400)
    s = ej.Strings.from_set(ss, DEV)
    params = [ej.Params(K=K, r=3, m=4, z=8, seed=1, L=600, alphabet=ss.alphabet) for K in (12, 16)]
    with torch.cuda.stream(stream):
        b = ctx.batch(s, params, stream=stream)
        for rep in range(2):
            b.run(stream)
            for i, p in enumerate(params):
                got, st = b.result(i, device=DEV, stream=stream)
                want, st_j = ctx.join(s, p, device=DEV, stream=stream)
                assert np.array_equal(_u64(got), _u64(want))
                assert st.n_candidates == st_j.n_candidates and st.max_bucket > 256
                if rep == 0:
                    ref = oracle.join(ss.data, ss.offsets, ss.alphabet, K=p.K, r=p.r, m=p.m, z=p.z, seed=p.seed,
                                      L=p.L)
                    assert st.n_candidates == ref.n_candidates
                    assert np.array_equal(_u64(got), ref.pairs)
        b.close()
