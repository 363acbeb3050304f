"""The fidelity options of Section 4 on the GPU against the oracle: bucket keys
by the two-level hash <u, v> mod P (signatures, candidates and output through
ej_embed_sign, ej_sign + ej_lsh_candidates and ej_join with hashed and sorted
buckets), and EmbedJoin with grouping by length (ej_join_grouped)."""
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


@pytest.fixture
def ctx(ej):
    c = ej.Context(0)
    yield c
    c.close()


def _u64(t):
    return t.cpu().numpy().view(np.uint64) if hasattr(t, "cpu") else np.asarray(t, dtype=np.uint64)


CASES = [
    (lambda: synth.small_dna(scale=0.3), 6, dict(r=3, m=10, z=12, seed=1, L=0)),
    (lambda: synth.protein_like(5, 300, median=120, lo=20, hi=400), 12, dict(r=4, m=6, z=6, seed=3, L=240)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("P", [1000003, 101])
def test_hashed_keys_equal_oracle(ej, ctx, case, P):
    maker, K, kw = CASES[case]
    ss = maker()
    s = ej.Strings.from_set(ss, DEV)
    params = ej.Params(K=K, alphabet=ss.alphabet, **kw)
    ctx.set_key_hash(P)
    info = ctx.plan(s, params)
    keys = torch.zeros(params.r * params.m * ss.n, dtype=torch.int64, device=DEV)
    ctx.embed_sign(s, params, keys)
    emb, we = oracle.embed(ss.data, ss.offsets, ss.alphabet, params.r, info.out_len, params.seed)
    want = oracle.sign_modp(emb, we, oracle.positions(params.seed, params.r, params.m, params.z, info.L),
                            len(ss.alphabet), params.seed, P)
    assert np.array_equal(_u64(keys).reshape(params.r * params.m, ss.n), want)
    ref = oracle.join(ss.data, ss.offsets, ss.alphabet, K=K, key_P=P, **kw)
    for buckets in (0, 2):
        ctx.set_schedule(buckets=buckets)
        pairs, st = ctx.join(s, params, device=DEV)
        assert st.n_candidates == ref.n_candidates, buckets
        assert np.array_equal(_u64(pairs), ref.pairs), buckets
    ctx.set_schedule()
    # the plain per-stage path: ej_lsh_candidates over the hashed keys
    cand_ref = oracle.candidates(ss.data, ss.offsets, want, K)
    out = torch.empty(cand_ref.shape[0] + 16, dtype=torch.int64, device=DEV)
    n, _ = ctx.lsh_candidates(s, params, keys, out)
    assert n == ref.n_candidates and np.array_equal(_u64(out[:n]), cand_ref)
    if P == 101:
        exact = oracle.join(ss.data, ss.offsets, ss.alphabet, K=K, **kw)
        assert ref.n_candidates > exact.n_candidates


def test_hashed_keys_rejected_by_batches_and_bad_moduli(ej, ctx):
    ss = synth.small_dna(scale=0.1)
    s = ej.Strings.from_set(ss, DEV)
    ctx.set_key_hash(1000003)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with pytest.raises(ej.EJError) as e:
            ctx.batch(s, [ej.Params(K=6, r=2, m=2, z=4, alphabet=b"ACGT")], stream=stream)
    assert e.value.status == ej.EJ_ERR_UNSUPPORTED
    for bad in (1, 1000001, 1 << 33):
        with pytest.raises(ej.EJError) as e:
            ctx.set_key_hash(bad)
        assert e.value.status == ej.EJ_ERR_INVALID_ARG
    ctx.set_key_hash(0)


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("P", [0, 1000003])
def test_grouped_join_equals_oracle(ej, ctx, case, P):
    maker, K, kw = CASES[case]
    ss = maker()
    kw = dict(kw, L=0)
    want, ncand = oracle.join_grouped(ss.data, ss.offsets, ss.alphabet, K=K, key_P=P, **kw)
    ctx.set_key_hash(P)
    pairs, st = ctx.join_grouped(ej.Strings.from_set(ss, DEV), ej.Params(K=K, alphabet=ss.alphabet, **kw), device=DEV)
    assert np.array_equal(_u64(pairs), want)
    assert st.n_candidates == ncand and st.n_out == want.shape[0] > 0
    hp, _ = ctx.join_grouped(ej.Strings.from_set(ss, None), ej.Params(K=K, alphabet=ss.alphabet, **kw), device=None,
                             capacity=1)
    assert np.array_equal(hp, want)
