"""The autotuner (ej_set_autotune, EJ_BATCH_AUTOTUNE): per (length class, K) it
times the fused walk's block sizes and the verifier choices on the join's own
data and keeps the fastest in the context's table; every autotuned join still
returns the oracle's pair set, a second join of the same class and K uses the
table without tuning again, and a batch records its choices in the same
table."""
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


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


SHAPES = [
    (lambda: synth.small_dna(scale=0.3), 6, dict(r=3, m=10, z=12, seed=1, L=0)),
    (lambda: synth.protein_like(5, 400, median=120, lo=20, hi=400), 12, dict(r=4, m=6, z=6, seed=3, L=240)),
    (lambda: synth.text_like(6, 200, len_lo=100, len_hi=500, rate_lo=0.01, rate_hi=0.1), 40, dict(r=4, m=6, z=5,
                                                                                                    seed=3, L=600)),
    (lambda: synth.dna_clusters(77, 4, 10, 4500, 5500, rate_lo=0.004, rate_hi=0.012), 150,
     dict(r=7, m=20, z=14, seed=1, L=5000)),
]


def test_autotuned_joins_equal_the_oracle_and_fill_the_table(ej):
    c = ej.Context(0)
    try:
        c.set_autotune(1)
        for k, (maker, K, kw) in enumerate(SHAPES):
            ss = maker()
            s = ej.Strings.from_set(ss, DEV)
            params = ej.Params(K=K, alphabet=ss.alphabet, **kw)
            ref = oracle.join(ss.data, ss.offsets, ss.alphabet, K=K, **kw)
            for rep in range(2):
                pairs, st = c.join(s, params, device=DEV)
                assert st.n_candidates == ref.n_candidates, (k, rep)
                assert np.array_equal(_u64(pairs), ref.pairs), (k, rep)
                assert len(c.autotune_table()) == k + 1   # tuned once per (class, K)
        table = c.autotune_table()
        assert all(e["configs_tried"] >= 4 and e["back_ms"] > 0 for e in table)
        assert {e["K"] for e in table} == {K for _, K, _ in SHAPES}
        c.set_autotune(-1)
        assert c.autotune_table() == []
    finally:
        c.close()


def test_autotuned_batch_equals_the_oracle(ej):
    c = ej.Context(0)
    stream = torch.cuda.Stream()
    try:
        ss = synth.protein_like(5, 400, median=120, lo=20, hi=400)
        s = ej.Strings.from_set(ss, DEV)
        kws = [dict(K=12, r=4, m=6, z=6, seed=3, L=240), dict(K=20, r=4, m=6, z=5, seed=3, L=240)]
        params = [ej.Params(alphabet=ss.alphabet, **kw) for kw in kws]
        with torch.cuda.stream(stream):
            b = c.batch(s, params, autotune=True, stream=stream)
            b.run(stream)
            for i, kw in enumerate(kws):
                got, st = b.result(i, device=DEV, stream=stream)
                ref = oracle.join(ss.data, ss.offsets, ss.alphabet, **kw)
                assert st.n_candidates == ref.n_candidates
                assert np.array_equal(_u64(got), ref.pairs)
            b.close()
        assert len(c.autotune_table()) == 2
    finally:
        c.close()
