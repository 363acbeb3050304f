"""EmbedJoin+ on the GPU (ej_join_plus, Section 5) against the oracle's
Algorithms 4 and 5: the same candidate count and the same output pair set on
DNA (2-bit codes) and larger alphabets (8-bit codes), with one substring per
string (where it is EmbedJoin), with several substrings and T = 2, on strings
shifted by inserted prefixes (where it finds what EmbedJoin misses), on long
strings and with host buffers."""
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


def _u64(t):
    return t.cpu().numpy().view(np.uint64) if hasattr(t, "cpu") else np.asarray(t, dtype=np.uint64)


def _shifted(seed, pairs=40, length=400, shift=(15, 31), edits=3):
    rng = np.random.default_rng(seed)
    lut = np.frombuffer(b"ACGT", np.uint8)
    strs = []
    for _ in range(pairs):
        x = rng.integers(0, 4, size=length).astype(np.uint8)
        y = np.concatenate([rng.integers(0, 4, size=int(rng.integers(*shift))).astype(np.uint8),
                            synth.mutate(rng, x, edits, 4)])
        strs += [lut[x].tobytes(), lut[y].tobytes()]
    return synth.pack(strs, b"ACGT")


def _check(ej, ctx, ss, K, r, m, z, seed, delta, T, L=0, device=DEV):
    ref = oracle.join_plus(ss.data, ss.offsets, ss.alphabet, K=K, r=r, m=m, z=z, seed=seed, L=L, delta=delta, T=T)
    s = ej.Strings.from_set(ss, device)
    pairs, st = ctx.join_plus(s, ej.Params(K=K, r=r, m=m, z=z, seed=seed, L=L, alphabet=ss.alphabet), delta, T,
                              device=device)
    assert st.n_candidates == ref.n_candidates
    assert st.n_raw_pairs == ref.n_tuples
    assert np.array_equal(_u64(pairs), ref.pairs)
    return ref, st


def test_one_substring_is_embedjoin(ej, ctx):
    ss = synth.small_dna(scale=0.3)
    p = synth.SMALL_DNA_PARAMS
    ref, st = _check(ej, ctx, ss, p["K"], p["r"], p["m"], p["z"], p["seed"], delta=p["K"], T=1)
    pairs, stj = ctx.join(ej.Strings.from_set(ss, DEV), ej.Params(alphabet=ss.alphabet, **p), device=DEV)
    assert stj.n_candidates == st.n_candidates and np.array_equal(_u64(pairs), ref.pairs)


@pytest.mark.parametrize("K,delta,T", [(6, 2, 2), (6, 3, 1), (9, 4, 3), (0, 5, 1)])
def test_small_dna_several_substrings(ej, ctx, K, delta, T):
    ss = synth.small_dna(scale=0.3)
    ref, st = _check(ej, ctx, ss, K, 3, 10, 12, 1, delta, T)
    if K:
        assert ref.n_candidates > 0


def test_shifted_strings(ej, ctx):
    ss = _shifted(3)
    ref, st = _check(ej, ctx, ss, 40, 7, 16, 12, 1, delta=10, T=2, L=400)
    truth = {(2 * i) << 32 | (2 * i + 1) for i in range(40)}
    assert len(truth & set(ref.pairs.tolist())) >= 32


@pytest.mark.parametrize("maker,K,delta", [
    (lambda: synth.protein_like(5, 300, median=120, lo=20, hi=400), 12, 5),
    (lambda: synth.text_like(6, 200, len_lo=50, len_hi=300, rate_lo=0.01, rate_hi=0.1), 20, 8),
])
def test_large_alphabets(ej, ctx, maker, K, delta):
    ss = maker()
    L = int(2 * ss.lengths().mean())
    _check(ej, ctx, ss, K, 4, 6, 5, 3, delta, 2, L=L)


def test_long_strings(ej, ctx):
    """Long DNA strings (4 clusters of 10 strings of 4500-5500 symbols, member
    edit rate 0.4-1.2%): K = 150 with delta = 70 (about the square root of the
    mean length), 3 substrings, T = 2, 16 functions."""
    ss = synth.dna_clusters(77, 4, 10, 4500, 5500, rate_lo=0.004, rate_hi=0.012)
    p = synth.long_dna_params(150)
    ref, _ = _check(ej, ctx, ss, 150, p["r"], 16, p["z"], p["seed"], delta=70, T=2, L=p["L"])
    assert len(ref.pairs) > 100


def test_host_buffers_and_capacity(ej, ctx):
    ss = _shifted(4, pairs=12)
    ref = oracle.join_plus(ss.data, ss.offsets, b"ACGT", K=40, r=7, m=16, z=12, seed=1, L=400, delta=10, T=2)
    pairs, st = ctx.join_plus(ej.Strings.from_set(ss, None), ej.Params(K=40, r=7, m=16, z=12, seed=1, L=400),
                              10, 2, device=None, capacity=1)
    assert np.array_equal(pairs, ref.pairs) and len(ref.pairs) > 1
    with pytest.raises(ej.EJError) as e:
        ctx.join_plus(ej.Strings.from_set(ss, DEV), ej.Params(K=40, r=7, m=16, z=12, seed=1, L=400), 0, 2)
    assert e.value.status == ej.EJ_ERR_INVALID_ARG
