"""GPU parity: every stage of the CUDA path (called through the C ABI) against
the CPU oracle on the same seeded inputs. All of this is integer work, so the
bar is bit-identical output: embeddings, walk ends, keys, candidate sets and
output pair sets."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1702_00093_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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


DEV = "cuda:0"


def _np_u64(t):
    return t.cpu().numpy().view(np.uint64) if t.dtype == torch.int64 else t.cpu().numpy().astype(np.uint64)


def gpu_embed(ej, ctx, ss, params):
    s = ej.Strings.from_set(ss, DEV)
    info = ctx.plan(s, params)
    emb = torch.zeros(max(info.embedding_bytes // 4, 1), dtype=torch.int32, device=DEV)
    we = torch.zeros(max(params.r * ss.n, 1), dtype=torch.int32, device=DEV)
    ctx.embed(s, params, emb, we)
    torch.cuda.synchronize()
    codes = ej.decode_embedding(emb.cpu().numpy().view(np.uint32)[: info.embedding_bytes // 4],
                                we.cpu().numpy()[: params.r * ss.n].reshape(params.r, ss.n),
                                params.r, ss.n, info.out_len, info.planes, len(ss.alphabet))
    return s, info, emb, we, codes


def gpu_keys(ej, ctx, s, params, emb, we, n):
    keys = torch.zeros(params.r * params.m * n, dtype=torch.int64, device=DEV)
    ctx.sign(s, params, emb, we, keys)
    torch.cuda.synchronize()
    return _np_u64(keys).reshape(params.r * params.m, n)


def gpu_candidates(ej, ctx, s, params, keys_np):
    keys = torch.from_numpy(keys_np.view(np.int64).ravel().copy()).to(DEV)
    try:
        n, mb = ctx.lsh_candidates(s, params, keys, torch.empty(1, dtype=torch.int64, device=DEV))
        out = torch.empty(max(n, 1), dtype=torch.int64, device=DEV)
    except ej.EJError as e:
        assert e.status == ej.EJ_ERR_CAPACITY
        out = torch.empty(e.needed, dtype=torch.int64, device=DEV)
    n, mb = ctx.lsh_candidates(s, params, keys, out)
    return _np_u64(out[:n])


def check_all_stages(ej, ctx, ss, params, check_join=True):
    s, info, emb, we, codes = gpu_embed(ej, ctx, ss, params)
    ref_emb, ref_we = oracle.embed(ss.data, ss.offsets, ss.alphabet, params.r, info.out_len, params.seed)
    assert np.array_equal(we.cpu().numpy()[: params.r * ss.n].reshape(params.r, ss.n), ref_we)
    assert np.array_equal(codes, ref_emb)
    pos = oracle.positions(params.seed, params.r, params.m, params.z, info.L)
    ref_keys = oracle.sign(ref_emb, ref_we, pos, len(ss.alphabet))
    keys = gpu_keys(ej, ctx, s, params, emb, we, ss.n)
    assert np.array_equal(keys, ref_keys)
    fused = torch.zeros(params.r * params.m * ss.n, dtype=torch.int64, device=DEV)
    ctx.embed_sign(s, params, fused)
    assert np.array_equal(_np_u64(fused).reshape(params.r * params.m, ss.n), ref_keys)
    cand = gpu_candidates(ej, ctx, s, params, keys)
    ref_cand = oracle.candidates(ss.data, ss.offsets, ref_keys, params.K)
    assert np.array_equal(cand, ref_cand)
    if len(cand):
        pt = torch.from_numpy(cand.view(np.int64).copy()).to(DEV)
        out = torch.empty_like(pt)
        k = ctx.verify(s, params, pt, out)
        flags = oracle.verify(ss.data, ss.offsets, cand, params.K)
        assert np.array_equal(_np_u64(out[:k]), cand[flags == 1])
    if check_join:
        pairs, stats = ctx.join(s, params, device=DEV)
        ref = oracle.join(ss.data, ss.offsets, ss.alphabet, K=params.K, r=params.r, m=params.m,
                          z=params.z, seed=params.seed, L=params.L, out_len=params.out_len)
        assert stats.n_candidates == ref.n_candidates
        assert np.array_equal(_np_u64(pairs), ref.pairs)
    return cand


# ---------------------------------------------------------------------------
# The paper's running example (Section 4, Tables 2-4) through the injection hook
# ---------------------------------------------------------------------------

def test_running_example_on_gpu(ej, ctx, golden):
    g = golden("running_example_sec4.json")
    ss = synth.pack([x.encode() for x in g["strings"]], b"ACGT")
    pi = np.zeros((2, 10, 4), dtype=np.uint8)
    for l, name in enumerate(["R1", "R2"]):
        for c, ch in enumerate("ACGT"):
            pi[l, :, c] = g["pi_steps_1_to_10"][name][ch]
    f = g["functions_1based_positions"]
    pos = np.array([[f["f1^1"], f["f2^1"]], [f["f1^2"], f["f2^2"]]], dtype=np.uint32) - 1
    params = ej.Params(K=3, r=2, m=2, z=2, seed=0, L=10, out_len=10, alphabet=b"ACGT")
    ctx.set_test_tables(pi, pos)
    try:
        s, info, emb, we, codes = gpu_embed(ej, ctx, ss, params)
        for i in range(4):
            for l in range(2):
                assert "".join("ACGT"[c] for c in codes[l, i]) == g["embedded_prefixes"][f"t{i + 1}^{l + 1}"]
        keys = gpu_keys(ej, ctx, s, params, emb, we, 4)
        fused = torch.zeros(16, dtype=torch.int64, device=DEV)
        ctx.embed_sign(s, params, fused)
        assert np.array_equal(_np_u64(fused).reshape(4, 4), keys)
        for i in range(4):
            for col in range(4):
                sig = g["signatures"][str(i + 1)][col]
                assert int(keys[col, i]) == "ACGT".index(sig[0]) + 5 * "ACGT".index(sig[1])
        cand = gpu_candidates(ej, ctx, s, params, keys)
        assert [(int(p >> 32) + 1, int(p & 0xFFFFFFFF) + 1) for p in cand] == [tuple(x) for x in g["candidates_1based"]]
        pairs, _ = ctx.join(s, params, device=DEV)
        got = [(int(p >> 32) + 1, int(p & 0xFFFFFFFF) + 1) for p in _np_u64(pairs)]
        assert got == [tuple(x) for x in g["output_1based"]]
    finally:
        ctx.set_test_tables()


def test_worked_example_on_gpu(ej, ctx, golden):
    g = golden("worked_example_sec1.json")
    ss = synth.pack([x.encode() for x in g["strings"]], b"ACGT")
    s = ej.Strings.from_set(ss, DEV)
    params = ej.Params(K=2, r=7, m=16, z=2, seed=5, alphabet=b"ACGT")
    pairs, _ = ctx.join(s, params, device=DEV)
    got = [(int(p >> 32), int(p & 0xFFFFFFFF)) for p in _np_u64(pairs)]
    assert got == [tuple(x) for x in g["expected_pairs_0based"]]
    # verification alone on all pairs equals the definition
    allp = np.array([(i << 32) | j for i, j in itertools.combinations(range(5), 2)], dtype=np.uint64)
    pt = torch.from_numpy(allp.view(np.int64).copy()).to(DEV)
    out = torch.empty_like(pt)
    k = ctx.verify(s, params, pt, out)
    assert [(int(p >> 32), int(p & 0xFFFFFFFF)) for p in _np_u64(out[:k])] == got


# ---------------------------------------------------------------------------
# Stage-by-stage parity on the workload shapes
# ---------------------------------------------------------------------------

def test_small_dna_full_config(ej, ctx):
    """n=1000 DNA, 100 clusters of 10, K=6, r=3, m=10, z=12 (L = 3N)."""
    ss = synth.small_dna()
    p = synth.SMALL_DNA_PARAMS
    params = ej.Params(K=p["K"], r=p["r"], m=p["m"], z=p["z"], seed=p["seed"], alphabet=ss.alphabet)
    cand = check_all_stages(ej, ctx, ss, params)
    assert len(cand) > 1000


@pytest.mark.parametrize("K", [50, 150, 250])
def test_long_dna_shape(ej, ctx, K):
    """Strings shaped like the long-DNA workload (length ~5000, 1-8% edits)."""
    ss = synth.long_dna(n_clusters=4, seed=77)
    p = synth.long_dna_params(K)
    params = ej.Params(K=K, r=p["r"], m=p["m"], z=p["z"], seed=p["seed"], L=p["L"], alphabet=ss.alphabet)
    check_all_stages(ej, ctx, ss, params)


@pytest.mark.parametrize("maker,K,z", [
    (lambda: synth.protein_like(5, 300, median=120, lo=20, hi=400), 12, 8),
    (lambda: synth.text_like(6, 300, len_lo=50, len_hi=300, rate_lo=0.01, rate_hi=0.1), 20, 6),
])
def test_large_alphabets(ej, ctx, maker, K, z):
    ss = maker()
    L = int(2 * ss.lengths().mean())
    params = ej.Params(K=K, r=4, m=6, z=z, seed=3, L=L, alphabet=ss.alphabet)
    check_all_stages(ej, ctx, ss, params)


def test_ragged_and_degenerate_strings(ej, ctx):
    """Empty strings, identical strings (one big bucket), n not a multiple of 32."""
    rng = np.random.default_rng(8)
    strs = [b"", b"", b"A", b"AC", b"ACGT" * 10, b"ACGT" * 10, b"ACGA" * 10]
    strs += [bytes(rng.choice(list(b"ACGT"), size=int(rng.integers(0, 90))).astype(np.uint8)) for _ in range(70)]
    strs += [b"GATTACA" * 5] * 12
    ss = synth.pack(strs, b"ACGT")
    for K in (0, 1, 3, 40):
        params = ej.Params(K=K, r=3, m=5, z=3, seed=11, alphabet=b"ACGT")
        check_all_stages(ej, ctx, ss, params)


@pytest.mark.parametrize("alphabet", [b"ACGT", synth.TEXT])
@pytest.mark.parametrize("shift", [0, 1, 2, 3])
def test_pack_at_every_alignment(ej, ctx, alphabet, shift):
    """Packing reads the byte array as aligned words where it can: strings of
    every length 0..70 start at every byte offset, in an array whose own start is
    shifted by 0..3 bytes; the embedding (which consumes every code) equals the
    oracle's."""
    rng = np.random.default_rng(11 + shift)
    lut = np.frombuffer(alphabet, np.uint8)
    strs = [lut[rng.integers(0, len(alphabet), size=int(L))].tobytes() for L in rng.permutation(71)]
    ss = synth.pack(strs, alphabet)
    big = torch.zeros(len(ss.data) + 8, dtype=torch.uint8, device=DEV)
    big[shift:shift + len(ss.data)] = torch.from_numpy(ss.data).to(DEV)
    s = ej.Strings(big[shift:shift + len(ss.data)], torch.from_numpy(ss.offsets).to(DEV))
    params = ej.Params(K=3, r=2, m=2, z=3, seed=7, alphabet=alphabet)
    info = ctx.plan(s, params)
    emb = torch.zeros(max(info.embedding_bytes // 4, 1), dtype=torch.int32, device=DEV)
    we = torch.zeros(max(params.r * ss.n, 1), dtype=torch.int32, device=DEV)
    ctx.embed(s, params, emb, we)
    torch.cuda.synchronize()
    codes = ej.decode_embedding(emb.cpu().numpy().view(np.uint32)[: info.embedding_bytes // 4],
                                we.cpu().numpy()[: params.r * ss.n].reshape(params.r, ss.n),
                                params.r, ss.n, info.out_len, info.planes, len(alphabet))
    ref_emb, ref_we = oracle.embed(ss.data, ss.offsets, alphabet, params.r, info.out_len, params.seed)
    assert np.array_equal(codes, ref_emb)
    assert np.array_equal(we.cpu().numpy()[: params.r * ss.n].reshape(params.r, ss.n), ref_we)


def test_tiny_inputs(ej, ctx):
    params = ej.Params(K=2, r=2, m=2, z=2, seed=1, alphabet=b"ACGT")
    for strs in ([], [b"ACGT"], [b"", b""], [b"A", b"C"]):
        ss = synth.pack(strs, b"ACGT")
        s = ej.Strings.from_set(ss, DEV) if strs else ej.Strings(
            torch.zeros(1, dtype=torch.uint8, device=DEV), torch.zeros(1, dtype=torch.int64, device=DEV))
        pairs, _ = ctx.join(s, params, device=DEV)
        want = oracle.join(ss.data, ss.offsets, b"ACGT", K=2, r=2, m=2, z=2, seed=1).pairs \
            if strs else np.zeros(0, np.uint64)
        assert np.array_equal(_np_u64(pairs), want)
        # precision: every output pair is a true pair
        truth = set(oracle.join_bruteforce(ss.data, ss.offsets, 2).tolist()) if strs else set()
        assert set(_np_u64(pairs).tolist()) <= truth


# ---------------------------------------------------------------------------
# Verification kernel: many thresholds, lengths and band widths
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("K", [0, 1, 5, 31, 32, 63, 64, 100, 200, 300, 500, 1000])
def test_verify_random_pairs(ej, ctx, K):
    rng = np.random.default_rng(K + 1)
    base = [rng.integers(0, 4, size=int(rng.integers(0, 1500))).astype(np.uint8) for _ in range(40)]
    strs = []
    for b in base:
        strs.append(b)
        strs.append(synth.mutate(rng, b, int(rng.integers(0, max(2, 2 * K + 5))), 4))
    strs = [np.frombuffer(b"ACGT", np.uint8)[s].tobytes() for s in strs]
    ss = synth.pack(strs, b"ACGT")
    n = ss.n
    pairs = sorted({(min(a, b), max(a, b)) for a, b in rng.integers(0, n, size=(600, 2)) if a != b}
                   | {(2 * i, 2 * i + 1) for i in range(len(base))})
    arr = np.array([(a << 32) | b for a, b in pairs], dtype=np.uint64)
    s = ej.Strings.from_set(ss, DEV)
    params = ej.Params(K=K, r=1, m=1, z=1, alphabet=b"ACGT")
    pt = torch.from_numpy(arr.view(np.int64).copy()).to(DEV)
    out = torch.empty_like(pt)
    k = ctx.verify(s, params, pt, out)
    flags = oracle.verify(ss.data, ss.offsets, arr, K)
    assert np.array_equal(_np_u64(out[:k]), arr[flags == 1])
    assert flags.sum() > 0


def test_verify_host_buffers_and_unsorted_pairs(ej, ctx):
    """Host (numpy) inputs and outputs through the same entry point; order kept."""
    rng = np.random.default_rng(3)
    ss = synth.dna_clusters(4, 10, 5, 50, 80, edits_mean=3.0)
    s = ej.Strings.from_set(ss, None)
    pairs = np.array([(int(a) << 32) | int(b) for a, b in rng.integers(0, ss.n, size=(300, 2)) if a != b],
                     dtype=np.uint64)
    out = np.zeros_like(pairs)
    params = ej.Params(K=4, r=1, m=1, z=1, alphabet=b"ACGT")
    k = ctx.verify(s, params, pairs, out)
    flags = oracle.verify(ss.data, ss.offsets, pairs, 4)
    assert np.array_equal(out[:k], pairs[flags == 1])


def test_join_host_buffers_equal_device(ej, ctx):
    ss = synth.small_dna(scale=0.2)
    p = synth.SMALL_DNA_PARAMS
    params = ej.Params(K=p["K"], r=p["r"], m=p["m"], z=p["z"], seed=p["seed"], alphabet=ss.alphabet)
    host_pairs, _ = ctx.join(ej.Strings.from_set(ss, None), params, device=None)
    dev_pairs, _ = ctx.join(ej.Strings.from_set(ss, DEV), params, device=DEV)
    assert np.array_equal(host_pairs, _np_u64(dev_pairs))


# ---------------------------------------------------------------------------
# Errors are reported, not faulted
# ---------------------------------------------------------------------------

def test_invalid_inputs_are_rejected(ej, ctx):
    ss = synth.pack([b"ACGT", b"ACGN"], b"ACGT")
    params = ej.Params(K=1, r=1, m=1, z=1, alphabet=b"ACGT")
    with pytest.raises(ej.EJError) as e:
        ctx.join(ej.Strings.from_set(ss, DEV), params, device=DEV)
    assert e.value.status == ej.EJ_ERR_INVALID_ARG
    bad = ej.Strings(torch.zeros(8, dtype=torch.uint8, device=DEV) + 65,
                     torch.tensor([0, 5, 3], dtype=torch.int64, device=DEV))
    with pytest.raises(ej.EJError) as e:
        ctx.join(bad, ej.Params(K=1, r=1, m=1, z=1, alphabet=b"A"), device=DEV)
    assert e.value.status == ej.EJ_ERR_INVALID_ARG
    # a string starting before the array (the one before it is negative too)
    bad = ej.Strings(torch.zeros(8, dtype=torch.uint8, device=DEV) + 65,
                     torch.tensor([0, -3, 5], dtype=torch.int64, device=DEV))
    with pytest.raises(ej.EJError) as e:
        ctx.join(bad, ej.Params(K=1, r=1, m=1, z=1, alphabet=b"A"), device=DEV)
    assert e.value.status == ej.EJ_ERR_INVALID_ARG
    with pytest.raises(ej.EJError) as e:
        ctx.join(ej.Strings.from_set(synth.pack([b"A", b"A"], b"A"), DEV),
                 ej.Params(K=1, r=1, m=1, z=100, alphabet=b"A"), device=DEV)
    assert e.value.status == ej.EJ_ERR_INVALID_ARG
    pairs = torch.tensor([(0 << 32) | 7], dtype=torch.int64, device=DEV)
    with pytest.raises(ej.EJError) as e:
        ctx.verify(ej.Strings.from_set(synth.pack([b"A", b"A"], b"A"), DEV),
                   ej.Params(K=1, r=1, m=1, z=1, alphabet=b"A"), pairs, torch.empty_like(pairs))
    assert e.value.status == ej.EJ_ERR_INVALID_ARG
    # the context still works afterwards
    test_tiny_inputs(ej, ctx)


def test_capacity_reports_needed_count(ej, ctx):
    ss = synth.pack([b"ACGT"] * 10, b"ACGT")
    params = ej.Params(K=0, r=1, m=1, z=2, alphabet=b"ACGT")
    s = ej.Strings.from_set(ss, DEV)
    with pytest.raises(ej.EJError) as e:
        ctx.join_into(s, params, torch.empty(3, dtype=torch.int64, device=DEV))
    assert e.value.status == ej.EJ_ERR_CAPACITY and e.value.needed == 45


@pytest.mark.parametrize("K,alphabet", [(5, b"ACGT"), (60, b"ACGT"), (150, b"ACGT"), (40, synth.PROTEIN)])
def test_verify_every_tiling_is_exact(ej, ctx, K, alphabet):
    """Every lanes-per-pair x words-per-lane tiling that covers the band gives the oracle's answer."""
    rng = np.random.default_rng(K)
    sigma = len(alphabet)
    base = [rng.integers(0, sigma, size=int(rng.integers(1, 700))).astype(np.uint8) for _ in range(24)]
    strs = []
    for b in base:
        strs += [b, synth.mutate(rng, b, int(rng.integers(0, 2 * K + 3)), sigma)]
    lut = np.frombuffer(alphabet, np.uint8)
    ss = synth.pack([lut[x].tobytes() for x in strs], alphabet)
    pairs = sorted({(min(a, b), max(a, b)) for a, b in rng.integers(0, ss.n, size=(200, 2)) if a != b}
                   | {(2 * i, 2 * i + 1) for i in range(len(base))})
    arr = np.array([(a << 32) | b for a, b in pairs], dtype=np.uint64)
    want = arr[oracle.verify(ss.data, ss.offsets, arr, K) == 1]
    s = ej.Strings.from_set(ss, DEV)
    params = ej.Params(K=K, r=1, m=1, z=1, alphabet=alphabet)
    pt = torch.from_numpy(arr.view(np.int64).copy()).to(DEV)
    tried = 0
    try:
        W = (2 * K + 1 + 63) // 64
        for G in (1, 2, 4, 8, 16, 32):
            Vs = {1: range(1, 9), 2: range(2, 13)}.get(G, range(1, 5))
            for V in Vs:
                cover = 64 * (V - 1) if G == 2 else 64 * G * V
                if cover < 2 * K + 1 or G * V > 4 * max(1, W) + 2:
                    continue
                ctx.set_verify_config(G, V, 0)
                out = torch.empty_like(pt)
                k = ctx.verify(s, params, pt, out)
                assert np.array_equal(_np_u64(out[:k]), want), (G, V)
                tried += 1
    finally:
        ctx.set_verify_config(0, 0, 0)
    assert tried >= 3


def _near_pair_set(rng, K, alphabet, n_base=20, max_len=700):
    """Bases of random length with one mutated copy each (0 .. 2K+2 edits): many
    candidates on both sides of the threshold."""
    sigma = len(alphabet)
    base = [rng.integers(0, sigma, size=int(rng.integers(1, max_len))).astype(np.uint8) for _ in range(n_base)]
    strs = []
    for b in base:
        strs += [b, synth.mutate(rng, b, int(rng.integers(0, 2 * K + 3)), sigma)]
    lut = np.frombuffer(alphabet, np.uint8)
    return synth.pack([lut[x].tobytes() for x in strs], alphabet)


@pytest.mark.parametrize("K,alphabet", [(6, b"ACGT"), (60, b"ACGT"), (150, b"ACGT"), (40, synth.PROTEIN),
                                        (90, synth.TEXT)])
def test_join_every_schedule_and_window_is_exact(ej, ctx, K, alphabet):
    """ej_join's back half under every schedule (persistent work queue with 1..16
    slots per warp and capped warps, grid-strided, shared-string; collision-count,
    hash, first-string, length-class or longer-string order; hashed or sorted
    buckets) and every two-lane window width gives the oracle's pair set."""
    rng = np.random.default_rng(1000 + K)
    ss = _near_pair_set(rng, K, alphabet)
    z = 3 if len(alphabet) == 4 else 2
    params = ej.Params(K=K, r=4, m=8, z=z, seed=5, L=200, alphabet=alphabet)
    ref = oracle.join(ss.data, ss.offsets, ss.alphabet, K=K, r=4, m=8, z=z, seed=5, L=200)
    assert ref.n_candidates > 20 and 0 < len(ref.pairs) < ref.n_candidates
    s = ej.Strings.from_set(ss, DEV)
    W = (2 * K + 1 + 63) // 64
    runs = 0
    try:
        for sched in [(0, 0, 0, 0, 0), (2, 0, 0, 0, 0), (1, 0, 0, 0, 0), (1, 1, 0, 0, 2), (1, 2, 0, 2, 0),
                      (1, 5, 1, 0, 2), (1, 16, 1, 1, 1), (1, 16, 2, 2, 0), (1, 3, 1, 0, 0), (2, 0, 0, 2, 2),
                      (2, 0, 0, 3, 0), (1, 16, 1, 3, 0), (0, 0, 0, 3, 2), (1, 16, 1, 4, 0), (2, 0, 0, 4, 2),
                      (3, 0, 0, 0, 0), (3, 0, 0, 0, 2), (3, 0, 0, 0, 1), (2, 0, 0, 5, 0), (1, 16, 1, 5, 0)]:
            ctx.set_schedule(*sched)
            pairs, stats = ctx.join(s, params, device=DEV)
            assert stats.n_candidates == ref.n_candidates
            assert np.array_equal(_np_u64(pairs), ref.pairs), sched
            runs += 1
        for mode in (1, 3):   # the persistent and shared-string verifiers at every window width
            ctx.set_schedule(mode, 0)
            for V in range(W + 1, 13):
                ctx.set_verify_config(2, V, 0)
                pairs, _ = ctx.join(s, params, device=DEV)
                assert np.array_equal(_np_u64(pairs), ref.pairs), (mode, V)
                runs += 1
    finally:
        ctx.set_schedule(0, 0)
        ctx.set_verify_config(0, 0, 0)
    assert runs >= 7


@pytest.mark.parametrize("n", [21845, 21846])
def test_buckets_in_shared_memory_and_global(ej, ctx, n):
    """Tables of up to 21845 records are bucketed in shared memory, larger ones in
    global memory: at the boundary both give the sorted path's pairs, and the
    smaller set's pairs equal the oracle's (short strings over ACGT with z = 4,
    so the buckets hold dozens of records)."""
    rng = np.random.default_rng(n)
    lut = np.frombuffer(b"ACGT", np.uint8)
    strs = [lut[rng.integers(0, 4, size=int(rng.integers(8, 13)))].tobytes() for _ in range(n)]
    ss = synth.pack(strs, b"ACGT")
    s = ej.Strings.from_set(ss, DEV)
    params = ej.Params(K=1, r=2, m=3, z=4, seed=9, alphabet=b"ACGT")
    try:
        ctx.set_schedule(buckets=0)
        hashed, st_h = ctx.join(s, params, device=DEV, capacity=1 << 20)
        ctx.set_schedule(buckets=2)
        srt, st_s = ctx.join(s, params, device=DEV, capacity=1 << 20)
    finally:
        ctx.set_schedule()
    assert st_h.n_candidates == st_s.n_candidates > 1000 and st_h.n_raw_pairs == st_s.n_raw_pairs
    assert st_h.max_bucket > 20
    assert np.array_equal(_np_u64(hashed), _np_u64(srt))
    if n == 21845:
        ref = oracle.join(ss.data, ss.offsets, b"ACGT", K=1, r=2, m=3, z=4, seed=9)
        assert ref.n_candidates == st_h.n_candidates
        assert np.array_equal(_np_u64(hashed), ref.pairs)


@pytest.mark.parametrize("maker,K", [
    (lambda: synth.protein_like(21, 2000, median=150, lo=30, hi=600), 40),
    (lambda: synth.text_like(22, 600, len_lo=200, len_hi=900, rate_lo=0.02, rate_hi=0.2), 150),
    (lambda: synth.dna_clusters(23, 40, 10, 200, 400, edits_mean=10.0), 30),
])
def test_shared_string_verifier_tasks(ej, ctx, maker, K):
    """The shared-string verifier on candidate sets whose longer strings have from
    one to hundreds of pairs (tasks of 1..16 pairs), ragged lengths, and 2-bit
    and 8-bit codes: the oracle's pair set, also through the plain ej_verify of
    the same candidates."""
    ss = maker()
    L = int(2 * ss.lengths().mean())
    params = ej.Params(K=K, r=4, m=6, z=4, seed=8, L=L, alphabet=ss.alphabet)
    ref = oracle.join(ss.data, ss.offsets, ss.alphabet, K=K, r=4, m=6, z=4, seed=8, L=L)
    assert ref.n_candidates > 200 and len(ref.pairs) > 0
    s = ej.Strings.from_set(ss, DEV)
    try:
        for mode in (3, 0):
            ctx.set_schedule(mode, 0)
            pairs, st = ctx.join(s, params, device=DEV)
            assert st.n_candidates == ref.n_candidates
            assert np.array_equal(_np_u64(pairs), ref.pairs), mode
    finally:
        ctx.set_schedule()
