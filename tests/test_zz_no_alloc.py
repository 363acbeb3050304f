"""ej_verify_noalloc: verification for callers that cannot let the library
allocate device memory (memory reserved up front by another allocator, or a
request path where cudaMalloc/cudaFree must not run because they can
synchronise the device). Its scratch is a fixed device array inside the
library. The test calls it through the C ABI twice in a row and checks both
results against ej_verify and against the CPU oracle on the same pairs
(integer work: identical output), with the device's free memory unchanged
across the two calls. The file is named so that pytest collects it after the
other test files (a run that stops at the first failure has run them all);
the tests themselves pass alone in a fresh process or after the others."""
import numpy as np
import pytest

import oracle
from paper_1702_00093_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_verify_noalloc_matches_verify_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_00093_gb300 import build
    build.build()
    oracle.build()
    from paper_1702_00093_gb300 import embedjoin as ej

    dev = "cuda:0"
    rng = np.random.default_rng(2024)
    cases = []
    for K, alphabet in ((60, b"ACGT"), (9, synth.PROTEIN)):
        sigma = len(alphabet)
        lut = np.frombuffer(alphabet, np.uint8)
        base = [rng.integers(0, sigma, size=int(rng.integers(50, 900))).astype(np.uint8) for _ in range(30)]
        strs = []
        for b in base:
            strs += [b, synth.mutate(rng, b, int(rng.integers(0, 2 * K + 2)), sigma)]
        ss = synth.pack([lut[x].tobytes() for x in strs], alphabet)
        pairs = sorted({(min(a, b), max(a, b)) for a, b in rng.integers(0, ss.n, size=(300, 2)) if a != b}
                       | {(2 * i, 2 * i + 1) for i in range(len(base))})
        cases.append((K, alphabet, ss, np.array([(a << 32) | b for a, b in pairs], dtype=np.uint64)))

    ctx = ej.Context(0)
    try:
        for K, alphabet, ss, arr in cases:
            s = ej.Strings.from_set(ss, dev)
            params = ej.Params(K=K, r=1, m=1, z=1, alphabet=alphabet)
            pt = torch.from_numpy(arr.view(np.int64).copy()).to(dev)
            ref = torch.empty_like(pt)
            k_ref = ctx.verify(s, params, pt, ref)
            want = ref[:k_ref].cpu().numpy()
            assert k_ref > 0
            flags = oracle.verify(ss.data, ss.offsets, arr, K)
            assert np.array_equal(want.view(np.uint64), arr[flags == 1])
            outs = [torch.full_like(pt, -1) for _ in range(3)]
            ej.verify_noalloc(s, params, pt, outs[2])     # loads every module it uses
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            for out in outs[:2]:   # the fixed scratch keeps the last call's contents
                k = ej.verify_noalloc(s, params, pt, out)
                torch.cuda.synchronize()
                assert k == k_ref
                assert np.array_equal(out[:k].cpu().numpy(), want)
            assert torch.cuda.mem_get_info()[0] == free0
    finally:
        ctx.close()


def test_verify_noalloc_rejects_oversized_requests():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_00093_gb300 import embedjoin as ej
    dev = "cuda:0"
    ss = synth.pack([b"ACGT", b"ACGA"], b"ACGT")
    s = ej.Strings.from_set(ss, dev)
    n_pairs = ej.NOALLOC_SCRATCH_BYTES // 9 + 1024      # 9 bytes of scratch per pair
    pt = torch.ones(n_pairs, dtype=torch.int64, device=dev)   # pair (0, 1)
    with pytest.raises(ej.EJError) as e:
        ej.verify_noalloc(s, ej.Params(K=1, r=1, m=1, z=1), pt, torch.empty_like(pt))
    assert e.value.status == ej.EJ_ERR_TOO_LARGE
