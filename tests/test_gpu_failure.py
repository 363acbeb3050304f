"""Failure detection without a GPU fault: the persistent verifier bounds the
passes of each warp's work loop. A test hook lowers the bound so that it runs
out on ordinary input; the kernel then records the event and returns, the call
reports EJ_ERR_TIMEOUT, and the same context afterwards answers exactly (the
oracle's pairs). Nothing here faults, traps or hangs the GPU: the bound is a
counter in the kernel's own loop."""
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


def _case():
    # 3 clusters of 8 DNA strings of 2500-3000 symbols, ~12 edits per member:
    # every pair of a cluster is a candidate and most pass K = 60
    ss = synth.dna_clusters(41, 3, 8, 2500, 3000, edits_mean=12.0)
    return ss, dict(K=60, r=4, m=8, z=10, seed=3, L=2500)


def test_loop_bound_runs_out_then_context_still_exact(ej):
    ss, p = _case()
    ref = oracle.join(ss.data, ss.offsets, ss.alphabet, K=p["K"], r=p["r"], m=p["m"], z=p["z"], seed=p["seed"],
                      L=p["L"])
    assert len(ref.pairs) > 0
    c = ej.Context(0)
    try:
        s = ej.Strings.from_set(ss, DEV)
        params = ej.Params(alphabet=ss.alphabet, **p)
        c.set_schedule(mode=1)                     # the persistent verifier
        c.set_loop_bound(2)                        # a pair of ~2700 columns needs ~22 passes
        with pytest.raises(ej.EJError) as e:
            c.join(s, params, device=DEV)
        assert e.value.status == ej.EJ_ERR_TIMEOUT
        torch.cuda.synchronize()                   # the device is fine
        c.set_loop_bound(0)
        pairs, st = c.join(s, params, device=DEV)
        assert st.n_candidates == ref.n_candidates
        assert np.array_equal(pairs.cpu().numpy().view(np.uint64), ref.pairs)
        with pytest.raises(ej.EJError) as e:
            c.set_loop_bound(-1)
        assert e.value.status == ej.EJ_ERR_INVALID_ARG
    finally:
        c.close()


def test_loop_bound_in_a_batch(ej):
    """A batch whose joins use the persistent verifier: with a tiny bound its
    creation (which runs every join once) reports EJ_ERR_TIMEOUT; with the
    default bound the same context builds the batch and every join is exact."""
    ss, p = _case()
    c = ej.Context(0)
    stream = torch.cuda.Stream()
    try:
        s = ej.Strings.from_set(ss, DEV)
        params = [ej.Params(alphabet=ss.alphabet, **dict(p, K=K)) for K in (20, 60)]
        c.set_schedule(mode=1)
        c.set_loop_bound(2)
        with torch.cuda.stream(stream):
            with pytest.raises(ej.EJError) as e:
                c.batch(s, params, stream=stream)
            assert e.value.status == ej.EJ_ERR_TIMEOUT
            c.set_loop_bound(0)
            b = c.batch(s, params, stream=stream)
            b.run(stream)
            for i, q in enumerate(params):
                got, _ = b.result(i, device=DEV, stream=stream)
                want = oracle.join(ss.data, ss.offsets, ss.alphabet, K=q.K, r=q.r, m=q.m, z=q.z, seed=q.seed, L=q.L)
                assert np.array_equal(got.cpu().numpy().view(np.uint64), want.pairs)
            b.close()
    finally:
        c.close()
