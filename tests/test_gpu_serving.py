"""Continuous-batching server: results alone == results in the mix.

Requests of short reads (150 bp) and long reads (lognormal lengths, indels)
are submitted together to a server with several slots; waiting requests are
merged into shared batched passes and slots run concurrently on their own
streams. Every request's anchors must equal those of the same reads seeded
alone through god_seed (integer results: exact), a sample must equal the
oracle's, the server must actually have merged requests and overlapped
batches, and a request larger than the memory budget must be refused with
GOD_ENOMEM while the others complete.
"""
import numpy as np
import pytest

import oracle
from paper_2211_08157_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2211_08157_gb300 as god
    god.load()
    ref = synth.reference(3_000_000, 51, synth.RepeatModel(30, 500, 3000, False, 0.0, 0.02, 0.05))
    idx = god.god_build_index(ref, "10", 21, 11, 500)
    return god, ref, idx


def make_requests(ref, n_req, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    long_len = synth.LengthModel("lognormal", mu=8.5, sigma=0.5, lo=500, hi=20_000)
    for r in range(n_req):
        g = np.random.default_rng(seed * 1000 + r)
        if rng.random() < 0.6:
            n = int(rng.integers(1, 3000))
            reads, offs, _ = synth.reads(ref, n, synth.SHORT, synth.ILLUMINA_INDEL, 0, rng=g)
        else:
            n = int(rng.integers(1, 60))
            reads, offs, _ = synth.reads(ref, n, long_len, synth.HIFI_ERR, 0, rng=g)
        reqs.append((reads, offs))
    return reqs


def test_serving_alone_equals_mix(env):
    god, ref, idx = env
    reqs = make_requests(ref, 40, 7)
    alone = [god.god_seed(idx, r, o) for r, o in reqs]
    srv = god.GodServer(idx, slots=4, max_batch_bases=400_000)
    ids = [srv.submit(r, o) for r, o in reqs]
    got = [srv.wait(i) for i in ids]
    st = srv.stats()
    srv.close()
    for a, b in zip(alone, got):
        assert a.size == b.size and np.array_equal(a, b)
    assert st["submitted"] == st["completed"] == len(reqs)
    assert st["merged_requests"] > 0
    assert st["batches"] < len(reqs)
    # oracle parity on a few requests
    o = oracle.Index(ref, "10", 21, 11, 500)
    for q in (0, 5, 17):
        want, _ = o.seed(reqs[q][0], reqs[q][1], 32)
        assert np.array_equal(got[q], want)


def test_serving_overlaps_batches(env):
    god, ref, idx = env
    reqs = make_requests(ref, 24, 8)
    srv = god.GodServer(idx, slots=4, max_batch_bases=100_000)
    ids = [srv.submit(r, o) for r, o in reqs]
    res = [srv.wait(i, with_latency=True) for i in ids]
    st = srv.stats()
    srv.close()
    assert st["max_inflight_batches"] >= 2
    assert all(lat >= 0 for _, lat in res)
    alone = [god.god_seed(idx, r, o) for r, o in reqs]
    for a, (b, _) in zip(alone, res):
        assert np.array_equal(a, b)


def test_serving_admission_refuses_oversized_request(env):
    god, ref, idx = env
    small = make_requests(ref, 6, 9)
    big_reads, big_offs, _ = synth.reads(ref, 200_000, synth.SHORT, synth.ILLUMINA_SUB, 0,
                                         rng=np.random.default_rng(3))
    srv = god.GodServer(idx, slots=2, mem_budget=64 << 20)
    ids = [srv.submit(r, o) for r, o in small]
    big = srv.submit(big_reads, big_offs)
    with pytest.raises(god.GodError) as e:
        srv.wait(big)
    assert e.value.rc == -2
    for (r, o), i in zip(small, ids):
        assert np.array_equal(srv.wait(i), god.god_seed(idx, r, o))
    assert srv.stats()["rejected"] == 1
    srv.close()
