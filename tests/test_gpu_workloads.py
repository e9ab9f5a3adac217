"""Long-read and serving workloads at their stated sizes, against the oracle.

HiFi-like: the 100 Mbp reference (5 % repeats at 2 % divergence), all 200,000
reads with lognormal lengths (mean 15 kb, sd 4 kb, 2-30 kb) and 0.1 % errors
(sub:ins:del 1:2:2), pattern 110, k = 19, w = 19, max_occ = 500, in one
batched device call. Every read's anchors and alignment index must equal the
oracle's (all 200,000 reads); hash and learned lookups must give identical
lists.

ONT-like at human scale: the 3.1 Gbp reference (45 % of bases from repeat
families of 300 bp-6 kb at 5-15 % divergence), pattern 10, k = 15, w = 10,
max_occ = 1000. The whole filtered index (~0.28 G minimizers) must equal the
oracle's; all 100,000 reads (lognormal, mean 10 kb, 0.5-100 kb, 8 % errors
1:1:1) are seeded in one device call with the hash and with the learned index
(identical lists) and a seeded 10 % sample (10,000 reads) is compared exactly
with the oracle. Location voting runs on every read of both long-read batches
and must equal the oracle's (all HiFi-like reads, the ONT-like sample).

Serving at human scale: the learned index of the same 3.1 Gbp reference stays
resident in a continuous-batching server; requests of the serving mix (short
batches of 1k-50k reads, HiFi-like and ONT-like batches of 10-2,000 reads) are
submitted together. Every request's anchors must equal those of the same reads
seeded alone, and a sample of requests (one of each kind and more) must equal
the oracle's.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2211_08157_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

THREADS = os.cpu_count() or 8


@pytest.fixture(scope="module")
def god():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2211_08157_gb300 as g
    g.load()
    return g


@pytest.fixture(scope="module")
def human(god):
    """The 3.1 Gbp reference and the oracle's index of it (built once)."""
    wl = synth.WORKLOADS["ont_3100mbp_100k"]
    ref = wl.make_reference()
    o = oracle.Index(ref, wl.pattern, wl.k, wl.w, wl.max_occ)
    yield wl, ref, o
    o.close()


def device_view(torch, ptr, m):
    class V:
        __cuda_array_interface__ = {"shape": (m, 4), "typestr": "<i4", "data": (ptr, False), "version": 2}
    return torch.as_tensor(V(), device="cuda")


def seed_on_device(god, torch, idx, d_reads, d_offs, n, via):
    shifts = torch.zeros(n, dtype=torch.int32, device="cuda")
    ptr, m = god.god_seed_device(idx, d_reads, d_offs, via=via, shifts_out=shifts)
    return ptr, m, shifts.cpu().numpy().view(np.uint32)


def sample_rows(torch, A, sample):
    """Rows of the device anchor list whose read_id is in `sample` (ascending),
    with read ids renumbered 0..len(sample)-1."""
    rid = A[:, 0].contiguous()
    s = torch.from_numpy(sample.astype(np.int32)).cuda()
    lo = torch.searchsorted(rid, s, side="left")
    hi = torch.searchsorted(rid, s, side="right")
    keep = torch.zeros(A.shape[0] + 1, dtype=torch.int32, device="cuda")
    keep.index_add_(0, lo, torch.ones_like(lo, dtype=torch.int32))
    keep.index_add_(0, hi, -torch.ones_like(hi, dtype=torch.int32))
    mask = torch.cumsum(keep, 0)[:-1] > 0
    got = A[mask].cpu().numpy().view(np.uint32).copy()
    got[:, 0] = np.repeat(np.arange(sample.size, dtype=np.uint32), (hi - lo).cpu().numpy())
    return got


def subset(reads, offs, sample):
    lens = (offs[sample + 1] - offs[sample]).astype(np.uint64)
    so = np.zeros(sample.size + 1, np.uint64)
    so[1:] = np.cumsum(lens)
    return np.concatenate([reads[int(offs[i]):int(offs[i + 1])] for i in sample]), so


def test_hifi_workload_full(god):
    import torch
    wl = synth.WORKLOADS["hifi_100mbp_200k"]
    ref = wl.make_reference()
    reads, offs, _ = wl.make_reads(ref)
    n = offs.size - 1
    assert n == 200_000
    d_ref = torch.from_numpy(ref).cuda()
    d_reads = torch.from_numpy(reads).cuda()
    d_offs = torch.from_numpy(offs.view(np.int64)).cuda()
    res = {}
    for via, kind in ((0, god.GOD_INDEX_HASH), (1, god.GOD_INDEX_LEARNED)):
        idx = god.god_build_index(d_ref, wl.pattern, wl.k, wl.w, wl.max_occ,
                                  params=god.god_params_init(index_kind=kind, pa_t=wl.t))
        ptr, m, shifts = seed_on_device(god, torch, idx, d_reads, d_offs, n, via)
        A = device_view(torch, ptr, m)
        res[via] = (A.cpu().numpy().view(np.uint32).copy(), shifts)
        god.god_free(ptr)
        idx.close()
    a0, s0 = res[0]
    a1, s1 = res[1]
    assert np.array_equal(a0, a1) and np.array_equal(s0, s1)
    assert a0.shape[0] > 10_000_000
    want, wshift = oracle.Index(ref, wl.pattern, wl.k, wl.w, wl.max_occ).seed(reads, offs, wl.t, threads=THREADS)
    assert np.array_equal(s0, wshift)
    assert want.size == a0.shape[0]
    assert np.array_equal(a0.reshape(-1), want.view(np.uint32))
    # location voting of every read (Sec. 3.4 step 5, long reads)
    gv, gc = god.god_vote(a0, offs, 100, 3, 8)
    wv, wc = oracle.vote(want, offs, 100, 3, 8)
    assert np.array_equal(gc, wc) and np.array_equal(gv, wv)


def test_ont_human_scale_index_and_sample(god, human):
    import torch
    wl, ref, o = human
    d_ref = torch.from_numpy(ref).cuda()
    idx = god.god_build_index(d_ref, wl.pattern, wl.k, wl.w, wl.max_occ,
                              params=god.god_params_init(index_kind=god.GOD_INDEX_LEARNED, pa_t=wl.t))
    del d_ref
    info = idx.info
    assert info["n_minimizers"] == o.sizes()[0] and info["n_minimizers"] > 250_000_000
    gk, gs, ge = god.god_index_export(idx)
    ok, os_, oe = o.dump()
    assert np.array_equal(gk, ok)
    assert np.array_equal(gs, os_)
    assert np.array_equal(ge, oe)
    del gk, gs, ge, ok, os_, oe
    reads, offs, _ = wl.make_reads(ref)
    n = offs.size - 1
    assert n == 100_000
    d_reads = torch.from_numpy(reads).cuda()
    d_offs = torch.from_numpy(offs.view(np.int64)).cuda()
    ptr0, m0, shifts0 = seed_on_device(god, torch, idx, d_reads, d_offs, n, 0)
    ptr1, m1, shifts1 = seed_on_device(god, torch, idx, d_reads, d_offs, n, 1)
    A0 = device_view(torch, ptr0, m0)
    A1 = device_view(torch, ptr1, m1)
    assert m0 == m1 and torch.equal(A0, A1) and np.array_equal(shifts0, shifts1)
    god.god_free(ptr1)
    rng = np.random.default_rng(404)
    sample = np.sort(rng.choice(n, n // 10, replace=False))
    sub, so = subset(reads, offs, sample)
    want, wshift = o.seed(sub, so, wl.t, threads=THREADS)
    assert np.array_equal(shifts0[sample], wshift)
    got = sample_rows(torch, A0, sample)
    assert got.shape[0] == want.size
    assert np.array_equal(got.reshape(-1), want.view(np.uint32))
    # location voting of all 100,000 reads on the device; the sample's records
    # must equal the oracle's voting over the oracle's anchors
    D, V, max_out = 100, 3, 8
    d_out = torch.zeros((n * max_out, 10), dtype=torch.int32, device="cuda")
    d_cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
    god.god_vote((ptr0, m0), d_offs, D, V, max_out, out=d_out, counts=d_cnt)
    god.god_free(ptr0)
    cnt = d_cnt.cpu().numpy().view(np.uint32)
    rec = d_out.cpu().numpy().view(oracle.VOTE_DTYPE).reshape(n, max_out)
    wv, wc = oracle.vote(want, so, D, V, max_out)
    assert np.array_equal(cnt[sample], wc)
    keep = np.arange(max_out)[None, :] < wc[:, None]
    gv = rec[sample][keep].copy()
    gv["read_id"] = np.repeat(np.arange(sample.size, dtype=np.uint32), wc)
    assert np.array_equal(gv, wv)
    idx.close()


def test_serving_human_scale_learned_index(god, human):
    import torch
    wl, ref, o = human
    idx = god.god_build_index(torch.from_numpy(ref).cuda(), wl.pattern, wl.k, wl.w, wl.max_occ,
                              params=god.god_params_init(index_kind=god.GOD_INDEX_LEARNED, pa_t=wl.t))
    pool = synth.serving_requests(ref, per_kind=4, long_max=2000, seed=21)
    rng = np.random.default_rng(22)
    reqs = []
    for kind in ("short", "hifi", "ont"):
        reqs += [(kind, r, off) for r, off in pool[kind]]
    order = rng.permutation(len(reqs))
    reqs = [reqs[i] for i in order]
    srv = god.GodServer(idx, slots=4)
    ids = [srv.submit(r, off) for _, r, off in reqs]
    got = [srv.wait(i) for i in ids]
    st = srv.stats()
    srv.close()
    assert st["submitted"] == st["completed"] == len(reqs)
    for (_, r, off), g in zip(reqs, got):
        alone = god.god_seed(idx, r, off)
        assert alone.size == g.size and np.array_equal(alone, g)
    # oracle parity: the first request of each kind and two more
    picked, seen = [], set()
    for q, (kind, _, _) in enumerate(reqs):
        if kind not in seen:
            seen.add(kind)
            picked.append(q)
    picked += [q for q in range(len(reqs)) if q not in picked][:2]
    for q in picked:
        _, r, off = reqs[q]
        want, _ = o.seed(r, off, wl.t, threads=THREADS)
        assert np.array_equal(got[q], want), f"request {q} ({reqs[q][0]}) differs from the oracle"
    idx.close()
