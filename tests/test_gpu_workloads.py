"""Long-read workloads against the oracle.

HiFi-like: the 100 Mbp reference (5 % repeats at 2 % divergence), 20,000
reads with lognormal lengths (mean 15 kb, sd 4 kb, 2-30 kb) and 0.1 % errors
(sub:ins:del 1:2:2), pattern 110, k = 19, w = 19, max_occ = 500: the
pattern-alignment prefix is capped and every read takes the second seeding
pass. 200 sampled reads are compared exactly with the oracle; hash and learned
lookups must give identical lists.

ONT-like at human scale: the 3.1 Gbp reference (45 % of bases from repeat
families of 300 bp-6 kb at 5-15 % divergence), pattern 10, k = 15, w = 10,
max_occ = 1000. The whole filtered index (~0.28 G minimizers) must equal the
oracle's; 4,000 reads (lognormal, mean 10 kb, 0.5-100 kb, 8 % errors 1:1:1)
are seeded on the GPU and a seeded 10 % sample is compared exactly with the
oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2211_08157_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def god():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2211_08157_gb300 as g
    g.load()
    return g


def device_view(torch, ptr, m):
    class V:
        __cuda_array_interface__ = {"shape": (m, 4), "typestr": "<i4", "data": (ptr, False), "version": 2}
    return torch.as_tensor(V(), device="cuda")


def seed_on_device(god, torch, idx, reads, offs, via):
    d_reads = torch.from_numpy(reads).cuda()
    d_offs = torch.from_numpy(offs.view(np.int64)).cuda()
    n = offs.size - 1
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
    parts = [A[int(l):int(h)] for l, h in zip(lo.tolist(), hi.tolist())]
    got = torch.cat(parts).cpu().numpy().view(np.uint32).copy() if parts else np.zeros((0, 4), np.uint32)
    got[:, 0] = np.repeat(np.arange(sample.size, dtype=np.uint32), (hi - lo).cpu().numpy())
    return got


def subset(reads, offs, sample):
    lens = (offs[sample + 1] - offs[sample]).astype(np.uint64)
    so = np.zeros(sample.size + 1, np.uint64)
    so[1:] = np.cumsum(lens)
    return np.concatenate([reads[int(offs[i]):int(offs[i + 1])] for i in sample]), so


def test_hifi_workload(god):
    import torch
    wl = synth.WORKLOADS["hifi_100mbp_200k"]
    ref = wl.make_reference()
    reads, offs, _ = wl.make_reads(ref, n=20_000)
    d_ref = torch.from_numpy(ref).cuda()
    res = {}
    for via, kind in ((0, god.GOD_INDEX_HASH), (1, god.GOD_INDEX_LEARNED)):
        idx = god.god_build_index(d_ref, wl.pattern, wl.k, wl.w, wl.max_occ,
                                  params=god.god_params_init(index_kind=kind, pa_t=wl.t))
        ptr, m, shifts = seed_on_device(god, torch, idx, reads, offs, via)
        A = device_view(torch, ptr, m)
        res[via] = (A.clone(), shifts)
        god.god_free(ptr)
        idx.close()
    A0, s0 = res[0]
    A1, s1 = res[1]
    assert torch.equal(A0, A1) and np.array_equal(s0, s1)
    assert A0.shape[0] > 1_000_000
    rng = np.random.default_rng(303)
    sample = np.sort(rng.choice(offs.size - 1, 200, replace=False))
    sub, so = subset(reads, offs, sample)
    want, wshift = oracle.Index(ref, wl.pattern, wl.k, wl.w, wl.max_occ).seed(sub, so, wl.t, threads=8)
    assert np.array_equal(s0[sample], wshift)
    got = sample_rows(torch, A0, sample)
    assert np.array_equal(got.reshape(-1), want.view(np.uint32))


def test_ont_human_scale_index_and_sample(god):
    import torch
    wl = synth.WORKLOADS["ont_3100mbp_100k"]
    ref = wl.make_reference()
    d_ref = torch.from_numpy(ref).cuda()
    idx = god.god_build_index(d_ref, wl.pattern, wl.k, wl.w, wl.max_occ,
                              params=god.god_params_init(pa_t=wl.t))
    info = idx.info
    o = oracle.Index(ref, wl.pattern, wl.k, wl.w, wl.max_occ)
    assert info["n_minimizers"] == o.sizes()[0] and info["n_minimizers"] > 250_000_000
    gk, gs, ge = god.god_index_export(idx)
    ok, os_, oe = o.dump()
    assert np.array_equal(gk, ok)
    assert np.array_equal(gs, os_)
    assert np.array_equal(ge, oe)
    del gk, gs, ge, ok, os_, oe
    reads, offs, _ = wl.make_reads(ref, n=4000)
    ptr, m, shifts = seed_on_device(god, torch, idx, reads, offs, 0)
    A = device_view(torch, ptr, m)
    rng = np.random.default_rng(404)
    sample = np.sort(rng.choice(offs.size - 1, 400, replace=False))
    sub, so = subset(reads, offs, sample)
    want, wshift = o.seed(sub, so, wl.t, threads=8)
    assert np.array_equal(shifts[sample], wshift)
    got = sample_rows(torch, A, sample)
    god.god_free(ptr)
    assert np.array_equal(got.reshape(-1), want.view(np.uint32))
    idx.close()
