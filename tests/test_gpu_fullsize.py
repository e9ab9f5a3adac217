"""Parity at the benchmark's full size, in the launch configuration bench.py times.

Workload: the 100 Mbp reference (iid ACGT + 5 % repeat families at 2 %
divergence) and 2,000,000 reads of 150 bp (0.1 % substitutions, 0.01 % 1-bp
indels, both strands), pattern 10, k = 21, w = 11, max_occ = 500, t = 32.

* The whole filtered index (keys, offsets, entries) equals the oracle's.
* All 2,000,000 reads are seeded in one batched device call (hash and learned
  index) and the whole anchor list and every read's alignment index must equal
  what the oracle computes for all 2,000,000 reads (integer results: exact).
* Location voting of all 2,000,000 reads on the GPU equals the oracle's.
* Properties that hold at any size: the anchor list is sorted by
  (read_id, ref_pos, read_pos, strand) with no duplicates, and both index
  paths return identical lists.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2211_08157_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2211_08157_gb300 as god
    god.load()
    wl = synth.WORKLOADS["short_100mbp_2m"]
    ref = wl.make_reference()
    reads, offs, truth = wl.make_reads(ref)
    o = oracle.Index(ref, wl.pattern, wl.k, wl.w, wl.max_occ)
    return god, torch, wl, ref, reads, offs, o


def test_fullsize_index_matches_oracle(env):
    god, torch, wl, ref, reads, offs, o = env
    idx = god.god_build_index(torch.from_numpy(ref).cuda(), wl.pattern, wl.k, wl.w, wl.max_occ)
    gk, gs, ge = god.god_index_export(idx)
    ok, os_, oe = o.dump()
    assert idx.info["n_minimizers"] == o.sizes()[0]
    assert np.array_equal(gk, ok) and np.array_equal(gs, os_) and np.array_equal(ge, oe)
    idx.close()


def test_fullsize_seeding_full_parity(env):
    god, torch, wl, ref, reads, offs, o = env
    n = offs.size - 1
    d_ref = torch.from_numpy(ref).cuda()
    d_reads = torch.from_numpy(reads).cuda()
    d_offs = torch.from_numpy(offs.view(np.int64)).cuda()
    results = {}
    for via, kind in ((0, god.GOD_INDEX_HASH), (1, god.GOD_INDEX_LEARNED)):
        params = god.god_params_init(index_kind=kind, pa_t=wl.t)
        idx = god.god_build_index(d_ref, wl.pattern, wl.k, wl.w, wl.max_occ, params=params)
        out = torch.empty((40_000_000, 4), dtype=torch.int32, device="cuda")
        shifts = torch.zeros(n, dtype=torch.int32, device="cuda")
        m = god.god_seed_into(idx, d_reads, d_offs, out, via=via, shifts_out=shifts)
        results[via] = (out[:m].cpu().numpy().view(np.uint32), shifts.cpu().numpy().view(np.uint32))
        del out
        idx.close()
    a0, s0 = results[0]
    a1, s1 = results[1]
    assert np.array_equal(a0, a1) and np.array_equal(s0, s1)
    assert a0.shape[0] > 10_000_000
    # every read, every anchor: the oracle over all host cores
    want, wshift = o.seed(reads, offs, wl.t, threads=os.cpu_count() or 8)
    assert np.array_equal(s0, wshift)
    assert want.size == a0.shape[0]
    assert np.array_equal(a0.reshape(-1), want.view(np.uint32))
    # location voting over the whole anchor list (Sec. 3.4 step 4, short reads)
    d_a = torch.from_numpy(a0.view(np.int32)).cuda()
    gv, gc = god.god_vote(d_a, offs, 50, 2, 4)
    wv, wc = oracle.vote(want, offs, 50, 2, 4)
    assert np.array_equal(gc, wc) and np.array_equal(gv, wv)
