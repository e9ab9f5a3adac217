"""Batched launch machinery: results do not depend on how the work is launched.

* The autotuner (several CTA shapes and tile sizes of the tile kernel timed on
  the batch itself) changes only the launch shape: anchors equal the fixed
  default's and the oracle's, and its choices are recorded.
* The CUDA-graph path (the sketch pass captured per call and applied to a
  cached executable with cudaGraphExecUpdate) gives the same anchors as direct
  launches, across calls whose sizes change between replays.
* Mixed read lengths (150 bp to 30 kb) in one batch give the same anchors as
  each length class seeded on its own.
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
    ref = synth.reference(2_000_000, 61, synth.RepeatModel(20, 500, 3000, False, 0.0, 0.02, 0.05))
    return god, torch, ref


def _seed(god, idx, reads, offs, stream=None):
    out = np.zeros((reads.size // 2 + 100_000, 4), np.uint32)
    m = god.god_seed_into(idx, reads, offs, out, stream=stream)
    return out[:m].copy()


def test_autotuned_launch_same_anchors(env):
    god, torch, ref = env
    reads, offs, _ = synth.reads(ref, 20_000, synth.SHORT, synth.ILLUMINA_INDEL, 61)
    base = god.god_build_index(ref, "10", 21, 11, 500)
    tuned = god.god_build_index(ref, "10", 21, 11, 500, params=god.god_params_init(tune=1))
    a = _seed(god, base, reads, offs)
    b = _seed(god, tuned, reads, offs)
    c = _seed(god, tuned, reads, offs)  # second call: cached choice
    want, _ = oracle.Index(ref, "10", 21, 11, 500).seed(reads, offs, 32)
    assert np.array_equal(a, b) and np.array_equal(b, c)
    assert np.array_equal(a.reshape(-1), want.view(np.uint32))
    ka, _, _ = god.god_index_export(base)
    kb, _, _ = god.god_index_export(tuned)
    assert np.array_equal(ka, kb)
    # short segments (the reads above, the reference's pieces) run the
    # one-thread-per-segment kernel, which has no shape to choose; long reads'
    # full-length segments run the tile kernel with a tuned shape
    lreads, loffs, _ = synth.reads(ref, 300, synth.HIFI, synth.HIFI_ERR, 62)
    la = _seed(god, base, lreads, loffs)
    lb = _seed(god, tuned, lreads, loffs)
    lwant, _ = oracle.Index(ref, "10", 21, 11, 500).seed(lreads, loffs, 32)
    assert np.array_equal(la, lb) and np.array_equal(la.reshape(-1), lwant.view(np.uint32))
    table = god.god_autotune_report()
    assert len(table) >= 1 and all(e["threads"] in (128, 256) and e["chunks"] in (1, 2) for e in table)


def test_graph_replay_matches_direct(env):
    god, torch, ref = env
    idx = god.god_build_index(ref, "10", 21, 11, 500)
    stream = torch.cuda.Stream()
    rng = np.random.default_rng(62)
    batches = [synth.reads(ref, int(n), synth.SHORT, synth.ILLUMINA_SUB, 0, rng=np.random.default_rng(int(n)))[:2]
               for n in rng.integers(100, 5000, 5)]
    god.god_set_graphs(True)
    with_graphs = [_seed(god, idx, r, o, stream=stream) for r, o in batches]
    again = [_seed(god, idx, r, o, stream=stream) for r, o in batches]  # replays with new sizes/pointers
    god.god_set_graphs(False)
    direct = [_seed(god, idx, r, o, stream=stream) for r, o in batches]
    god.god_set_graphs(True)
    for x, y, z in zip(with_graphs, again, direct):
        assert np.array_equal(x, y) and np.array_equal(x, z)


def test_mixed_lengths_in_one_batch(env):
    god, torch, ref = env
    idx = god.god_build_index(ref, "110", 19, 19, 500, params=god.god_params_init(tune=1))
    short = synth.reads(ref, 3000, synth.SHORT, synth.ILLUMINA_SUB, 0, rng=np.random.default_rng(1))[:2]
    long_len = synth.LengthModel("lognormal", mu=9.2, sigma=0.6, lo=2000, hi=30_000)
    long = synth.reads(ref, 150, long_len, synth.HIFI_ERR, 0, rng=np.random.default_rng(2))[:2]
    reads = np.concatenate([short[0], long[0]])
    offs = np.concatenate([short[1], long[1][1:] + short[1][-1]])
    mixed = _seed(god, idx, reads, offs, stream=torch.cuda.Stream())
    a = _seed(god, idx, *short)
    b = _seed(god, idx, *long)
    b[:, 0] += short[1].size - 1
    assert np.array_equal(mixed, np.concatenate([a, b]))
    want, _ = oracle.Index(ref, "110", 19, 19, 500).seed(reads, offs, 32)
    assert np.array_equal(mixed.reshape(-1), want.view(np.uint32))
