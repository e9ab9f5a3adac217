"""Seeding through the one-thread-per-segment sketch kernel against the oracle.

Batches of at least 1024 short segments (reads at every shift, or the capped
pattern-alignment prefixes of long reads) with w in {10, 11, 19} run the
per-segment kernel instead of the tile kernel. Anchors and alignment indices
must equal the oracle's exactly for every key width and hash form (k from 12
to 28: 32-bit keys, the 32-bit, narrow and full 64-bit hash), odd and even k
(palindromes), patterns of weight 1-3, reads of 0-400 bases with N, lower
case and other bytes, reads shorter than k, and capped prefixes with an N
(which send their read to the full-length fallback).
"""
import numpy as np
import pytest

import oracle
from paper_2211_08157_gb300 import synth

pytestmark = pytest.mark.gpu

CASES = [(21, 11, "10"), (19, 19, "110"), (15, 10, "10"), (16, 10, "1"), (28, 19, "101"), (12, 11, "1110"),
         (24, 10, "10"), (14, 19, "11"), (20, 11, "100")]


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2211_08157_gb300 as god
    god.load()
    ref = synth.reference(400_000, 81, synth.RepeatModel(20, 300, 2000, False, 0.0, 0.02, 0.1))
    rng = np.random.default_rng(82)
    reads, offs, _ = synth.reads(ref, 3000, synth.LengthModel("lognormal", mu=4.8, sigma=0.6, lo=0, hi=400),
                                 synth.ILLUMINA_INDEL, 0, rng=rng)
    reads = reads.copy()
    odd = rng.choice(reads.size, reads.size // 300, replace=False)
    reads[odd] = np.frombuffer(b"NNNNacgtX-\x00\xff", np.uint8)[rng.integers(0, 12, odd.size)]
    # empty reads, reads shorter than k, exactly k, one more
    extra = [ref[:0], ref[100:103], ref[200:220], ref[300:321], ref[400:422], ref[500:530]]
    reads = np.concatenate([reads] + extra)
    offs = np.concatenate([offs, offs[-1] + np.cumsum([e.size for e in extra]).astype(np.uint64)])
    return god, ref, reads, offs


@pytest.mark.parametrize("k,w,pattern", CASES)
def test_segment_kernel_seeding_matches_oracle(env, k, w, pattern):
    god, ref, reads, offs = env
    idx = god.god_build_index(ref, pattern, k, w, 500)
    n = offs.size - 1
    out = np.zeros((max(1, int(offs[-1]) // 2), 4), np.uint32)
    shifts = np.zeros(n, np.uint32)
    m = god.god_seed_into(idx, reads, offs, out, shifts_out=shifts)
    want, wshift = oracle.Index(ref, pattern, k, w, 500).seed(reads, offs, 32, threads=8)
    assert np.array_equal(shifts, wshift)
    assert m == want.size and np.array_equal(out[:m].reshape(-1), want.view(np.uint32))
    idx.close()


def test_segment_kernel_capped_prefixes(env):
    """Long reads: the pattern-alignment pass sketches capped prefixes with the
    per-segment kernel; reads with an N in the prefix take the fallback."""
    god, ref, _, _ = env
    rng = np.random.default_rng(83)
    reads, offs, _ = synth.reads(ref, 1500, synth.LengthModel("lognormal", mu=7.5, sigma=0.5, lo=500, hi=5000),
                                 synth.HIFI_ERR, 0, rng=rng)
    reads = reads.copy()
    for r in rng.choice(1500, 100, replace=False):
        reads[int(offs[r]) + int(rng.integers(0, 200))] = ord("N")
    for k, w, pattern in ((19, 19, "110"), (15, 10, "10")):
        idx = god.god_build_index(ref, pattern, k, w, 500)
        n = offs.size - 1
        out = np.zeros((int(offs[-1]), 4), np.uint32)
        shifts = np.zeros(n, np.uint32)
        m = god.god_seed_into(idx, reads, offs, out, shifts_out=shifts)
        want, wshift = oracle.Index(ref, pattern, k, w, 500).seed(reads, offs, 32, threads=8)
        assert np.array_equal(shifts, wshift)
        assert m == want.size and np.array_equal(out[:m].reshape(-1), want.view(np.uint32))
        idx.close()
