"""Seed matching evaluation on the GPU (god_seed_match) against the oracle
(Sec. 2.1.1, Fig. 4): Levenshtein distance and matched / total seeds of All
Seeds, Minimizers, Spaced and Genome-on-Diet seeding must be equal for every
pair (integer results).

* 1000-base pairs with 0-300 substitutions at random positions, at the
  paper's settings: k = 8 (w = 6) with patterns 110, 10, 101001 and 100, and
  k = 13 / 18 / 21 (w = 9 / 12 / 11) with pattern 10 and the spaced patterns
  1110110110111, 111001011001010111, 111101101101011101111.
* Edge cases: indels (different lengths), empty sequences, N and lower-case
  bytes, the 1024-base maximum; a longer sequence is refused.
"""
import numpy as np
import pytest

import oracle
from paper_2211_08157_gb300 import synth

pytestmark = pytest.mark.gpu

SETTINGS = [(8, 6, "110", "110"), (8, 6, "10", "10"), (8, 6, "101001", "101001"), (8, 6, "100", "100"),
            (13, 9, "10", "1110110110111"), (18, 12, "10", "111001011001010111"),
            (21, 11, "10", "111101101101011101111")]


@pytest.fixture(scope="module")
def god():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2211_08157_gb300 as g
    g.load()
    return g


def substituted_pairs(rng, n, length=1000, max_sub=300):
    seqs = []
    for _ in range(n):
        s = synth.ACGT[rng.integers(0, 4, length)]
        t = s.copy()
        j = int(rng.integers(0, max_sub + 1))
        pos = rng.choice(length, j, replace=False)
        t[pos] = synth.ACGT[(np.searchsorted(synth.ACGT, t[pos]) + rng.integers(1, 4, j)) % 4]
        seqs += [s, t]
    off = np.zeros(len(seqs) + 1, np.uint64)
    off[1:] = np.cumsum([x.size for x in seqs])
    return np.concatenate(seqs), off


@pytest.mark.parametrize("k,w,pattern,spaced", SETTINGS)
def test_seed_match_paper_settings(god, k, w, pattern, spaced):
    rng = np.random.default_rng(k * 100 + len(pattern))
    seqs, off = substituted_pairs(rng, 600)
    want = oracle.seed_match(seqs, off, pattern, spaced, k, w)
    got = god.god_seed_match(seqs, off, pattern, spaced, k, w)
    for x, y in zip(got, want):
        assert np.array_equal(x, y)


def test_seed_match_edge_cases(god):
    rng = np.random.default_rng(9)
    seqs = []
    for _ in range(200):
        la, lb = int(rng.integers(0, 1025)), int(rng.integers(0, 1025))
        alpha = np.frombuffer(b"ACGTACGTACGTACGTNacgtX", np.uint8)
        s = alpha[rng.integers(0, alpha.size, la)]
        t = s[:lb].copy() if lb <= la else np.concatenate([s, alpha[rng.integers(0, alpha.size, lb - la)]])
        if t.size:
            pos = rng.choice(t.size, min(t.size, int(rng.integers(0, 40))), replace=False)
            t[pos] = alpha[rng.integers(0, alpha.size, pos.size)]
        seqs += [s, t]
    seqs += [synth.ACGT[rng.integers(0, 4, 1024)]] * 2 + [np.zeros(0, np.uint8), np.zeros(0, np.uint8)]
    off = np.zeros(len(seqs) + 1, np.uint64)
    off[1:] = np.cumsum([x.size for x in seqs])
    buf = np.concatenate(seqs)
    for k, w, pattern, spaced in ((8, 6, "110", "110"), (21, 11, "10", "111101101101011101111")):
        want = oracle.seed_match(buf, off, pattern, spaced, k, w)
        got = god.god_seed_match(buf, off, pattern, spaced, k, w)
        for x, y in zip(got, want):
            assert np.array_equal(x, y)
    long = np.concatenate([synth.ACGT[rng.integers(0, 4, 1025)], synth.ACGT[rng.integers(0, 4, 10)]])
    with pytest.raises(god.GodError):
        god.god_seed_match(long, np.array([0, 1025, 1035], np.uint64), "10", "10", 8, 6)
