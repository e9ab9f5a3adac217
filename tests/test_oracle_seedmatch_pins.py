"""Pins of the oracle's seed matching evaluation (Sec. 2.1.1, Fig. 4).

* Levenshtein distance: a memoised recursion over the textbook definition on
  random short byte strings (different lengths, bytes outside ACGT), the
  kitten / sitting example (3), empty strings, and d <= number of
  substitutions for substitution-only copies.
* Identical pairs match every seed of every algorithm.
* Pattern 1 turns Genome-on-Diet seeds and spaced seeds into all k-mers.
* One substitution at position x of a 1000-base random sequence (no repeated
  k-mers): All Seeds lose exactly the k k-mers covering x; Genome-on-Diet
  seeds under pattern 10 lose k when x is kept (even) and none when it is
  dropped (odd); spaced seeds with the mask 10 repeated to k = 13 lose the 7
  starts that read x.
"""
import functools

import numpy as np

import oracle
from paper_2211_08157_gb300 import synth


def pairs(seqs):
    buf = np.concatenate([np.frombuffer(bytes(s), np.uint8) if isinstance(s, (bytes, bytearray)) else s
                          for s in seqs]) if seqs else np.zeros(0, np.uint8)
    off = np.zeros(len(seqs) + 1, np.uint64)
    off[1:] = np.cumsum([len(s) for s in seqs])
    return buf, off


def lev_rec(a, b):
    @functools.lru_cache(maxsize=None)
    def d(i, j):
        if i == 0:
            return j
        if j == 0:
            return i
        return min(d(i - 1, j) + 1, d(i, j - 1) + 1, d(i - 1, j - 1) + (a[i - 1] != b[j - 1]))
    return d(len(a), len(b))


def test_levenshtein_against_recursion():
    rng = np.random.default_rng(3)
    seqs = [b"kitten", b"sitting", b"", b"ACGT", b"ACGT", b""]
    for _ in range(150):
        la, lb = int(rng.integers(0, 14)), int(rng.integers(0, 14))
        alpha = np.frombuffer(b"ACGTN", np.uint8)
        seqs.append(bytes(alpha[rng.integers(0, 5, la)]))
        seqs.append(bytes(alpha[rng.integers(0, 5, lb)]))
    buf, off = pairs(seqs)
    ed, _, _ = oracle.seed_match(buf, off, "10", "110", 3, 2)
    assert ed[0] == 3 and ed[1] == 4 and ed[2] == 4
    for i in range(len(seqs) // 2):
        assert ed[i] == lev_rec(seqs[2 * i], seqs[2 * i + 1])


def test_substitutions_bound_distance_and_identity_matches_all():
    rng = np.random.default_rng(4)
    seqs = []
    for _ in range(30):
        s = synth.ACGT[rng.integers(0, 4, 1000)]
        t = s.copy()
        j = int(rng.integers(0, 60))
        pos = rng.choice(1000, j, replace=False)
        t[pos] = synth.ACGT[(np.searchsorted(synth.ACGT, t[pos]) + rng.integers(1, 4, j)) % 4]
        seqs += [s, t, s, s.copy()]
    buf, off = pairs(seqs)
    ed, mt, tt = oracle.seed_match(buf, off, "10", "1110110110111", 13, 9)
    for i in range(0, len(seqs) // 2, 2):
        assert ed[i] <= np.count_nonzero(seqs[2 * i] != seqs[2 * i + 1])
        assert ed[i + 1] == 0 and np.array_equal(mt[i + 1], tt[i + 1]) and (tt[i + 1] > 0).all()


def test_pattern_one_reduces_to_all_seeds():
    rng = np.random.default_rng(5)
    seqs = [synth.ACGT[rng.integers(0, 4, 500)] for _ in range(20)]
    buf, off = pairs(seqs)
    _, mt, tt = oracle.seed_match(buf, off, "1", "1", 8, 6)
    assert np.array_equal(mt[:, 3], mt[:, 0]) and np.array_equal(tt[:, 3], tt[:, 0])
    assert np.array_equal(mt[:, 2], mt[:, 0]) and np.array_equal(tt[:, 2], tt[:, 0])


def test_single_substitution_closed_forms():
    rng = np.random.default_rng(6)
    k = 13
    s = synth.ACGT[rng.integers(0, 4, 1000)]
    seqs = []
    xs = [400, 401, 500, 777]
    for x in xs:
        t = s.copy()
        t[x] = synth.ACGT[(np.searchsorted(synth.ACGT, t[x]) + 1) % 4]
        seqs += [s, t]
    buf, off = pairs(seqs)
    ed, mt, tt = oracle.seed_match(buf, off, "10", "10", k, 9)
    for i, x in enumerate(xs):
        assert ed[i] == 1
        assert tt[i, 0] - mt[i, 0] == k                       # All Seeds
        assert tt[i, 3] - mt[i, 3] == (k if x % 2 == 0 else 0)  # Genome-on-Diet, pattern 10
        assert tt[i, 2] - mt[i, 2] == 7                       # mask 1010101010101: starts x-12, x-10, ..., x
        assert mt[i, 1] <= tt[i, 1]
