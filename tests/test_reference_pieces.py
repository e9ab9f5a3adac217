"""The index build sketches a long reference as overlapping pieces, each
emitting only the minimizers of the k-mers it owns. This checks, with the
oracle as the minimizer function, the identity that decomposition rests on:
a piece that owns the k-mers [i S, (i + 1) S) of the patterned sequence and
spans [a_i, b_i) with a_0 = 0, a_i = i S - cw (cw = w - 1 rounded up to a
multiple of the pattern weight x, so the piece starts at pattern phase 0),
b_i = min(m, (i + 1) S + w + k - 2) holds every window containing an owned
k-mer, so the owned minimizers of all pieces, in piece order, are exactly the
whole sequence's (windows past a piece's ends contain no owned k-mer; N runs
break windows the same way inside a piece as in the whole sequence)."""
import numpy as np
import pytest

import oracle
from paper_2211_08157_gb300 import synth


def pieces(m, k, w, x, S):
    cw = -(-(w - 1) // x) * x
    nk = m - k + 1
    out = []
    for i in range(-(-nk // S)):
        lo, hi = i * S, min(nk, (i + 1) * S)
        a = i * S - cw if i else 0
        b = min(m, (i + 1) * S + w + k - 2)
        out.append((a, b, lo, hi))
    return out


@pytest.mark.parametrize("pattern,k,w,S", [("10", 21, 11, 216), ("110", 19, 19, 284), ("10", 15, 10, 100),
                                           ("1", 9, 5, 7), ("1110", 13, 7, 33)])
def test_owned_piece_minimizers_equal_whole_sequence(pattern, k, w, S):
    rng = np.random.default_rng(91)
    seq = synth.ACGT[rng.integers(0, 4, 60_000)]
    seq[rng.integers(0, seq.size, 40)] = ord("N")          # N runs break windows
    seq[20_000:20_300] = seq[30_000:30_300]                 # a repeat: equal keys inside windows
    p, x = len(pattern), pattern.count("1")
    off = [i for i, c in enumerate(pattern) if c == "1"]
    S = S // x * x
    keys, pos, z, j = oracle.minimizers(seq, pattern, 0, k, w)
    m = oracle.sparsify(seq, pattern)[0].size
    got_k, got_p, got_z = [], [], []
    for a, b, lo, hi in pieces(m, k, w, x, S):
        start = p * (a // x)                                 # first byte of patterned position a
        end = p * ((b - 1) // x) + off[(b - 1) % x] + 1      # one past the byte of position b - 1
        pk, pp, pz, pj = oracle.minimizers(seq[start:end], pattern, 0, k, w)
        keep = (pj >= lo - a) & (pj < hi - a)
        got_k.append(pk[keep])
        got_p.append(pp[keep] + start)
        got_z.append(pz[keep])
    assert np.array_equal(np.concatenate(got_k), keys)
    assert np.array_equal(np.concatenate(got_p), pos)
    assert np.array_equal(np.concatenate(got_z), z)
