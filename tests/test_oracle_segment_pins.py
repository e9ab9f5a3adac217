"""Pins of the oracle's segmented seeding (Sec. 2.2.2: ultra-long reads are
split into segments of at most 30,000 bases; Sec. 3.2: each segment gets its
own pattern alignment).

* A segment length at least as long as every read changes nothing.
* One alignment index per segment: ceil(len / seg_len) of them for a longer
  read, in read then segment order.
* Bookkeeping: a segmented read's anchors equal those of its pieces seeded as
  separate reads, with the piece's start added to read_pos and the read's id.
* Phase recovery: an error-free read with one deleted base at position p loses
  the diagonal after p when aligned once (pattern 10: the deletion flips the
  phase), while with segments cut at p the second segment re-aligns to the
  other shift and its minimizers land on the shifted diagonal start + 1.
"""
import numpy as np

import oracle
from paper_2211_08157_gb300 import synth


def test_long_segment_length_changes_nothing():
    ref = synth.reference(500_000, 41)
    reads, offs, _ = synth.reads(ref, 60, synth.LengthModel("lognormal", mu=8.0, sigma=0.7, lo=100, hi=9000),
                                 synth.HIFI_ERR, 0, rng=np.random.default_rng(1))
    idx = oracle.Index(ref, "110", 19, 19, 500)
    a0, s0 = idx.seed(reads, offs, 32)
    a1, s1 = idx.seed(reads, offs, 32, seg_len=9000)
    assert np.array_equal(a0, a1) and np.array_equal(s0, s1) and s1.size == offs.size - 1


def test_segments_equal_pieces_seeded_alone():
    ref = synth.reference(800_000, 42, synth.RepeatModel(10, 500, 2000, False, 0.0, 0.02, 0.1))
    reads, offs, _ = synth.reads(ref, 40, synth.LengthModel("lognormal", mu=8.7, sigma=0.6, lo=300, hi=20_000),
                                 synth.ONT_ERR, 0, rng=np.random.default_rng(2))
    S = 2500
    idx = oracle.Index(ref, "10", 15, 10, 1000)
    got, shifts = idx.seed(reads, offs, 32, seg_len=S)
    lens = np.diff(offs).astype(np.int64)
    nseg = np.maximum(1, -(-lens // S))
    assert shifts.size == nseg.sum()
    pieces, owner, start = [], [], []
    for r in range(offs.size - 1):
        for j in range(int(nseg[r])):
            b = int(offs[r]) + j * S
            e = min(b + S, int(offs[r + 1])) if nseg[r] > 1 else int(offs[r + 1])
            pieces.append(reads[b:e])
            owner.append(r)
            start.append(j * S)
    po = np.zeros(len(pieces) + 1, np.uint64)
    po[1:] = np.cumsum([p.size for p in pieces])
    alone, ps = idx.seed(np.concatenate(pieces), po, 32)
    assert np.array_equal(ps, shifts)
    want = alone.copy()
    want["read_pos"] += np.array(start, np.uint32)[alone["read_id"]]
    want["read_id"] = np.array(owner, np.uint32)[alone["read_id"]]
    order = np.lexsort((want["strand"], want["read_pos"], want["ref_pos"], want["read_id"]))
    assert np.array_equal(got, want[order])


def test_segment_realigns_after_deletion():
    ref = synth.reference(200_000, 43)
    start, p, L = 50_000, 3000, 6000
    tpl = ref[start:start + L + 1]
    read = np.concatenate([tpl[:p], tpl[p + 1:]])          # base p deleted
    offs = np.array([0, read.size], np.uint64)
    idx = oracle.Index(ref, "10", 21, 11, 500)
    one, s_one = idx.seed(read, offs, 32)
    seg, s_seg = idx.seed(read, offs, 32, seg_len=p)
    assert s_one.size == 1 and s_seg.size == 2 and s_seg[0] != s_seg[1]
    d_one = one["ref_pos"].astype(np.int64) - one["read_pos"]
    d_seg = seg["ref_pos"].astype(np.int64) - seg["read_pos"]
    after_one = (one["read_pos"] >= p) & (d_one == start + 1)
    after_seg = (seg["read_pos"] >= p) & (d_seg == start + 1)
    before_seg = (seg["read_pos"] < p) & (d_seg == start)
    assert after_one.sum() == 0                             # one alignment index: phase lost after p
    assert after_seg.sum() > 200 and before_seg.sum() > 200
