"""Pins of the oracle's location voting (Sec. 3.4 steps 1-5, Fig. 8, Sec. 3.6.3).

* Brute force: a multiset formulation with no sorting (repeatedly take the
  smallest remaining location of a strand and every location within D of it)
  gives the same groups as the oracle on random tiny anchor lists.
* Fig. 8 (caption values, tests/golden/fig8_voting.txt): 12 votes at location
  1017 win for a short read; with D = 100 and V = 3 a long read's anchors on
  three diagonals give exactly the stretches [3004 - 7832], [10020 - 15000] and
  [71303 - 72437] with 7, 8 and 3 votes, most votes first, while groups with
  fewer than 3 votes are dropped.
* Rescue (Sec. 3.6.3): when no group reaches V, the single best group is
  reported, flagged; with no anchors nothing is reported.
* Invariants: every anchor votes exactly once; a group spans at most D; group
  starts on a strand are more than D apart; the list is cut at max_out.
* Error-free reads put the winner at the true location: ref start for forward
  reads, ref start - (span - 1) for reverse reads (span = 2k - 1 under
  pattern 10), which pins the strand rebasing of step 1.
"""
import os

import numpy as np

import oracle
from paper_2211_08157_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def anchors_array(rows):
    a = np.array(sorted(rows, key=lambda x: (x[0], x[2], x[1], x[3])), dtype=np.uint32).reshape(-1, 4)
    return a


def brute_groups(rows, length, D):
    """Every group of one read by the multiset definition: (strand, v0, votes, ref_lo, ref_hi, read_lo, read_hi)."""
    out = []
    for strand in (0, 1):
        left = []
        for _, rp, ref, s in rows:
            if s != strand:
                continue
            v = ref - rp if strand == 0 else ref - (length - 1 - rp)
            left.append((v, ref, rp))
        while left:
            v0 = min(x[0] for x in left)
            mem = [x for x in left if x[0] - v0 <= D]
            left = [x for x in left if x[0] - v0 > D]
            out.append((strand, v0, len(mem), min(m[1] for m in mem), max(m[1] for m in mem),
                        min(m[2] for m in mem), max(m[2] for m in mem)))
    return out


def as_tuples(rec):
    return [(int(r["strand"]), int(r["loc"]), int(r["votes"]), int(r["ref_lo"]), int(r["ref_hi"]),
             int(r["read_lo"]), int(r["read_hi"])) for r in rec]


def test_vote_matches_bruteforce_random():
    rng = np.random.default_rng(81)
    for case in range(300):
        n_reads = int(rng.integers(1, 6))
        lens = rng.integers(20, 400, n_reads)
        offs = np.zeros(n_reads + 1, np.uint64)
        offs[1:] = np.cumsum(lens)
        rows = []
        for r in range(n_reads):
            m = int(rng.integers(0, 40))
            for _ in range(m):
                rp = int(rng.integers(0, lens[r]))
                ref = int(rng.integers(0, 3000)) if rng.random() < 0.5 else int(rng.integers(0, 60))
                rows.append((r, rp, ref, int(rng.integers(0, 2))))
        rows = sorted(set(rows))
        a = anchors_array(rows) if rows else np.zeros((0, 4), np.uint32)
        D = int(rng.integers(0, 200))
        V = int(rng.integers(1, 5))
        max_out = int(rng.integers(1, 9))
        rec, counts = oracle.vote(a, offs, D, V, max_out)
        at = 0
        for r in range(n_reads):
            mine = [x for x in rows if x[0] == r]
            groups = brute_groups(mine, int(lens[r]), D)
            assert sum(g[2] for g in groups) == len(mine)
            win = sorted([g for g in groups if g[2] >= V], key=lambda g: (-g[2], g[0], g[1]))[:max_out]
            rescue = 0
            if not win and groups:
                win = [sorted(groups, key=lambda g: (-g[2], g[0], g[1]))[0]]
                rescue = 1
            got = rec[at:at + counts[r]]
            at += counts[r]
            assert as_tuples(got) == win, (case, r)
            assert (got["rescue"] == rescue).all() and (got["read_id"] == r).all()


def golden():
    A, B, B_out = None, None, []
    for line in open(os.path.join(GOLDEN, "fig8_voting.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        if f[0] == "A":
            A = (int(f[1]), int(f[2]))
        elif f[0] == "B":
            B = (int(f[1]), int(f[2]))
        else:
            B_out.append((int(f[1]), int(f[2]), int(f[3])))
    return A, B, B_out


def test_fig8a_short_read_location():
    (loc, votes), _, _ = golden()
    rng = np.random.default_rng(5)
    rows = [(0, rp, loc + rp, 0) for rp in sorted(rng.choice(140, votes, replace=False).tolist())]
    rows += [(0, 3, 52_000, 0), (0, 9, 52_400, 0), (0, 20, 900_000, 1)]      # scattered single votes
    rec, counts = oracle.vote(anchors_array(rows), np.array([0, 150], np.uint64), 20, 3, 4)
    assert counts[0] == 1
    assert int(rec[0]["loc"]) == loc and int(rec[0]["votes"]) == votes and rec[0]["strand"] == 0


def test_fig8b_long_read_stretches():
    _, (D, V), stretches = golden()
    rng = np.random.default_rng(6)
    rows = []
    read_base = 0
    for lo, hi, votes in stretches:
        # `votes` anchors on one diagonal (jitter < D) whose reference positions
        # run from lo to hi
        refs = np.sort(np.concatenate([[lo, hi], rng.integers(lo + 1, hi, votes - 2)]))
        jit = rng.integers(0, D // 2, votes)
        for ref, j in zip(refs.tolist(), jit.tolist()):
            rows.append((0, read_base + (ref - lo) + int(j), int(ref), 0))
        read_base += hi - lo + 500
    rows += [(0, 200, 40_000, 0), (0, 900, 40_900, 0), (0, 50, 200_000, 1)]   # groups of 2 and 1 votes: dropped
    length = read_base + 1000
    rec, counts = oracle.vote(anchors_array(rows), np.array([0, length], np.uint64), D, V, 8)
    want = sorted(stretches, key=lambda s: -s[2])
    assert counts[0] == len(stretches)
    assert [(int(r["ref_lo"]), int(r["ref_hi"]), int(r["votes"])) for r in rec] == want
    assert not rec["rescue"].any()


def test_rescue_and_empty():
    rows = [(0, 10, 1000, 0), (0, 40, 1030, 0), (0, 12, 5000, 1), (2, 5, 70, 0)]
    offs = np.array([0, 100, 200, 300], np.uint64)
    rec, counts = oracle.vote(anchors_array(rows), offs, 50, 3, 4)
    assert list(counts) == [1, 0, 1]
    assert rec[0]["rescue"] == 1 and rec[0]["votes"] == 2 and int(rec[0]["loc"]) == 990
    assert rec[1]["rescue"] == 1 and rec[1]["read_id"] == 2 and rec[1]["votes"] == 1
    # ties: the first group in (strand, location) order is the rescue
    rows = [(0, 0, 100, 0), (0, 0, 9000, 0), (0, 0, 50, 1)]
    rec, counts = oracle.vote(anchors_array(rows), np.array([0, 10], np.uint64), 5, 2, 4)
    assert counts[0] == 1 and int(rec[0]["loc"]) == 100 and rec[0]["strand"] == 0


def test_vote_invariants_on_seeded_reads():
    ref = synth.reference(400_000, 31, synth.RepeatModel(20, 300, 2000, False, 0.0, 0.03, 0.2))
    reads, offs, _ = synth.reads(ref, 300, synth.LengthModel("lognormal", mu=8.0, sigma=0.6, lo=200, hi=8000),
                                 synth.ONT_ERR, 0, rng=np.random.default_rng(3))
    idx = oracle.Index(ref, "10", 15, 10, 1000)
    a, _ = idx.seed(reads, offs, 32)
    D = 60
    rec, counts = oracle.vote(a, offs, D, 1, 1_000_000)
    per_read = np.bincount(a["read_id"], minlength=offs.size - 1)
    got = np.zeros(offs.size - 1, np.int64)
    np.add.at(got, rec["read_id"], rec["votes"])
    assert np.array_equal(got, per_read)                          # every anchor votes once
    for r in range(offs.size - 1):
        g = rec[rec["read_id"] == r]
        for s in (0, 1):
            starts = np.sort(g["loc"][g["strand"] == s])
            assert (np.diff(starts) > D).all()                   # group starts more than D apart
    assert (rec["ref_hi"] >= rec["ref_lo"]).all() and (rec["read_hi"] >= rec["read_lo"]).all()
    cut, c2 = oracle.vote(a, offs, D, 1, 3)
    assert c2.max() <= 3 and np.array_equal(c2, np.minimum(counts, 3))


def test_error_free_reads_vote_for_true_location():
    ref = synth.reference(300_000, 32)
    k, w = 21, 11
    reads, offs, truth = synth.reads(ref, 400, synth.SHORT, synth.ErrorModel(0.0, 1, 0, 0), 0,
                                     rng=np.random.default_rng(4))
    idx = oracle.Index(ref, "10", k, w, 500)
    a, _ = idx.seed(reads, offs, 32)
    rec, counts = oracle.vote(a, offs, 10, 2, 4)
    span = 2 * k - 1
    for r in range(offs.size - 1):
        top = rec[rec["read_id"] == r][0]
        want = int(truth["start"][r]) - (span - 1 if truth["strand"][r] else 0)
        assert int(top["strand"]) == int(truth["strand"][r])
        assert int(top["loc"]) == want
