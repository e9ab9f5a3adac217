"""Pins of the C++ oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: the paper's
Fig. 3 worked example, closed forms (patterned length, kept-position arithmetic,
the hash for small k), invariants (hash bijectivity, reverse-complement symmetry,
minimizer density 2/(w+1), index shrinkage x/p), and brute force on tiny inputs
written along a different route (string k-mers, shift-add hash, window scan).
"""
import os
import random

import numpy as np
import pytest

import oracle
from paper_2211_08157_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
COMP = str.maketrans("ACGT", "TGCA")


# ----------------------------------------------------------------------------- helpers
def ones_positions(P):
    return [i for i, c in enumerate(P) if c == "1"]


def kept_positions_closed_form(L, P, s):
    """orig(j) = s + p * (j // x) + off[j mod x] (arithmetic, no scan)."""
    off = ones_positions(P)
    p, x = len(P), len(off)
    out = []
    j = 0
    while True:
        o = s + p * (j // x) + off[j % x]
        if o >= L:
            return out
        out.append(o)
        j += 1


def wang_shift_add(v, k):
    """The hash in its shift-add form on Python integers (independent of the oracle's
    multiplicative form)."""
    mask = (1 << (2 * k)) - 1
    v = (~v + (v << 21)) & mask
    v ^= v >> 24
    v = (v + (v << 3) + (v << 8)) & mask
    v ^= v >> 14
    v = (v + (v << 2) + (v << 4)) & mask
    v ^= v >> 28
    v = (v + (v << 31)) & mask
    return v


def brute_minimizers(seq: str, P: str, s: int, k: int, w: int):
    """Set of (key, orig_pos, z) by enumerating every window of the patterned string."""
    pos = kept_positions_closed_form(len(seq), P, s)
    pat = "".join(seq[i] for i in pos).upper()  # lower case reads as upper case
    nk = len(pat) - k + 1
    info = []
    for j in range(max(nk, 0)):
        km = pat[j:j + k]
        if any(c not in "ACGT" for c in km):
            info.append(None)
            continue
        rc = km[::-1].translate(COMP)
        f = int(km.translate(str.maketrans("ACGT", "0123")), 4)
        r = int(rc.translate(str.maketrans("ACGT", "0123")), 4)
        info.append((wang_shift_add(min(f, r), k), int(r < f), f == r))
    out = set()
    for i in range(0, nk - w + 1):
        win = info[i:i + w]
        if any(v is None for v in win):
            continue
        cands = [v[0] for v in win if not v[2]]
        if not cands:
            continue
        mn = min(cands)
        for d, v in enumerate(win):
            if not v[2] and v[0] == mn:
                out.add((v[0], pos[i + d], v[1]))
    return out


def oracle_set(seq, P, s, k, w):
    keys, pos, z, _ = oracle.minimizers(seq.encode() if isinstance(seq, str) else seq, P, s, k, w)
    return set(zip(keys.tolist(), pos.tolist(), z.tolist()))


def rand_seq(rng, n, n_rate=0.0, lower=0.0):
    s = [rng.choice("ACGT") for _ in range(n)]
    for i in range(n):
        if rng.random() < n_rate:
            s[i] = rng.choice("NRY-")
        elif rng.random() < lower:
            s[i] = s[i].lower()
    return "".join(s)


# ----------------------------------------------------------------------------- sparsify
def test_sparsify_identity_pattern():
    rng = random.Random(1)
    seq = rand_seq(rng, 500, n_rate=0.05)
    codes, orig = oracle.sparsify(seq.encode(), "1", 0)
    assert orig.tolist() == list(range(500))
    want = ["ACGT".index(c) if c in "ACGT" else 4 for c in seq]
    assert codes.tolist() == want


@pytest.mark.parametrize("P", ["1", "10", "01", "110", "100", "1110", "1000101001", "0110"])
def test_sparsify_length_and_positions_closed_form(P):
    """Sec. 3.1: patterned length = number of 1s of the diet pattern laid over the
    sequence = x * floor(L' / p) + ones(P[:L' mod p]) with L' = L - s."""
    p, x = len(P), P.count("1")
    for L in [0, 1, 2, 7, 30, 101, 1000]:
        for s in range(p):
            codes, orig = oracle.sparsify(b"A" * L, P, s)
            Lp = max(L - s, 0)
            assert len(orig) == x * (Lp // p) + P[: Lp % p].count("1")
            assert orig.tolist() == kept_positions_closed_form(L, P, s)


def test_fig3_seed_spans():
    """Fig. 3(b): pattern 1000101001, k = 4: seeds 0,1,2 have gap sequences
    (4,2,3), (2,3,1), (3,1,4) between the original positions of their bases."""
    lines = [l.split() for l in open(os.path.join(GOLDEN, "fig3_seed_gaps.txt")) if l.strip() and not l.startswith("#")]
    P = lines[0][1]
    k = int(lines[1][1])
    _, orig = oracle.sparsify(b"ACGT" * 20, P, 0)
    for row in lines[2:]:
        j = int(row[0])
        gaps = [int(g) for g in row[1:]]
        span = orig[j:j + k].astype(np.int64)
        assert np.diff(span).tolist() == gaps


def test_reduction_ratio_beta():
    """beta = p / x: the patterned genome is p/x times shorter (Sec. 3)."""
    for P in ["10", "110", "1110", "100"]:
        codes, _ = oracle.sparsify(b"C" * 60000, P, 0)
        assert abs(60000 / len(codes) - len(P) / P.count("1")) < 1e-9


# ----------------------------------------------------------------------------- hash
@pytest.mark.parametrize("k", list(range(1, 12)))
def test_hash_is_permutation(k):
    x = np.arange(4 ** k, dtype=np.uint64)
    h = oracle.wang_hash(x, k)
    assert np.array_equal(np.sort(h), x)


def test_hash_small_k_closed_forms():
    """For k <= 7 every right shift (>= 14) and every 2^21 / 2^31 term vanishes mod
    2^(2k), so H(x) = (2^(2k) - 1 - x) * 265 * 21 mod 2^(2k); worked by hand for k = 1..3:
    k=1: H(x) = 3 - x; k=2: H(x) = 13 (15 - x) mod 16; k=3: H(x) = 61 (63 - x) mod 64."""
    assert oracle.wang_hash(np.arange(4), 1).tolist() == [3, 2, 1, 0]
    assert oracle.wang_hash(np.arange(16), 2).tolist() == [(13 * (15 - v)) % 16 for v in range(16)]
    assert oracle.wang_hash(np.arange(64), 3).tolist() == [(61 * (63 - v)) % 64 for v in range(64)]
    for k in range(1, 8):
        m = 1 << (2 * k)
        x = np.arange(m, dtype=np.uint64)
        want = [((m - 1 - v) * 265 * 21) % m for v in range(m)]
        assert oracle.wang_hash(x, k).tolist() == want


@pytest.mark.parametrize("k", [8, 11, 13, 15, 19, 21, 28])
def test_hash_matches_shift_add_form(k):
    rng = np.random.default_rng(k)
    x = rng.integers(0, 4 ** k, 2000, dtype=np.uint64)
    got = oracle.wang_hash(x, k).tolist()
    assert got == [wang_shift_add(int(v), k) for v in x.tolist()]


def _inverse_hash(v, k):
    """Undo each step: odd multipliers by their inverse mod 2^(2k); x ^= x >> s by
    repeated application."""
    bits = 2 * k
    m = 1 << bits
    mask = m - 1

    def unxs(y, s):
        x = y
        for _ in range(bits // max(s, 1) + 1):
            x = y ^ (x >> s)
        return x & mask

    v = (v * pow((1 << 31) + 1, -1, m)) & mask
    v = unxs(v, 28)
    v = (v * pow(21, -1, m)) & mask
    v = unxs(v, 14)
    v = (v * pow(265, -1, m)) & mask
    v = unxs(v, 24)
    v = ((v + 1) * pow((1 << 21) - 1, -1, m)) & mask
    return v


@pytest.mark.parametrize("k", [15, 19, 21, 28])
def test_hash_invertible_large_k(k):
    rng = np.random.default_rng(100 + k)
    x = rng.integers(0, 4 ** k, 500, dtype=np.uint64)
    h = oracle.wang_hash(x, k)
    assert [_inverse_hash(int(v), k) for v in h.tolist()] == x.tolist()


# ----------------------------------------------------------------------------- minimizers
@pytest.mark.parametrize("trial", range(40))
def test_minimizers_brute_force(trial):
    rng = random.Random(trial)
    k = rng.randint(1, 12)
    w = rng.randint(1, 16)
    P = rng.choice(["1", "10", "01", "110", "100", "1000101001", "1101"])
    s = rng.randrange(len(P))
    seq = rand_seq(rng, rng.randint(0, 160), n_rate=rng.choice([0, 0.01, 0.05]), lower=0.1)
    if trial % 5 == 0:   # low-complexity stretch: ties and palindromes
        seq = seq[:20] + "ACGT" * 10 + "AAAAAAAAAAAA" + seq[20:]
    assert oracle_set(seq, P, s, k, w) == brute_minimizers(seq, P, s, k, w)


def test_any_other_byte_reads_as_n():
    """Sec. 3.6.1 alphabet: A, C, G, T in either case are bases; every other
    byte value (all 256 are planted) breaks k-mers exactly like N."""
    rng = np.random.default_rng(3)
    seq = synth.ACGT[rng.integers(0, 4, 6000)].copy()
    lower = rng.random(seq.size) < 0.1
    seq[lower] |= 0x20
    others = np.array([b for b in range(256) if b not in b"ACGTacgt"], dtype=np.uint8)
    hit = rng.random(seq.size) < 0.02
    seq[hit] = rng.choice(others, int(hit.sum()))
    seq[3000:3248] = others
    canon = seq.copy()
    canon[np.isin(canon, others)] = ord("N")
    canon[np.isin(canon, np.frombuffer(b"acgt", np.uint8))] -= 0x20
    for P, k, w in [("1", 15, 10), ("10", 21, 11), ("110", 19, 19), ("1101", 9, 4)]:
        for s in range(len(P)):
            a = oracle.minimizers(seq, P, s, k, w)
            b = oracle.minimizers(canon, P, s, k, w)
            for x, y in zip(a[:3], b[:3]):
                assert np.array_equal(x, y), (P, s)


def test_minimizers_even_k_palindromes():
    # ACGT is its own reverse complement (k = 4): it keeps its window slot but is
    # never a minimizer.
    seq = "ACGT" * 8
    for w in (1, 2, 5):
        got = oracle_set(seq, "1", 0, 4, w)
        assert got == brute_minimizers(seq, "1", 0, 4, w)
    assert oracle_set("ACGT", "1", 0, 4, 1) == set()


def test_minimizers_reverse_complement_symmetry():
    """Identity pattern: minimizers of rc(S) are those of S mirrored, z flipped."""
    rng = np.random.default_rng(7)
    S = synth.ACGT[rng.integers(0, 4, 5001)]
    R = synth.revcomp(S)
    for k, w in [(15, 10), (21, 11), (19, 19)]:
        a = oracle_set(S, "1", 0, k, w)
        b = oracle_set(R, "1", 0, k, w)
        L = S.size
        assert b == {(key, L - k - pos, 1 - z) for key, pos, z in a}


def test_minimizers_reverse_complement_pattern10():
    """Pattern 10, odd L: the patterned rc(S) is the rc of the patterned S, so the
    minimizers mirror with rc position L - 1 - (q + 2(k - 1))."""
    rng = np.random.default_rng(8)
    S = synth.ACGT[rng.integers(0, 4, 4001)]
    R = synth.revcomp(S)
    k, w = 21, 11
    a = oracle_set(S, "10", 0, k, w)
    b = oracle_set(R, "10", 0, k, w)
    L = S.size
    assert b == {(key, L - 1 - (pos + 2 * (k - 1)), 1 - z) for key, pos, z in a}


@pytest.mark.parametrize("k,w", [(21, 11), (19, 19), (15, 10)])
def test_minimizer_density(k, w):
    """Sec. 3.1: density of random minimizers is 2/(w+1) of the k-mer positions."""
    ref = synth.reference(1_000_000, 91)
    keys, _, _, _ = oracle.minimizers(ref, "1", 0, k, w)
    dens = keys.size / (ref.size - k + 1)
    assert abs(dens / (2.0 / (w + 1)) - 1) < 0.03


@pytest.mark.parametrize("P", ["10", "110", "1110", "100"])
def test_index_shrinks_by_pattern_weight(P):
    """Sec. 2.3 / Fig. 6: the seed index shrinks to x/p of the unpatterned one."""
    ref = synth.reference(1_000_000, 92)
    n1 = oracle.minimizers(ref, "1", 0, 15, 10)[0].size
    nP = oracle.minimizers(ref, P, 0, 15, 10)[0].size
    assert abs((nP / n1) / (P.count("1") / len(P)) - 1) < 0.03


# ----------------------------------------------------------------------------- index
def test_index_counts_by_linear_scan():
    ref = synth.reference(200_000, 93, synth.RepeatModel(5, 500, 800, False, 0.0, 0.01, 0.3))
    for max_occ in (1, 2, 5, 1000):
        idx = oracle.Index(ref, "10", 15, 10, max_occ)
        keys, start, ent = idx.dump()
        mk, mp, mz, _ = oracle.minimizers(ref, "10", 0, 15, 10)
        uk, cnt = np.unique(mk, return_counts=True)
        keep = cnt <= max_occ
        assert np.array_equal(keys, uk[keep])
        assert np.array_equal(np.diff(start.astype(np.int64)), cnt[keep])
        # entries: every minimizer of a kept key, sorted by position inside the key
        kept = set(uk[keep].tolist())
        want = sorted((int(a), int(b) * 2 + int(c)) for a, b, c in zip(mk.tolist(), mp.tolist(), mz.tolist()) if a in kept)
        got = [(int(keys[i]), int(e)) for i in range(keys.size) for e in ent[start[i]:start[i + 1]]]
        assert got == want
        assert idx.sizes()[0] == mk.size


def test_index_filter_boundary():
    """A key seen exactly max_occ times is kept; max_occ + 1 times is dropped."""
    rng = np.random.default_rng(3)
    unit = synth.ACGT[rng.integers(0, 4, 80)]
    for copies in (3, 4):
        parts = []
        for c in range(copies):
            parts.append(synth.ACGT[rng.integers(0, 4, 200)])
            parts.append(unit)
        parts.append(synth.ACGT[rng.integers(0, 4, 200)])
        ref = np.concatenate(parts)
        idx = oracle.Index(ref, "1", 13, 5, 3)
        # interior minimizers of the unit recur once per copy
        inner = oracle.minimizers(ref, "1", 0, 13, 5)[0]
        uk, cnt = np.unique(inner, return_counts=True)
        rec = uk[cnt == copies]
        assert rec.size > 0
        got = idx.count(rec)
        assert (got == (copies if copies <= 3 else 0)).all()


# ----------------------------------------------------------------------------- seeding
def _brute_anchors(ref, reads, offs, P, k, w, max_occ, shifts):
    mk, mp, mz, _ = oracle.minimizers(ref, P, 0, k, w)
    uk, cnt = np.unique(mk, return_counts=True)
    cmap = dict(zip(uk.tolist(), cnt.tolist()))
    out = []
    for r in range(offs.size - 1):
        q = reads[int(offs[r]):int(offs[r + 1])]
        qk, qp, qz, _ = oracle.minimizers(q, P, int(shifts[r]), k, w)
        for key, qpos, z in zip(qk.tolist(), qp.tolist(), qz.tolist()):
            if cmap.get(key, 0) > max_occ:
                continue
            for rkey, rpos, rz in zip(mk.tolist(), mp.tolist(), mz.tolist()):
                if rkey == key:
                    out.append((r, rpos, qpos, z ^ rz))
    out.sort()
    return out


def test_anchors_linear_scan():
    ref = synth.reference(30_000, 94, synth.RepeatModel(4, 300, 600, False, 0.0, 0.01, 0.2))
    wl = synth.Workload("t", 94, 30_000, None, 60, synth.SHORT, synth.ILLUMINA_INDEL, "10", 13, 6, 3)
    reads, offs, _ = synth.reads(ref, 60, synth.LengthModel("fixed", fixed=120), synth.ErrorModel(0.02, 1, 1, 1), 94)
    idx = oracle.Index(ref, "10", 13, 6, 3)
    anchors, shifts = idx.seed(reads, offs, 8)
    got = [(int(a["read_id"]), int(a["ref_pos"]), int(a["read_pos"]), int(a["strand"])) for a in anchors]
    assert got == _brute_anchors(ref, reads, offs, "10", 13, 6, 3, shifts)
    assert len(got) > 0


def _pa_brute(idx, read, P, k, w, t):
    sums = []
    for s in range(len(P)):
        keys = oracle.minimizers(read, P, s, k, w)[0]
        if t:
            keys = keys[:t]
        sums.append(int(idx.count(keys).sum()))
    best = max(sums)
    return (sums.index(best) if best > 0 else 0), sums


@pytest.mark.parametrize("P,k,w", [("10", 21, 11), ("110", 19, 19), ("1110", 15, 10)])
def test_pattern_alignment_error_free_reads(P, k, w):
    """Sec. 3.2: error-free reads align to the phase of their origin. Forward read at
    r: a = (-r) mod p. Reverse read of R[r:r+q]: for "10" a = (r + q - 1) mod 2;
    for "110" a = (r + q - 2) mod 3 (reverse(P) is a rotation of P)."""
    ref = synth.reference(300_000, 95)
    idx = oracle.Index(ref, P, k, w, 500)
    rng = np.random.default_rng(5)
    p = len(P)
    for trial in range(60):
        q = int(rng.integers(150, 400))
        r = int(rng.integers(0, ref.size - q))
        fwd = ref[r:r + q]
        a, sums = idx.pattern_align(fwd, 32)
        assert a == (-r) % p
        assert (a, sums.tolist()) == _pa_brute(idx, fwd, P, k, w, 32)
        if P == "10":
            rc_a = (r + q - 1) % 2
        elif P == "110":
            rc_a = (r + q - 2) % 3
        else:
            continue
        a2, _ = idx.pattern_align(synth.revcomp(fwd), 32)
        assert a2 == rc_a


def test_pattern_alignment_sums_brute_force_with_limit():
    ref = synth.reference(100_000, 96)
    idx = oracle.Index(ref, "110", 13, 5, 2)
    rng = np.random.default_rng(9)
    for t in (0, 1, 3, 8):
        for _ in range(20):
            q = int(rng.integers(20, 300))
            r = int(rng.integers(0, ref.size - q))
            read = synth._substitute(ref[r:r + q], 0.05, rng)
            a, sums = idx.pattern_align(read, t)
            assert (a, sums.tolist()) == _pa_brute(idx, read, "110", 13, 5, t)


def test_error_free_read_anchors_on_diagonal():
    """Forward error-free read at offset r with the right phase: every read
    minimizer whose windows lie inside the read matches the reference minimizer at
    the same position, so an anchor with ref_pos - read_pos = r exists."""
    ref = synth.reference(200_000, 97)
    P, k, w = "10", 21, 11
    idx = oracle.Index(ref, P, k, w, 500)
    rng = np.random.default_rng(11)
    for _ in range(30):
        q = 300
        r = int(rng.integers(1000, ref.size - q - 1000))
        read = ref[r:r + q]
        offs = np.array([0, q], np.uint64)
        anchors, shifts = idx.seed(read, offs, 32)
        assert shifts[0] == (-r) % 2
        qk, qp, qz, qj = oracle.minimizers(read, P, int(shifts[0]), k, w)
        m = (q - shifts[0] + 1) // 2
        nk = m - k + 1
        interior = [int(pp) for pp, jj in zip(qp, qj) if w - 1 <= jj <= nk - w]
        diag = {int(a["read_pos"]) for a in anchors if int(a["ref_pos"]) - int(a["read_pos"]) == r and a["strand"] == 0}
        assert set(interior) <= diag
        assert len(interior) > 0


def test_anchor_order_is_total():
    ref = synth.reference(100_000, 98)
    wl = synth.WORKLOADS["tiny_1mbp_short"]
    reads, offs, _ = synth.reads(ref, 300, synth.SHORT, synth.ILLUMINA_SUB, 98)
    idx = oracle.Index(ref, "10", 21, 11, 500)
    a, _ = idx.seed(reads, offs, 32)
    t = list(zip(a["read_id"].tolist(), a["ref_pos"].tolist(), a["read_pos"].tolist(), a["strand"].tolist()))
    assert t == sorted(t) and len(set(t)) == len(t)
    b, _ = idx.seed(reads, offs, 32, threads=4)
    assert np.array_equal(a, b)
