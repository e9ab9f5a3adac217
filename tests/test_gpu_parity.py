"""GPU path vs the oracle, element by element, through the C ABI.

Every comparison is exact (integer work): the same minimizer set (key,
position, strand) per sequence, the same filtered index (keys, offsets,
entries), the same per-read alignment index, the same sorted anchor list.
Sizes span several sketch tiles (2048 positions) with ragged tails; edge cases
cover empty and tiny inputs, N and lower-case bases, even k (palindromes),
long reads (prefix-capped pattern alignment + a second seeding pass), reads
with N in the pattern-alignment prefix (full-length fallback), and reads whose
anchor lists exceed one shared-memory sort (merge passes).
"""
import random

import numpy as np
import pytest

import oracle
from paper_2211_08157_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def god():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2211_08157_gb300 as g
    g.load()
    return g


def rand_bytes(rng, n, n_rate=0.0, lower=0.0):
    s = synth.ACGT[rng.integers(0, 4, n)].copy()
    if n_rate:
        m = rng.random(n) < n_rate
        s[m] = np.frombuffer(b"N", dtype=np.uint8)[0]
    if lower:
        m = rng.random(n) < lower
        s[m] = s[m] | 0x20
    return s


def assert_anchors_equal(got, want):
    assert got.size == want.size, (got.size, want.size)
    if got.size:
        bad = np.nonzero(got.view(np.uint32).reshape(-1, 4) != want.view(np.uint32).reshape(-1, 4))[0]
        assert bad.size == 0, f"first mismatch at {bad[0]}: got {got[bad[0]]} want {want[bad[0]]}"


# ----------------------------------------------------------------- sketch
SKETCH_CASES = [
    (0, "10", 0, 21, 11, 0.0), (1, "10", 0, 21, 11, 0.0), (60, "1", 0, 15, 10, 0.0),
    (5_000, "10", 0, 21, 11, 0.0), (5_000, "10", 1, 21, 11, 0.01), (20_003, "110", 2, 19, 19, 0.002),
    (33_333, "1", 0, 16, 5, 0.001), (12_345, "1000101001", 3, 12, 7, 0.0), (9_999, "01", 0, 8, 4, 0.02),
    (40_000, "1110", 1, 28, 40, 0.0), (4_321, "1", 0, 1, 1, 0.01), (7_777, "10", 0, 4, 3, 0.0),
    (100_000, "10", 0, 15, 10, 0.0005), (2_500, "1", 0, 11, 255, 0.0), (3_000, "11", 1, 2, 2, 0.0),
    # hash-width boundaries (2k = 34, 46, 50) with register window stages
    (15_000, "1", 0, 17, 12, 0.0), (20_000, "110", 0, 23, 19, 0.001), (30_000, "10", 0, 25, 11, 0.001),
]


@pytest.mark.parametrize("case", SKETCH_CASES, ids=[f"L{c[0]}-{c[1]}-s{c[2]}-k{c[3]}w{c[4]}" for c in SKETCH_CASES])
def test_sketch_matches_oracle(god, case):
    L, P, s, k, w, nr = case
    rng = np.random.default_rng(L + k * 31 + w)
    seq = rand_bytes(rng, L, n_rate=nr, lower=0.05)
    gk, gp, gz = god.god_sketch(seq, P, s, k, w)
    ok, op, oz, _ = oracle.minimizers(seq, P, s, k, w)
    assert np.array_equal(gk, ok)
    assert np.array_equal(gp.astype(np.uint64), op)
    assert np.array_equal(gz.astype(np.uint32), oz)


def test_sketch_low_complexity(god):
    # homopolymers and dinucleotide repeats: every position ties, palindromes for even k
    seq = np.frombuffer(b"A" * 5000 + b"AT" * 3000 + b"ACGT" * 2000 + b"C" * 100, dtype=np.uint8)
    for k, w in [(15, 10), (16, 10), (4, 3), (21, 11), (2, 5)]:
        gk, gp, gz = god.god_sketch(seq, "1", 0, k, w)
        ok, op, oz, _ = oracle.minimizers(seq, "1", 0, k, w)
        assert np.array_equal(gk, ok) and np.array_equal(gp.astype(np.uint64), op), (k, w)


def test_sketch_every_byte_value(god):
    """Bytes other than ACGT/acgt (all 256 values, at random positions) read as
    N, for contiguous and spread-out patterns at every shift."""
    rng = np.random.default_rng(41)
    seq = rand_bytes(rng, 24_000, lower=0.2)
    hit = rng.random(seq.size) < 0.01
    seq[hit] = rng.integers(0, 256, int(hit.sum()))
    seq[1000:1256] = np.arange(256)
    seq[5000:5512] = np.repeat(np.arange(256), 2)
    for P, k, w in [("10", 21, 11), ("110", 19, 19), ("1", 15, 10), ("1110", 17, 9), ("1000101001", 12, 7)]:
        for s in range(len(P)):
            gk, gp, gz = god.god_sketch(seq, P, s, k, w)
            ok, op, oz, _ = oracle.minimizers(seq, P, s, k, w)
            assert np.array_equal(gk, ok) and np.array_equal(gp.astype(np.uint64), op), (P, s)
            assert np.array_equal(gz.astype(np.uint32), oz), (P, s)


# ----------------------------------------------------------------- index
# hash slots hold (start, count) where the fields fit (k <= 21 here) and the
# key's rank otherwise (k = 28: a 40-bit quotient leaves too few bits)
@pytest.mark.parametrize("P,k,w,occ", [("10", 21, 11, 500), ("110", 19, 19, 3), ("1", 15, 10, 2), ("1010", 13, 6, 1),
                                       ("10", 28, 11, 500), ("1", 28, 5, 2**32 - 1), ("1", 15, 10, 2**32 - 1)])
def test_index_matches_oracle(god, P, k, w, occ):
    ref = synth.reference(300_000, 7, synth.RepeatModel(20, 300, 900, False, 0.0, 0.02, 0.3))
    idx = god.god_build_index(ref, P, k, w, occ)
    gk, gs, ge = god.god_index_export(idx)
    o = oracle.Index(ref, P, k, w, occ)
    ok, os_, oe = o.dump()
    assert idx.info["n_minimizers"] == o.sizes()[0]
    assert np.array_equal(gk, ok)
    assert np.array_equal(gs, os_)
    assert np.array_equal(ge, oe)
    # lookups of present and absent keys
    absent = np.random.default_rng(1).integers(0, 4 ** k, 5000, dtype=np.uint64)
    q = np.concatenate([ok, absent])
    cnt, first = god.god_index_lookup(idx, q, via=0)
    assert np.array_equal(cnt.astype(np.uint64), o.count(q))
    present = cnt > 0
    assert np.array_equal(first[: ok.size], os_[:-1])
    idx.close()


def test_index_empty_and_tiny(god):
    for ref in [b"", b"A", b"ACGTN" * 3, b"N" * 100]:
        idx = god.god_build_index(np.frombuffer(ref, dtype=np.uint8) if ref else np.zeros(0, np.uint8),
                                  "10", 5, 3, 10)
        gk, gs, ge = god.god_index_export(idx)
        o = oracle.Index(ref, "10", 5, 3, 10)
        ok, os_, oe = o.dump()
        assert np.array_equal(gk, ok) and np.array_equal(gs, os_) and np.array_equal(ge, oe)
        idx.close()


# ----------------------------------------------------------------- seeding
def _seed_compare(god, ref, reads, offs, P, k, w, occ, t=32, params=None, check_shifts=True):
    idx = god.god_build_index(ref, P, k, w, occ, params=params)
    n = offs.size - 1
    shifts = np.zeros(max(n, 1), np.uint32)
    out = np.zeros((max(reads.size, 1000) + 1000, 4), np.uint32)
    try:
        m = god.god_seed_into(idx, reads, offs, out, pa_t=t, shifts_out=shifts)
    except god.GodError as e:
        assert e.rc == -5
        out = np.zeros((e.needed, 4), np.uint32)
        m = god.god_seed_into(idx, reads, offs, out, pa_t=t, shifts_out=shifts)
    got = out[:m].copy().view(god.ANCHOR_DTYPE).reshape(-1)
    want, oshift = oracle.Index(ref, P, k, w, occ).seed(reads, offs, t)
    if check_shifts:
        assert np.array_equal(shifts[:n], oshift)
    assert_anchors_equal(got, want)
    return idx, got


def test_seed_tiny_config_full(god):
    """1 Mbp iid reference, 10,000 x 150 bp reads, 0.1% substitutions, pattern 10, k21 w11."""
    wl = synth.WORKLOADS["tiny_1mbp_short"]
    ref = wl.make_reference()
    reads, offs, _ = wl.make_reads(ref)
    idx, got = _seed_compare(god, ref, reads, offs, wl.pattern, wl.k, wl.w, wl.max_occ)
    # the plain god_seed entry point returns the same list
    assert_anchors_equal(god.god_seed(idx, reads, offs), got)
    assert got.size > 50_000


@pytest.mark.parametrize("P,k,w,t", [("110", 19, 19, 32), ("10", 15, 10, 8), ("1", 12, 5, 4), ("10", 14, 6, 16),
                                     ("1110", 17, 9, 0)])
def test_seed_long_reads(god, P, k, w, t):
    """Long reads: prefix-capped pattern alignment (odd k) and the second
    seeding pass at full length; even k runs uncapped."""
    ref = synth.reference(400_000, 11, synth.RepeatModel(30, 500, 2000, False, 0.0, 0.03, 0.2))
    lens = synth.LengthModel("lognormal", mu=8.0, sigma=0.6, lo=50, hi=20_000)
    reads, offs, _ = synth.reads(ref, 300, lens, synth.ErrorModel(0.01, 1, 2, 2), 11)
    _seed_compare(god, ref, reads, offs, P, k, w, 200, t=t)


def test_seed_reads_with_n_and_edge_lengths(god):
    """N in the pattern-alignment prefix forces the full-length fallback; empty
    and shorter-than-window reads yield no anchors."""
    rng = np.random.default_rng(21)
    ref = synth.reference(200_000, 12)
    parts, offs = [], [0]
    for i in range(400):
        L = int(rng.choice([0, 1, 5, 30, 150, 700, 3000]))
        s = int(rng.integers(0, ref.size - L)) if L else 0
        r = ref[s:s + L].copy()
        if L and i % 3 == 0:
            r[rng.integers(0, L, max(1, L // 200))] = ord("N")
        if L and i % 5 == 0:
            r = synth.revcomp(r)
        parts.append(r)
        offs.append(offs[-1] + L)
    reads = np.concatenate(parts)
    offs = np.array(offs, np.uint64)
    _seed_compare(god, ref, reads, offs, "110", 19, 9, 500, t=4)
    _seed_compare(god, ref, reads, offs, "10", 21, 11, 500, t=32)


def test_seed_short_segments_and_odd_bytes(god):
    """Reads of 0-40 and 150 bases with non-ACGT bytes: chunks that straddle
    one, two or more segment ends and separators next to N."""
    rng = np.random.default_rng(23)
    ref = synth.reference(100_000, 14)
    parts, offs = [], [0]
    for i in range(3000):
        L = int(rng.choice([0, 1, 2, 7, 8, 9, 15, 16, 17, 23, 33, 40, 150]))
        s = int(rng.integers(0, ref.size - L)) if L else 0
        r = ref[s:s + L].copy()
        if L and i % 4 == 0:
            r[rng.integers(0, L, max(1, L // 30))] = rng.integers(0, 256, max(1, L // 30))
        if L and i % 3 == 0:
            r = r | np.uint8(0x20) * (rng.random(L) < 0.3).astype(np.uint8)
        parts.append(r)
        offs.append(offs[-1] + L)
    reads = np.concatenate(parts)
    offs = np.array(offs, np.uint64)
    _seed_compare(god, ref, reads, offs, "10", 9, 3, 200, t=0)
    _seed_compare(god, ref, reads, offs, "110", 10, 4, 200, t=0)
    _seed_compare(god, ref, reads, offs, "1", 11, 3, 200, t=0)


def test_seed_rank_slots(god):
    """k = 28: the index's hash slots hold ranks (no room for the entry range),
    so lookups go through the offsets array."""
    ref = synth.reference(300_000, 15, synth.RepeatModel(20, 300, 900, False, 0.0, 0.02, 0.3))
    lens = synth.LengthModel("fixed", fixed=150)
    reads, offs, _ = synth.reads(ref, 2000, lens, synth.ErrorModel(0.002, 1, 1, 1), 15)
    _seed_compare(god, ref, reads, offs, "10", 28, 11, 500)
    _seed_compare(god, ref, reads, offs, "1", 28, 9, 3)


def test_seed_long_anchor_lists(god):
    """Reads whose anchor list exceeds one shared-memory sort (8192): chunked
    sorts plus merge-path passes."""
    rng = np.random.default_rng(5)
    unit = synth.ACGT[rng.integers(0, 4, 3000)]
    parts = []
    for _ in range(60):  # 60 near-exact copies separated by random spacers
        parts.append(synth.ACGT[rng.integers(0, 4, 100)])
        parts.append(synth._substitute(unit, 0.002, rng))
    ref = np.concatenate(parts)
    reads = np.concatenate([unit, unit[:1500], synth.revcomp(unit), ref[5000:25000]])
    offs = np.array([0, 3000, 4500, 7500, 27500], np.uint64)
    _, got = _seed_compare(god, ref, reads, offs, "1", 15, 5, 1000, t=0)
    per_read = np.bincount(got["read_id"], minlength=4)
    assert per_read.max() > 8192


def test_seed_empty_batch(god):
    ref = synth.reference(50_000, 13)
    idx = god.god_build_index(ref, "10", 21, 11, 500)
    got = god.god_seed(idx, np.zeros(0, np.uint8), np.zeros(1, np.uint64))
    assert got.size == 0
    got = god.god_seed(idx, np.zeros(0, np.uint8), np.zeros(4, np.uint64))  # 3 empty reads
    assert got.size == 0


def test_seed_device_entry_point(god):
    import torch
    wl = synth.WORKLOADS["tiny_1mbp_short"]
    ref = wl.make_reference()
    reads, offs, _ = wl.make_reads(ref, n=2000)
    idx = god.god_build_index(torch.from_numpy(ref).cuda(), "10", 21, 11, 500)
    dr = torch.from_numpy(reads).cuda()
    do = torch.from_numpy(offs.view(np.int64)).cuda()
    ptr, m = god.god_seed_device(idx, dr, do)
    torch.cuda.synchronize()

    class DevView:  # wraps the library's device array for torch without a copy
        __cuda_array_interface__ = {"shape": (m * 4,), "typestr": "<i4", "data": (ptr, False), "version": 2}

    got = torch.as_tensor(DevView(), device="cuda").cpu().numpy().view(np.uint32).view(god.ANCHOR_DTYPE)
    god.god_free(ptr)
    got = got.reshape(-1)
    want, _ = oracle.Index(ref, "10", 21, 11, 500).seed(reads, offs, 32)
    assert_anchors_equal(got, want)
    # caller-owned device output through god_seed_into; too-small buffers report the size
    out = torch.empty((m, 4), dtype=torch.int32, device="cuda")
    assert god.god_seed_into(idx, dr, do, out) == m
    assert_anchors_equal(out.cpu().numpy().view(np.uint32).view(god.ANCHOR_DTYPE).reshape(-1), want)
    small = torch.empty((m // 2, 4), dtype=torch.int32, device="cuda")
    with pytest.raises(god.GodError) as e:
        god.god_seed_into(idx, dr, do, small)
    assert e.value.rc == -5


def test_pinned_host_buffers_in_place(god):
    """Page-locked host inputs are read in place by the kernels (no staging
    copies; the output is copied back into page-locked memory); results equal
    the pageable-host path and the oracle."""
    import torch
    wl = synth.WORKLOADS["tiny_1mbp_short"]
    ref = wl.make_reference()
    reads, offs, _ = wl.make_reads(ref, n=3000)
    h_ref = torch.from_numpy(ref).pin_memory()
    h_reads = torch.from_numpy(reads).pin_memory()
    h_offs = torch.from_numpy(offs.view(np.int64)).pin_memory()
    idx = god.god_build_index(h_ref.numpy(), "10", 21, 11, 500)
    want, _ = oracle.Index(ref, "10", 21, 11, 500).seed(reads, offs, 32)
    h_out = torch.zeros((want.size + 64, 4), dtype=torch.int32).pin_memory()
    m = god.god_seed_into(idx, h_reads.numpy(), h_offs.numpy().view(np.uint64), h_out.numpy())
    got = h_out.numpy()[:m].view(np.uint32).view(god.ANCHOR_DTYPE).reshape(-1)
    assert_anchors_equal(got, want)
    ka, sa, ea = god.god_index_export(idx)
    kb, sb, eb = god.god_index_export(god.god_build_index(ref, "10", 21, 11, 500))
    assert np.array_equal(ka, kb) and np.array_equal(sa, sb) and np.array_equal(ea, eb)


def test_seed_rejects_bad_offsets(god):
    ref = synth.reference(50_000, 14)
    idx = god.god_build_index(ref, "10", 21, 11, 500)
    reads = ref[:1000].copy()
    with pytest.raises(god.GodError) as e:
        god.god_seed(idx, reads, np.array([0, 500, 400, 1000], np.uint64))
    assert e.value.rc == -1
