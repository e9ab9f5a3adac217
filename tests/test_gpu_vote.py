"""Location voting on the GPU (god_vote) against the oracle (Sec. 3.4, Fig. 8, Sec. 3.6.3).

Integer results, so every record must be equal: read id, votes, strand, the
rescue flag, the location v0 and the reference / read stretches, in the same
order (votes descending, then strand and location), and every per-read count.

* Random anchor lists per read of every size class: none, up to 32 votes (a
  warp sorts them in registers), 33-4096 (a CTA sorts them in shared memory)
  and past 4096 (sorted chunks merged in a global buffer), with clustered and
  scattered locations on both strands, several (D, V, max_out), host and
  device buffers.
* Anchors of seeded reads: the 1 Mbp / 10,000-read workload (short-read
  voting) and long HiFi-like reads over low-divergence repeats (long-read
  voting, lists past 4096 votes, rescue).
* Errors: anchors not grouped by read, a read id out of range and bad
  parameters are refused before any result is written.
"""
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


def random_anchors(rng, sizes, lens):
    rows = []
    for r, m in enumerate(sizes):
        if m == 0:
            continue
        n_diag = int(rng.integers(1, 6))
        diags = rng.integers(0, 5_000_000, n_diag)
        rp = rng.integers(0, lens[r], m)
        which = rng.integers(0, n_diag, m)
        jitter = rng.integers(-80, 80, m)
        scatter = rng.random(m) < 0.3
        ref = np.where(scatter, rng.integers(0, 5_000_000, m), diags[which] + rp + jitter)
        ref = np.clip(ref, 0, 2**32 - 1)
        strand = rng.integers(0, 2, m)
        rows.append(np.stack([np.full(m, r), rp, ref, strand], axis=1))
    a = np.concatenate(rows).astype(np.uint32) if rows else np.zeros((0, 4), np.uint32)
    order = np.lexsort((a[:, 3], a[:, 1], a[:, 2], a[:, 0]))
    return np.ascontiguousarray(a[order])


def test_vote_random_lists_match_oracle(god):
    import torch
    rng = np.random.default_rng(90)
    sizes = [0, 1, 2, 5, 31, 32, 33, 100, 1000, 4095, 4096, 4097, 9000, 20_000, 0, 7, 64, 3000]
    sizes += rng.integers(0, 60, 300).tolist()
    lens = rng.integers(150, 60_000, len(sizes))
    offs = np.zeros(len(sizes) + 1, np.uint64)
    offs[1:] = np.cumsum(lens)
    a = random_anchors(rng, sizes, lens)
    for D, V, max_out in ((100, 3, 8), (0, 1, 1), (5000, 2, 32), (60, 10, 4)):
        want, wc = oracle.vote(a, offs, D, V, max_out)
        got, gc = god.god_vote(a, offs, D, V, max_out)                    # host buffers
        assert np.array_equal(gc, wc), (D, V, max_out)
        assert np.array_equal(got, want), (D, V, max_out)
        # device buffers
        n = offs.size - 1
        d_a = torch.from_numpy(a.view(np.int32)).cuda()
        d_o = torch.from_numpy(offs.view(np.int64)).cuda()
        d_out = torch.zeros((n * max_out, 10), dtype=torch.int32, device="cuda")
        d_cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
        god.god_vote(d_a, d_o, D, V, max_out, out=d_out, counts=d_cnt)
        cnt = d_cnt.cpu().numpy().view(np.uint32)
        rec = d_out.cpu().numpy().view(oracle.VOTE_DTYPE).reshape(-1)
        keep = (np.arange(max_out)[None, :] < cnt[:, None]).reshape(-1)
        assert np.array_equal(cnt, wc) and np.array_equal(rec[keep], want)


def test_vote_seeded_short_reads(god):
    wl = synth.WORKLOADS["tiny_1mbp_short"]
    ref = wl.make_reference()
    reads, offs, truth = wl.make_reads(ref)
    idx = god.god_build_index(ref, wl.pattern, wl.k, wl.w, wl.max_occ)
    a = god.god_seed(idx, reads, offs)
    for D, V, max_out in ((20, 2, 4), (150, 3, 8)):
        want, wc = oracle.vote(a, offs, D, V, max_out)
        got, gc = god.god_vote(a, offs, D, V, max_out)
        assert np.array_equal(gc, wc) and np.array_equal(got, want)
    # most reads vote for their true start (forward) on the true strand
    first = np.zeros(offs.size - 1, np.int64) - 1
    starts = np.concatenate([[0], np.cumsum(gc.astype(np.int64))[:-1]]).astype(np.int64)
    has = gc > 0
    first[has] = got["loc"][starts[has]]
    fwd = (truth["strand"] == 0) & has
    assert np.mean(first[fwd] == truth["start"][fwd]) > 0.95
    idx.close()


def test_vote_seeded_long_reads(god):
    # long reads over a reference with low-divergence repeats: lists of up to
    # ~25,000 votes, a third of the reads past 4096
    ref = synth.reference(3_000_000, 71, synth.RepeatModel(20, 1000, 5000, False, 0.0, 0.02, 0.5))
    reads, offs, _ = synth.reads(ref, 200, synth.LengthModel("lognormal", mu=9.6, sigma=0.5, lo=2000, hi=60_000),
                                 synth.HIFI_ERR, 0, rng=np.random.default_rng(72))
    idx = god.god_build_index(ref, "10", 15, 10, 1000)
    a = god.god_seed(idx, reads, offs)
    assert (np.bincount(a["read_id"]) > 4096).sum() > 20       # chunked lists are exercised
    for D, V, max_out in ((100, 3, 16), (500, 40, 2), (50, 1_000_000, 4)):
        want, wc = oracle.vote(a, offs, D, V, max_out)
        got, gc = god.god_vote(a, offs, D, V, max_out)
        assert np.array_equal(gc, wc) and np.array_equal(got, want)
    assert want["rescue"].all()                                # V out of reach: every read rescued
    idx.close()


def test_vote_rejects_bad_input(god):
    offs = np.array([0, 100, 200], np.uint64)
    a = np.array([[1, 5, 50, 0], [0, 5, 70, 0]], np.uint32)            # not grouped by ascending read
    with pytest.raises(god.GodError) as e:
        god.god_vote(a, offs, 10, 1, 4)
    assert e.value.rc == -1
    a = np.array([[0, 5, 50, 0], [2, 5, 70, 0]], np.uint32)            # read 2 of 2
    with pytest.raises(god.GodError):
        god.god_vote(a, offs, 10, 1, 4)
    a = np.array([[0, 5, 50, 0]], np.uint32)
    for V, max_out in ((0, 4), (1, 0), (1, 33)):
        with pytest.raises(god.GodError):
            god.god_vote(a, offs, 10, V, max_out)
