"""Pins of the oracle's containment search (Sec. 2.3): reads mapped against a
database of genomes indexed on the fly in batches; a mapped read is one whose
location voting gives a winning location; per genome, mapped reads and bases.

* Planted truth: reads drawn from two of four unrelated genomes map to exactly
  those genomes (every read), in the numbers drawn; the other two get none;
  mapped bases are the drawn reads' lengths.
* Batch invariance: one batch holding every contig and one batch per contig
  give the same per-read genomes and votes.
* Ties: a region shared by two genomes sends its reads to the genome listed
  first, in one batch (first winner in location order) and across batches
  (earlier batch on ties).
* Pattern 1 (no sparsification) and pattern 10 find the same planted genomes.
"""
import numpy as np

import oracle
from paper_2211_08157_gb300 import synth


def database(rng, sizes):
    """Genomes of 1-3 contigs each: (bytes, contig offsets, contig genome ids, per-genome contig list)."""
    contigs, gen, per = [], [], []
    for g, size in enumerate(sizes):
        n = int(rng.integers(1, 4))
        cuts = np.sort(rng.choice(np.arange(1000, size - 1000), n - 1, replace=False)) if n > 1 else []
        edges = [0, *cuts, size]
        seq = synth.ACGT[rng.integers(0, 4, size)]
        per.append([])
        for a, b in zip(edges[:-1], edges[1:]):
            per[-1].append(len(contigs))
            contigs.append(seq[a:b])
            gen.append(g)
    off = np.zeros(len(contigs) + 1, np.uint64)
    off[1:] = np.cumsum([c.size for c in contigs])
    return np.concatenate(contigs), off, np.array(gen, np.uint32), contigs, per


def sample_reads(rng, contigs, ids, n, length):
    reads, truth = [], []
    for _ in range(n):
        c = int(rng.choice(ids))
        s = int(rng.integers(0, contigs[c].size - length))
        r = contigs[c][s:s + length].copy()
        if rng.random() < 0.5:
            r = synth.revcomp(r)
        reads.append(r)
        truth.append(c)
    off = np.zeros(n + 1, np.uint64)
    off[1:] = np.cumsum([r.size for r in reads])
    return np.concatenate(reads), off, np.array(truth)


ARGS = dict(k=21, w=11, max_occ=500, t=32, D=50, V=3)


def run(db, off, gen, ng, reads, roff, pattern="10", batch=1 << 40):
    return oracle.contain(db, off, gen, ng, reads, roff, pattern, ARGS["k"], ARGS["w"], ARGS["max_occ"], ARGS["t"],
                          ARGS["D"], ARGS["V"], batch, threads=4)


def test_planted_genomes():
    rng = np.random.default_rng(11)
    db, off, gen, contigs, per = database(rng, [150_000, 200_000, 120_000, 180_000])
    ids1 = per[1]
    ids3 = per[3]
    reads, roff, truth_c = sample_reads(rng, contigs, ids1 + ids3, 600, 1000)
    truth_g = gen[truth_c]
    rg, rv, gr, gb = run(db, off, gen, 4, reads, roff)
    assert np.array_equal(rg, truth_g)
    assert gr[0] == 0 and gr[2] == 0
    assert gr[1] == (truth_g == 1).sum() and gr[3] == (truth_g == 3).sum()
    assert gb[1] == 1000 * gr[1] and gb[3] == 1000 * gr[3]
    assert (rv >= ARGS["V"]).all()
    rg1, _, gr1, _ = run(db, off, gen, 4, reads, roff, pattern="1")
    assert np.array_equal(rg1, truth_g) and np.array_equal(gr1, gr)


def test_batch_invariance():
    rng = np.random.default_rng(12)
    db, off, gen, contigs, per = database(rng, [100_000, 90_000, 130_000])
    reads, roff, _ = sample_reads(rng, contigs, list(range(len(contigs))), 400, 800)
    one = run(db, off, gen, 3, reads, roff, batch=1 << 40)
    each = run(db, off, gen, 3, reads, roff, batch=1)       # every contig alone
    mid = run(db, off, gen, 3, reads, roff, batch=150_000)
    for x, y in zip(one, each):
        assert np.array_equal(x, y)
    for x, y in zip(one, mid):
        assert np.array_equal(x, y)


def test_shared_region_goes_to_first_genome():
    rng = np.random.default_rng(13)
    shared = synth.ACGT[rng.integers(0, 4, 6000)]
    a = np.concatenate([synth.ACGT[rng.integers(0, 4, 50_000)], shared, synth.ACGT[rng.integers(0, 4, 50_000)]])
    b = np.concatenate([synth.ACGT[rng.integers(0, 4, 70_000)], shared, synth.ACGT[rng.integers(0, 4, 30_000)]])
    db = np.concatenate([a, b])
    off = np.array([0, a.size, a.size + b.size], np.uint64)
    gen = np.array([0, 1], np.uint32)
    reads = np.concatenate([shared[s:s + 1000] for s in range(0, 5000, 500)])
    roff = np.arange(0, reads.size + 1, 1000, dtype=np.uint64)
    for batch in (1 << 40, 1):
        rg, rv, gr, _ = run(db, off, gen, 2, reads, roff, batch=batch)
        assert (rg == 0).all() and gr[0] == 10 and gr[1] == 0
