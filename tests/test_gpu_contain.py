"""Containment search on the GPU (god_contain) against the oracle (Sec. 2.3).

Integer results, so per read the genome and votes, and per genome the mapped
reads and read bases, must be equal.

* A planted database (four unrelated genomes of 1-3 contigs, reads from two
  of them, both strands) with the batch holding everything, one contig per
  batch and batches in between; hash and learned index.
* A synthetic metagenome at the paper's containment setting (pattern 10,
  k = 28, w = 40): 40 genomes of 0.2-2 Mbp, HiFi-like reads (about 2 kb, 0.1 %
  errors) drawn from 10 of them at uneven abundance, the database indexed in
  batches of 16 Mbp.
"""
import numpy as np
import pytest

import oracle
from paper_2211_08157_gb300 import synth

from test_oracle_contain_pins import database, sample_reads

pytestmark = pytest.mark.gpu

LEN = synth.LengthModel("lognormal", mu=7.6, sigma=0.3, lo=800, hi=6000)


@pytest.fixture(scope="module")
def god():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2211_08157_gb300 as g
    g.load()
    return g


def both(god, db, off, gen, ng, reads, roff, pattern, k, w, max_occ, t, D, V, batch, kind=0):
    want = oracle.contain(db, off, gen, ng, reads, roff, pattern, k, w, max_occ, t, D, V, batch, threads=8)
    got = god.god_contain(db, off, gen, ng, reads, roff, pattern=pattern, k=k, w=w, max_occ=max_occ, pa_t=t, D=D,
                          V=V, batch_bases=batch, index_kind=kind)
    for x, y in zip(got, want):
        assert np.array_equal(x, y)
    return got


def test_contain_planted(god):
    rng = np.random.default_rng(11)
    db, off, gen, contigs, per = database(rng, [150_000, 200_000, 120_000, 180_000])
    reads, roff, truth_c = sample_reads(rng, contigs, per[1] + per[3], 600, 1000)
    for batch, kind in ((1 << 40, 0), (1, 0), (250_000, 1)):
        rg, rv, gr, gb = both(god, db, off, gen, 4, reads, roff, "10", 21, 11, 500, 32, 50, 3, batch, kind)
        assert np.array_equal(rg, gen[truth_c])


def test_contain_metagenome(god):
    rng = np.random.default_rng(21)
    sizes = rng.integers(200_000, 2_000_000, 40).tolist()
    db, off, gen, contigs, per = database(rng, sizes)
    present = rng.choice(40, 10, replace=False)
    abundance = rng.dirichlet(np.ones(10))
    n = 30_000
    parts, roffs = [], [np.zeros(1, np.uint64)]
    counts = rng.multinomial(n, abundance)
    for g, c in zip(present, counts):
        ref_g = np.concatenate([contigs[j] for j in per[g]])
        r, o, _ = synth.reads(ref_g, int(c), LEN, synth.HIFI_ERR, 0, rng=np.random.default_rng(1000 + int(g)))
        parts.append(r)
        roffs.append(o[1:] + roffs[-1][-1])
    reads = np.concatenate(parts)
    roff = np.concatenate(roffs)
    rg, rv, gr, gb = both(god, db, off, gen, 40, reads, roff, "10", 28, 40, 1000, 32, 100, 3, 16_000_000)
    absent = np.setdiff1d(np.arange(40), present)
    assert gr[absent].sum() == 0
    assert gr[present].sum() >= 0.95 * n
