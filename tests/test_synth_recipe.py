"""The seeded synthetic inputs follow the stated recipe: uniform reference with
repeat families at a target coverage, reads with uniform starts and strands,
the stated length distributions and error rates, and bit-for-bit determinism.
CPU only; small samples with tolerances of several standard errors."""
import math

import numpy as np
import pytest

from paper_2211_08157_gb300 import synth


def test_reference_is_uniform_and_deterministic():
    ref = synth.reference(1_000_000, 17)
    freq = np.bincount(ref, minlength=256)[synth.ACGT] / ref.size
    assert np.all(np.abs(freq - 0.25) < 0.003)            # sd of a fraction: 0.0004
    assert np.array_equal(ref, synth.reference(1_000_000, 17))
    assert not np.array_equal(ref, synth.reference(1_000_000, 18))
    assert set(np.unique(ref).tolist()) <= set(synth.ACGT.tolist())


def _dup_kmers(seq: np.ndarray, k: int) -> int:
    codes = np.searchsorted(synth.ACGT, seq).astype(np.uint64)
    v = np.zeros(seq.size - k + 1, dtype=np.uint64)
    for i in range(k):
        v = (v << np.uint64(2)) | codes[i:i + v.size]
    _, cnt = np.unique(v, return_counts=True)
    return int((cnt - 1).sum())


def test_repeat_families_cover_the_target_and_duplicate_kmers():
    L = 2_000_000
    rep = synth.RepeatModel(20, 1000, 6000, False, 0.02, 0.02, 0.05)
    plain = synth.reference(L, 21)
    ref = synth.reference(L, 21, rep)
    changed = np.count_nonzero(ref != plain) / L
    # copies overwrite >= 5 % of the bases, three quarters of which differ from the iid base
    assert 0.75 * 0.05 * 0.9 < changed < 0.75 * 0.05 * 1.6
    # copies of a family (2 % divergent, same orientation) share most of their 21-mers; iid
    # bases share almost none
    assert _dup_kmers(plain, 21) < 10
    assert _dup_kmers(ref, 21) > 2000


def test_short_reads_uniform_starts_strands_and_substitution_rate():
    ref = synth.reference(500_000, 31)
    n = 20_000
    reads, offs, truth = synth.reads(ref, n, synth.SHORT, synth.ErrorModel(0.001, 1, 0, 0), 31)
    assert np.array_equal(offs, np.arange(n + 1, dtype=np.uint64) * 150)
    st, sd = truth["start"], truth["strand"]
    assert abs(sd.mean() - 0.5) < 0.015                   # sd 0.0035
    assert abs(st.mean() / (ref.size - 150) - 0.5) < 0.01  # sd 0.002
    tpl = ref[st[:, None] + np.arange(150)[None, :]]
    rc = sd == 1
    tpl[rc] = synth.revcomp(tpl[rc].reshape(-1)).reshape(-1, 150)[::-1]
    diff = np.count_nonzero(reads.reshape(n, 150) != tpl)
    assert abs(diff - 0.001 * n * 150) < 5 * math.sqrt(0.001 * n * 150)   # binomial, 3000 expected


@pytest.mark.parametrize("sub,ins,dele", [(1, 0, 0), (0, 1, 0), (0, 0, 1)])
def test_error_model_rates_by_kind(sub, ins, dele):
    rng = np.random.default_rng(5)
    tpl = synth.ACGT[rng.integers(0, 4, 400_000)]
    rate = 0.08
    out = synth._mutate_one(tpl, synth.ErrorModel(rate, sub, ins, dele), rng)
    exp, sdv = rate * tpl.size, math.sqrt(rate * (1 - rate) * tpl.size)
    if sub:
        assert out.size == tpl.size
        d = np.count_nonzero(out != tpl)                   # a substitution never keeps the base
        assert abs(d - exp) < 5 * sdv
    elif ins:
        assert abs((out.size - tpl.size) - exp) < 5 * sdv
    else:
        assert abs((tpl.size - out.size) - exp) < 5 * sdv


def test_hifi_lengths_mean_15kb_sd_4kb():
    rng = np.random.default_rng(7)
    lens = synth._lengths(40_000, synth.HIFI, rng)
    assert lens.min() >= 2000 and lens.max() <= 30000
    assert abs(lens.mean() / 15_000 - 1) < 0.01
    assert abs(lens.std() / 4_000 - 1) < 0.04


def test_ont_lengths_truncated_mean_10kb():
    m = synth.ONT
    assert (m.lo, m.hi, m.sigma) == (500, 100_000, synth.ONT_SIGMA)
    # the sigma is the paper's ONT mean/median ratio: median e^mu, mean e^(mu + sigma^2 / 2)
    assert abs(math.exp(m.sigma ** 2 / 2) - 15806.4 / 5045) < 0.01
    lens = synth._lengths(200_000, m, np.random.default_rng(9))
    assert lens.min() >= 500 and lens.max() <= 100_000
    assert abs(lens.mean() / 10_000 - 1) < 0.02           # sd of the mean ~ 0.5 %


def test_reads_are_deterministic_per_seed():
    ref = synth.reference(200_000, 41)
    a = synth.reads(ref, 500, synth.SHORT, synth.ILLUMINA_INDEL, 41)
    b = synth.reads(ref, 500, synth.SHORT, synth.ILLUMINA_INDEL, 41)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    c = synth.reads(ref, 500, synth.SHORT, synth.ILLUMINA_INDEL, 42)
    assert not np.array_equal(a[0][:1000], c[0][:1000])
