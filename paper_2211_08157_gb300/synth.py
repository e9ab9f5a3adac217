"""Seeded synthetic genomes and reads (inputs only; none of the method's arithmetic).

Stand-ins for the paper's data (GRCh38 and GIAB HG002 Illumina / HiFi / ONT reads,
Sec. 2.2), which are not available here. Every array is a deterministic function
of its seed: ``numpy.random.Generator(PCG64(seed))`` with
``seed = 1000 * config + stream`` (stream 0 = reference bases, 1 = repeats,
2 = reads), so the same call gives the same bytes on any machine with the same
numpy major version.

* Reference: iid uniform ACGT, then copies of repeat families written over it
  until a target fraction of bases is covered. Each copy has its own orientation
  and iid substitutions at a per-copy divergence.
* Reads: start uniform over the reference, strand 50/50 (reverse complement),
  then per-base errors: substitution = one of the other three bases uniformly,
  insertion = a uniform random base before the template base, deletion = drop
  the template base. A truth record keeps (start, strand, template length).

Sizes, rates and length models of the five workloads live in ``WORKLOADS``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ACGT = np.frombuffer(b"ACGT", dtype=np.uint8)
_COMP = np.zeros(256, dtype=np.uint8)
for _a, _b in zip(b"ACGTNacgtn", b"TGCANtgcan"):
    _COMP[_a] = _b


def rng_for(config: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(1000 * config + stream))


def revcomp(seq: np.ndarray) -> np.ndarray:
    return _COMP[seq[::-1]]


# --------------------------------------------------------------------------- reference
@dataclass
class RepeatModel:
    families: int
    len_lo: int
    len_hi: int
    log_uniform: bool         # family length log-uniform instead of uniform
    div_lo: float             # per-copy substitution divergence ~ U[div_lo, div_hi]
    div_hi: float
    coverage: float           # stop once this fraction of bases has been written


def _substitute(seq: np.ndarray, rate: float, rng: np.random.Generator) -> np.ndarray:
    """Copy of seq (ASCII ACGT) with iid substitutions to one of the other 3 bases."""
    out = seq.copy()
    n = out.size
    if n == 0 or rate <= 0:
        return out
    cnt = rng.binomial(n, rate)
    if cnt == 0:
        return out
    where = np.unique(rng.integers(0, n, cnt))
    code = np.searchsorted(ACGT, out[where])            # 0..3 for ACGT
    shift = rng.integers(1, 4, where.size)
    out[where] = ACGT[(code + shift) & 3]
    return out


def reference(length: int, config: int, repeats: RepeatModel | None = None) -> np.ndarray:
    """Seeded uniform ACGT reference with optional repeat families (uint8 ASCII)."""
    rng = rng_for(config, 0)
    ref = np.empty(length, dtype=np.uint8)
    chunk = 1 << 26
    for s in range(0, length, chunk):
        e = min(length, s + chunk)
        ref[s:e] = ACGT[rng.integers(0, 4, e - s, dtype=np.uint8)]
    if repeats is None or repeats.coverage <= 0:
        return ref
    rr = rng_for(config, 1)
    if repeats.log_uniform:
        lens = np.exp(rr.uniform(math.log(repeats.len_lo), math.log(repeats.len_hi), repeats.families))
    else:
        lens = rr.uniform(repeats.len_lo, repeats.len_hi + 1, repeats.families)
    lens = np.minimum(lens.astype(np.int64), length)
    fams = [ACGT[rr.integers(0, 4, int(L), dtype=np.uint8)] for L in lens]
    target = int(repeats.coverage * length)
    written = 0
    while written < target:
        f = int(rr.integers(0, repeats.families))
        src = fams[f]
        L = src.size
        start = int(rr.integers(0, length - L + 1))
        div = float(rr.uniform(repeats.div_lo, repeats.div_hi))
        copy = _substitute(src, div, rr)
        if rr.integers(0, 2):
            copy = revcomp(copy)
        ref[start:start + L] = copy
        written += L
    return ref


# --------------------------------------------------------------------------- reads
@dataclass
class ErrorModel:
    rate: float               # total per-template-base error rate
    sub: float                # relative weights of substitution : insertion : deletion
    ins: float
    dele: float


@dataclass
class LengthModel:
    kind: str                 # "fixed" or "lognormal"
    fixed: int = 150
    mu: float = 0.0
    sigma: float = 0.0
    lo: int = 0
    hi: int = 0


def lognormal_mu_for_mean(mean: float, sigma: float, lo: float, hi: float) -> float:
    """mu such that a lognormal(mu, sigma) truncated to [lo, hi] has the given mean."""
    def phi(v):
        return 0.5 * (1.0 + math.erf(v / math.sqrt(2.0)))

    def tmean(mu):
        a, b = math.log(lo), math.log(hi)
        num = phi((b - mu - sigma * sigma) / sigma) - phi((a - mu - sigma * sigma) / sigma)
        den = phi((b - mu) / sigma) - phi((a - mu) / sigma)
        return math.exp(mu + sigma * sigma / 2) * num / den

    lo_mu, hi_mu = math.log(lo) - 5, math.log(hi) + 5
    for _ in range(200):
        mid = 0.5 * (lo_mu + hi_mu)
        if tmean(mid) < mean:
            lo_mu = mid
        else:
            hi_mu = mid
    return 0.5 * (lo_mu + hi_mu)


def _lengths(n: int, model: LengthModel, rng: np.random.Generator) -> np.ndarray:
    if model.kind == "fixed":
        return np.full(n, model.fixed, dtype=np.int64)
    out = np.empty(n, dtype=np.int64)
    todo = np.arange(n)
    while todo.size:
        v = rng.lognormal(model.mu, model.sigma, todo.size)
        ok = (v >= model.lo) & (v <= model.hi)
        out[todo[ok]] = np.rint(v[ok]).astype(np.int64)
        todo = todo[~ok]
    return out


def _mutate_one(tpl: np.ndarray, em: ErrorModel, rng: np.random.Generator) -> np.ndarray:
    """Apply substitutions, insertions and deletions to one template (ASCII)."""
    n = tpl.size
    tot = em.sub + em.ins + em.dele
    u = rng.random(n)
    ev = np.zeros(n, dtype=np.int8)                      # 0 none, 1 sub, 2 ins, 3 del
    hit = u < em.rate
    if not hit.any():
        return tpl.copy()
    r = u[hit] / em.rate * tot
    ev[hit] = np.where(r < em.sub, 1, np.where(r < em.sub + em.ins, 2, 3))
    base = tpl.copy()
    subs = np.nonzero(ev == 1)[0]
    if subs.size:
        code = np.searchsorted(ACGT, base[subs])
        base[subs] = ACGT[(code + rng.integers(1, 4, subs.size)) & 3]
    reps = np.where(ev == 3, 0, np.where(ev == 2, 2, 1))
    out = np.repeat(base, reps)
    ins_idx = np.nonzero(ev == 2)[0]
    if ins_idx.size:
        # position of the inserted base = first output slot of that template base
        first = np.cumsum(reps) - reps
        out[first[ins_idx]] = ACGT[rng.integers(0, 4, ins_idx.size)]
    return out


def reads(ref: np.ndarray, n: int, lengths: LengthModel, errors: ErrorModel, config: int,
          rng: np.random.Generator | None = None):
    """n reads: (concatenated ASCII bytes, uint64 CSR offsets [n + 1], truth dict)."""
    rng = rng if rng is not None else rng_for(config, 2)
    L = ref.size
    tl = np.minimum(_lengths(n, lengths, rng), L)
    starts = (rng.random(n) * (L - tl + 1)).astype(np.int64)
    strands = rng.integers(0, 2, n).astype(np.uint8)
    indel_w = (errors.ins + errors.dele) / max(errors.sub + errors.ins + errors.dele, 1e-30)
    per_read_indel = errors.rate * indel_w
    parts = []
    # Substitution-only or rare-indel reads go through one vectorised pass per
    # chunk; reads that draw an indel are rebuilt one by one.
    if lengths.kind == "fixed" and per_read_indel * lengths.fixed < 0.05:
        m = lengths.fixed
        out = np.empty(n * m, dtype=np.uint8)
        chunk = 1 << 17
        for s in range(0, n, chunk):
            e = min(n, s + chunk)
            idx = starts[s:e, None] + np.arange(m)[None, :]
            blk = ref[idx]
            rc = strands[s:e] == 1
            blk[rc] = _COMP[blk[rc][:, ::-1]]
            out[s * m:e * m] = blk.reshape(-1)
        sub_rate = errors.rate * errors.sub / (errors.sub + errors.ins + errors.dele)
        out = _substitute(out, sub_rate, rng)
        if per_read_indel > 0:
            k_ev = rng.binomial(n * m, per_read_indel)
            hit_reads = np.unique(rng.integers(0, n, k_ev))
        else:
            hit_reads = np.zeros(0, dtype=np.int64)
        seqs = out.reshape(n, m)
        ins_share = errors.ins / max(errors.ins + errors.dele, 1e-30)
        fixed = {}
        for r in hit_reads.tolist():
            s = seqs[r]
            p = int(rng.integers(0, m))
            if rng.random() < ins_share:
                s2 = np.concatenate([s[:p], ACGT[rng.integers(0, 4, 1)], s[p:]])
            else:
                s2 = np.concatenate([s[:p], s[p + 1:]])
            fixed[r] = s2
        if not fixed:
            offs = np.arange(n + 1, dtype=np.uint64) * m
            return out, offs, {"start": starts, "strand": strands, "tlen": tl}
        lens_out = np.full(n, m, dtype=np.int64)
        for r, s2 in fixed.items():
            lens_out[r] = s2.size
        offs = np.zeros(n + 1, dtype=np.uint64)
        offs[1:] = np.cumsum(lens_out)
        buf = np.empty(int(offs[-1]), dtype=np.uint8)
        # copy unchanged reads in runs between the rebuilt ones
        prev = 0
        for r in sorted(fixed):
            if r > prev:
                buf[int(offs[prev]):int(offs[r])] = seqs[prev:r].reshape(-1)
            buf[int(offs[r]):int(offs[r + 1])] = fixed[r]
            prev = r + 1
        if prev < n:
            buf[int(offs[prev]):] = seqs[prev:].reshape(-1)
        return buf, offs, {"start": starts, "strand": strands, "tlen": tl}
    for i in range(n):
        tpl = ref[starts[i]:starts[i] + tl[i]]
        if strands[i]:
            tpl = revcomp(tpl)
        parts.append(_mutate_one(tpl, errors, rng))
    lens_out = np.array([p.size for p in parts], dtype=np.int64)
    offs = np.zeros(n + 1, dtype=np.uint64)
    offs[1:] = np.cumsum(lens_out)
    buf = np.concatenate(parts) if parts else np.zeros(0, np.uint8)
    return buf, offs, {"start": starts, "strand": strands, "tlen": tl}


# --------------------------------------------------------------------------- workloads
SHORT = LengthModel("fixed", fixed=150)
HIFI = LengthModel("lognormal", mu=9.58146, sigma=0.26210, lo=2000, hi=30000)
ONT_SIGMA = 1.5113
ONT = LengthModel("lognormal", mu=lognormal_mu_for_mean(10000.0, ONT_SIGMA, 500, 100000),
                  sigma=ONT_SIGMA, lo=500, hi=100000)

ILLUMINA_SUB = ErrorModel(0.001, 1, 0, 0)
ILLUMINA_INDEL = ErrorModel(0.0011, 10, 0.5, 0.5)        # 0.1 % subs + 0.01 % 1-bp indels
HIFI_ERR = ErrorModel(0.001, 1, 2, 2)
ONT_ERR = ErrorModel(0.08, 1, 1, 1)

REP_100M = RepeatModel(200, 1000, 6000, False, 0.02, 0.02, 0.05)
REP_HUMAN = RepeatModel(1000, 300, 6000, True, 0.05, 0.15, 0.45)


@dataclass
class Workload:
    name: str
    config: int
    ref_len: int
    repeats: RepeatModel | None
    n_reads: int
    lengths: LengthModel
    errors: ErrorModel
    pattern: str
    k: int
    w: int
    max_occ: int
    t: int = 32
    ref_config: int = 0       # seed family of the reference (0 = own config)
    notes: str = ""
    extra: dict = field(default_factory=dict)

    def make_reference(self, ref_len: int | None = None) -> np.ndarray:
        return reference(ref_len or self.ref_len, self.ref_config or self.config, self.repeats)

    def make_reads(self, ref: np.ndarray, n: int | None = None, seed_stream: int = 2):
        return reads(ref, n if n is not None else self.n_reads, self.lengths, self.errors, self.config,
                     rng=rng_for(self.config, seed_stream))


WORKLOADS = {
    "tiny_1mbp_short": Workload("tiny_1mbp_short", 1, 1_000_000, None, 10_000, SHORT, ILLUMINA_SUB,
                                "10", 21, 11, 500),
    "short_100mbp_2m": Workload("short_100mbp_2m", 2, 100_000_000, REP_100M, 2_000_000, SHORT,
                                ILLUMINA_INDEL, "10", 21, 11, 500),
    "hifi_100mbp_200k": Workload("hifi_100mbp_200k", 3, 100_000_000, REP_100M, 200_000, HIFI, HIFI_ERR,
                                 "110", 19, 19, 500, ref_config=2),
    "ont_3100mbp_100k": Workload("ont_3100mbp_100k", 4, 3_100_000_000, REP_HUMAN, 100_000, ONT, ONT_ERR,
                                 "10", 15, 10, 1000),
}


def serving_requests(ref: np.ndarray, per_kind: int = 8, long_max: int = 2000, seed: int = 5):
    """Request payloads of the serving workload: short-read batches (1k-50k x
    150 bp, 0.1 % substitutions + 0.01 % 1-bp indels), HiFi-like and ONT-like
    long-read batches (10-long_max reads, the length and error models above);
    per_kind requests of each kind, as {kind: [(reads, offsets), ...]}."""
    rng = np.random.default_rng(seed)
    pool = {"short": [], "hifi": [], "ont": []}
    for i in range(per_kind):
        g = np.random.default_rng(seed * 100 + i)
        pool["short"].append(reads(ref, int(rng.integers(1000, 50001)), SHORT, ILLUMINA_INDEL, 0, rng=g)[:2])
        pool["hifi"].append(reads(ref, int(rng.integers(10, long_max + 1)), HIFI, HIFI_ERR, 0, rng=g)[:2])
        pool["ont"].append(reads(ref, int(rng.integers(10, long_max + 1)), ONT, ONT_ERR, 0, rng=g)[:2])
    return pool
