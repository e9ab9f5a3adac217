"""ctypes front-end of the plain C++ Genome-on-Diet oracle (``god_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers. The product package never
imports this module, and this module imports nothing from the product package.

Every function mirrors one step of the method (paper sections in the C++ file):
sparsification (Sec. 3, 3.2), the Wang integer hash (Sec. 3.6.1), (w,k)-minimizers
(Sec. 3.1), the filtered seed index (Sec. 3.1, 3.2), pattern alignment (Sec. 3.2),
compressed seeding to sorted anchors (Sec. 3.3), location voting with the rescue
location (Sec. 3.4, Sec. 3.6.3), containment search (Sec. 2.3), the seed matching
evaluation (Sec. 2.1.1), and the learned-index reference.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "god_oracle.cpp")
_LIB = os.path.join(_HERE, "libgod_oracle.so")
_lock = threading.Lock()
_lib = None

ANCHOR_DTYPE = np.dtype([("read_id", "<u4"), ("read_pos", "<u4"), ("ref_pos", "<u4"), ("strand", "<u4")])
VOTE_DTYPE = np.dtype([("read_id", "<u4"), ("votes", "<u4"), ("strand", "<u4"), ("rescue", "<u4"), ("loc", "<i8"),
                       ("ref_lo", "<u4"), ("ref_hi", "<u4"), ("read_lo", "<u4"), ("read_hi", "<u4")])


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/libgod_oracle.so`` (g++, -O2, no ISA flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
                               "-ffp-contract=off", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            p = C.c_void_p
            u64, i64, u32, i32 = C.c_uint64, C.c_int64, C.c_uint32, C.c_int
            L.orc_sparsify.restype = i64
            L.orc_sparsify.argtypes = [p, u64, C.c_char_p, u64, p, p, u64]
            L.orc_hash_array.restype = None
            L.orc_hash_array.argtypes = [p, u64, i32, p]
            L.orc_minimizers.restype = i64
            L.orc_minimizers.argtypes = [p, u64, C.c_char_p, u64, i32, i32, p, p, p, p, u64]
            L.orc_build_index.restype = p
            L.orc_build_index.argtypes = [p, u64, C.c_char_p, i32, i32, u32]
            L.orc_free_index.restype = None
            L.orc_free_index.argtypes = [p]
            L.orc_index_sizes.restype = None
            L.orc_index_sizes.argtypes = [p, p]
            L.orc_index_dump.restype = None
            L.orc_index_dump.argtypes = [p, p, p, p]
            L.orc_index_count.restype = None
            L.orc_index_count.argtypes = [p, p, u64, p]
            L.orc_pattern_align.restype = u32
            L.orc_pattern_align.argtypes = [p, p, u64, u32, p]
            L.orc_seed.restype = C.POINTER(C.c_uint32)
            L.orc_seed.argtypes = [p, p, p, u32, u32, i32, C.POINTER(u64), p]
            L.orc_seed_segments.restype = C.POINTER(C.c_uint32)
            L.orc_seed_segments.argtypes = [p, p, p, u32, u32, i32, u64, C.POINTER(u64), p]
            L.orc_vote.restype = i32
            L.orc_vote.argtypes = [p, u64, p, u32, u32, u32, u32, p, p]
            L.orc_contain.restype = i32
            L.orc_contain.argtypes = [p, p, u32, p, u32, p, p, u32, C.c_char_p, i32, i32, u32, u32, u32, u32, u64,
                                      i32, p, p, p, p]
            L.orc_seed_match.restype = i32
            L.orc_seed_match.argtypes = [p, p, u32, C.c_char_p, C.c_char_p, i32, i32, p, p, p]
            L.orc_free.restype = None
            L.orc_free.argtypes = [p]
            L.orc_root_loss_grad_f64.restype = C.c_double
            L.orc_root_loss_grad_f64.argtypes = [p, i32, p, p, u64, p]
            L.orc_root_loss_grad_f32.restype = C.c_float
            L.orc_root_loss_grad_f32.argtypes = [p, i32, p, p, u64, p]
            L.orc_root_route.restype = None
            L.orc_root_route.argtypes = [p, i32, p, u64, u64, C.c_float, u32, p, p]
            L.orc_rmi_fit_leaves.restype = None
            L.orc_rmi_fit_leaves.argtypes = [p, i32, p, u64, u64, C.c_float, u32, p, p, p, p]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _bytes(seq) -> np.ndarray:
    if isinstance(seq, (bytes, bytearray)):
        return np.frombuffer(bytes(seq), dtype=np.uint8)
    return np.ascontiguousarray(seq, dtype=np.uint8)


def sparsify(seq, pattern: str, shift: int = 0):
    """Kept 2-bit codes (4 = N) and their original indices (Sec. 3, 3.2)."""
    s = _bytes(seq)
    n = lib().orc_sparsify(_ptr(s), s.size, pattern.encode(), shift, None, None, 0)
    if n < 0:
        raise ValueError("bad pattern")
    codes = np.zeros(max(n, 1), np.uint8)
    orig = np.zeros(max(n, 1), np.uint64)
    lib().orc_sparsify(_ptr(s), s.size, pattern.encode(), shift, _ptr(codes), _ptr(orig), n)
    return codes[:n], orig[:n]


def wang_hash(x, k: int) -> np.ndarray:
    a = np.ascontiguousarray(x, dtype=np.uint64)
    out = np.empty_like(a)
    lib().orc_hash_array(_ptr(a), a.size, k, _ptr(out))
    return out


def minimizers(seq, pattern: str, shift: int, k: int, w: int):
    """(key, orig_pos, z, patterned_j) arrays in ascending patterned position."""
    s = _bytes(seq)
    n = lib().orc_minimizers(_ptr(s), s.size, pattern.encode(), shift, k, w, None, None, None, None, 0)
    if n < 0:
        raise ValueError("bad parameters")
    keys = np.zeros(max(n, 1), np.uint64)
    pos = np.zeros(max(n, 1), np.uint64)
    z = np.zeros(max(n, 1), np.uint32)
    j = np.zeros(max(n, 1), np.uint64)
    lib().orc_minimizers(_ptr(s), s.size, pattern.encode(), shift, k, w, _ptr(keys), _ptr(pos), _ptr(z), _ptr(j), n)
    return keys[:n], pos[:n], z[:n], j[:n]


class Index:
    """The oracle's filtered seed index (Sec. 3.1 step 3, Sec. 3.2 filter)."""

    def __init__(self, ref, pattern: str, k: int, w: int, max_occ: int):
        self._ref = _bytes(ref)
        self.pattern, self.k, self.w, self.max_occ = pattern, k, w, max_occ
        self.h = lib().orc_build_index(_ptr(self._ref), self._ref.size, pattern.encode(), k, w, max_occ)
        if not self.h:
            raise ValueError("bad index parameters")

    def close(self):
        if self.h:
            lib().orc_free_index(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sizes(self):
        out = np.zeros(3, np.uint64)
        lib().orc_index_sizes(self.h, _ptr(out))
        return int(out[0]), int(out[1]), int(out[2])

    def dump(self):
        """(kept keys ascending, CSR start offsets, entries (pos << 1 | z))."""
        _, nk, ne = self.sizes()
        keys = np.zeros(max(nk, 1), np.uint64)
        start = np.zeros(nk + 1, np.uint64)
        ent = np.zeros(max(ne, 1), np.uint64)
        lib().orc_index_dump(self.h, _ptr(keys), _ptr(start), _ptr(ent))
        return keys[:nk], start, ent[:ne]

    def count(self, keys) -> np.ndarray:
        k = np.ascontiguousarray(keys, dtype=np.uint64)
        out = np.zeros(k.size, np.uint64)
        lib().orc_index_count(self.h, _ptr(k), k.size, _ptr(out))
        return out

    def pattern_align(self, read, t: int):
        r = _bytes(read)
        sums = np.zeros(len(self.pattern), np.uint64)
        a = lib().orc_pattern_align(self.h, _ptr(r), r.size, t, _ptr(sums))
        return int(a), sums

    def seed(self, reads: np.ndarray, offsets: np.ndarray, t: int, threads: int = 1, seg_len: int = 0):
        """Sorted anchors (structured array) and the alignment indices: one per
        read, or with seg_len > 0 one per segment (reads longer than seg_len
        bases are seeded in segments of seg_len; read order, then segment)."""
        reads = _bytes(reads)
        offs = np.ascontiguousarray(offsets, dtype=np.uint64)
        n = offs.size - 1
        lens = np.diff(offs)
        nseg = np.where((seg_len > 0) & (lens > seg_len), (lens + max(seg_len, 1) - 1) // max(seg_len, 1), 1)
        n_sh = int(nseg.sum()) if n else 0
        shifts = np.zeros(max(n_sh, 1), np.uint32)
        cnt = C.c_uint64(0)
        buf = lib().orc_seed_segments(self.h, _ptr(reads), _ptr(offs), n, t, threads, seg_len, C.byref(cnt),
                                      _ptr(shifts))
        m = int(cnt.value)
        arr = np.ctypeslib.as_array(buf, shape=(max(m, 1) * 4,))[: m * 4].copy()
        lib().orc_free(C.cast(buf, C.c_void_p))
        return arr.view(ANCHOR_DTYPE), shifts[:n_sh]


def vote(anchors, offsets, D: int, V: int, max_out: int):
    """Location voting (Sec. 3.4, Sec. 3.6.3) over an anchor list grouped by
    ascending read id. Returns (records of every read in read order, as
    VOTE_DTYPE, and the per-read record counts)."""
    a = np.ascontiguousarray(np.asarray(anchors).view(np.uint32).reshape(-1, 4))
    offs = np.ascontiguousarray(offsets, dtype=np.uint64)
    n = offs.size - 1
    out = np.zeros(max(n * max_out, 1), VOTE_DTYPE)
    counts = np.zeros(max(n, 1), np.uint32)
    rc = lib().orc_vote(_ptr(a), a.shape[0], _ptr(offs), n, D, V, max_out, _ptr(out), _ptr(counts))
    if rc != 0:
        raise ValueError("anchors must be grouped by ascending read id < number of reads")
    counts = counts[:n]
    keep = (np.arange(max_out)[None, :] < counts[:, None]).reshape(-1)
    return out[: n * max_out][keep], counts


def contain(db, contig_offsets, contig_genome, n_genomes: int, reads, read_offsets, pattern: str, k: int, w: int,
            max_occ: int, t: int, D: int, V: int, batch_bases: int, threads: int = 1):
    """Containment search (Sec. 2.3): (read genome (-1 = unmapped), read votes,
    genome mapped reads, genome mapped read bases)."""
    dbb = _bytes(db)
    co = np.ascontiguousarray(contig_offsets, dtype=np.uint64)
    cg = np.ascontiguousarray(contig_genome, dtype=np.uint32)
    rb = _bytes(reads)
    ro = np.ascontiguousarray(read_offsets, dtype=np.uint64)
    nr = ro.size - 1
    rg = np.zeros(max(nr, 1), np.int32)
    rv = np.zeros(max(nr, 1), np.uint32)
    gr = np.zeros(max(n_genomes, 1), np.uint64)
    gb = np.zeros(max(n_genomes, 1), np.uint64)
    rc = lib().orc_contain(_ptr(dbb), _ptr(co), co.size - 1, _ptr(cg), n_genomes, _ptr(rb), _ptr(ro), nr,
                           pattern.encode(), k, w, max_occ, t, D, V, batch_bases, threads, _ptr(rg), _ptr(rv),
                           _ptr(gr), _ptr(gb))
    if rc != 0:
        raise ValueError("bad pattern or genome id")
    return rg[:nr], rv[:nr], gr[:n_genomes], gb[:n_genomes]


SEED_KINDS = ("all", "minimizer", "spaced", "god")


def seed_match(seqs, offsets, pattern: str, spaced: str, k: int, w: int):
    """Seed matching evaluation (Sec. 2.1.1): pair i = (seq 2i, seq 2i + 1).
    Returns (Levenshtein distance [n], matched [n, 4], total [n, 4]) with the
    columns in SEED_KINDS order."""
    sb = _bytes(seqs)
    so = np.ascontiguousarray(offsets, dtype=np.uint64)
    n = (so.size - 1) // 2
    ed = np.zeros(max(n, 1), np.uint32)
    mt = np.zeros((max(n, 1), 4), np.uint32)
    tt = np.zeros((max(n, 1), 4), np.uint32)
    rc = lib().orc_seed_match(_ptr(sb), _ptr(so), n, pattern.encode(), spaced.encode(), k, w, _ptr(ed), _ptr(mt),
                              _ptr(tt))
    if rc != 0:
        raise ValueError("bad pattern, k or w")
    return ed[:n], mt[:n], tt[:n]


def root_loss_grad_f64(theta: np.ndarray, H: int, x: np.ndarray, y: np.ndarray):
    th = np.ascontiguousarray(theta, np.float64)
    xs = np.ascontiguousarray(x, np.float64)
    ys = np.ascontiguousarray(y, np.float64)
    g = np.zeros(3 * H + 1, np.float64)
    loss = lib().orc_root_loss_grad_f64(_ptr(th), H, _ptr(xs), _ptr(ys), xs.size, _ptr(g))
    return float(loss), g


def root_loss_grad_f32(theta: np.ndarray, H: int, x: np.ndarray, y: np.ndarray):
    th = np.ascontiguousarray(theta, np.float32)
    xs = np.ascontiguousarray(x, np.float32)
    ys = np.ascontiguousarray(y, np.float32)
    g = np.zeros(3 * H + 1, np.float32)
    loss = lib().orc_root_loss_grad_f32(_ptr(th), H, _ptr(xs), _ptr(ys), xs.size, _ptr(g))
    return float(loss), g


def root_route(theta: np.ndarray, H: int, keys: np.ndarray, kmin: int, inv_span: float, n_leaves: int):
    th = np.ascontiguousarray(theta, np.float32)
    k = np.ascontiguousarray(keys, np.uint64)
    x = np.zeros(k.size, np.float32)
    leaf = np.zeros(k.size, np.uint32)
    lib().orc_root_route(_ptr(th), H, _ptr(k), k.size, kmin, inv_span, n_leaves, _ptr(x), _ptr(leaf))
    return x, leaf


def rmi_fit_leaves(theta: np.ndarray, H: int, keys: np.ndarray, kmin: int, inv_span: float, n_leaves: int):
    th = np.ascontiguousarray(theta, np.float32)
    k = np.ascontiguousarray(keys, np.uint64)
    slope = np.zeros(n_leaves, np.float32)
    icept = np.zeros(n_leaves, np.float32)
    base = np.zeros(n_leaves, np.uint64)
    eps = np.zeros(n_leaves, np.uint32)
    lib().orc_rmi_fit_leaves(_ptr(th), H, _ptr(k), k.size, kmin, inv_span, n_leaves,
                             _ptr(slope), _ptr(icept), _ptr(base), _ptr(eps))
    return slope, icept, base, eps
