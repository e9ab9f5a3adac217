"""GB300-native Genome-on-Diet seeding (arXiv 2211.08157): Python binding.

A thin ctypes layer over ``libgod.so`` whose functions carry the C ABI's names
(include/god.h) and only marshal arguments: every step of the path runs in the
library's CUDA kernels. Host inputs are numpy arrays (or bytes); device inputs
are torch CUDA tensors (PyTorch provides device memory and streams only).
There is no CPU fallback: a missing or unloadable library raises.
"""
from __future__ import annotations

import ctypes as C
import weakref

import numpy as np

from . import _lib
from ._lib import (ContainParams, GodError, IndexInfo, Params, SeedOpts, ServerConfig, ServerStats, VoteParams,
                   build, check, load)

ANCHOR_DTYPE = np.dtype([("read_id", "<u4"), ("read_pos", "<u4"), ("ref_pos", "<u4"), ("strand", "<u4")])
VOTE_DTYPE = np.dtype([("read_id", "<u4"), ("votes", "<u4"), ("strand", "<u4"), ("rescue", "<u4"), ("loc", "<i8"),
                       ("ref_lo", "<u4"), ("ref_hi", "<u4"), ("read_lo", "<u4"), ("read_hi", "<u4")])

GOD_INDEX_HASH, GOD_INDEX_LEARNED = 0, 1
GOD_ROOT_MLP, GOD_ROOT_UNTRAINED, GOD_ROOT_LINEAR = 0, 1, 2


def _ptr(x):
    """Address of a numpy array, bytes object or torch tensor."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported buffer {type(x)}")


def _u8(x):
    if isinstance(x, (bytes, bytearray)):
        return np.frombuffer(bytes(x), dtype=np.uint8)
    return x


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def god_params_init(**overrides) -> Params:
    p = Params()
    load().god_params_init(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


class GodIndex:
    """Owns a ``god_index*``; released with god_free when closed or collected."""

    def __init__(self, handle: int):
        self.h = C.c_void_p(handle)

    def close(self):
        if self.h and self.h.value:
            load().god_free(self.h)
            self.h = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def info(self) -> dict:
        return god_index_get_info(self)


def god_build_index(ref, pattern: str, k: int, w: int, max_occ: int, params: Params | None = None,
                    stream=None) -> GodIndex:
    ref = _u8(ref)
    n = ref.size if isinstance(ref, np.ndarray) else ref.numel()
    out = C.c_void_p()
    L = load()
    if params is None:
        check(L.god_build_index(_ptr(ref), n, pattern.encode(), k, w, max_occ, C.byref(out)))
    else:
        check(L.god_build_index_ex(_ptr(ref), n, pattern.encode(), k, w, max_occ, C.byref(params),
                                   _stream_ptr(stream), C.byref(out)))
    return GodIndex(out.value)


def god_index_get_info(index: GodIndex) -> dict:
    info = IndexInfo()
    check(load().god_index_get_info(index.h, C.byref(info)))
    return {name: getattr(info, name) for name, _ in IndexInfo._fields_}


def god_index_export(index: GodIndex):
    info = god_index_get_info(index)
    keys = np.zeros(max(info["n_keys"], 1), np.uint64)
    start = np.zeros(info["n_keys"] + 1, np.uint64)
    ent = np.zeros(max(info["n_entries"], 1), np.uint64)
    check(load().god_index_export(index.h, _ptr(keys), _ptr(start), _ptr(ent)))
    return keys[: info["n_keys"]], start, ent[: info["n_entries"]]


def god_index_lookup(index: GodIndex, keys, via: int = 0, stream=None):
    keys = np.ascontiguousarray(keys, dtype=np.uint64) if isinstance(keys, (np.ndarray, list)) else keys
    n = keys.size if isinstance(keys, np.ndarray) else keys.numel()
    if isinstance(keys, np.ndarray):
        count = np.zeros(n, np.uint32)
        first = np.zeros(n, np.uint64)
    else:
        import torch
        count = torch.zeros(n, dtype=torch.int32, device=keys.device)
        first = torch.zeros(n, dtype=torch.int64, device=keys.device)
    check(load().god_index_lookup(index.h, _ptr(keys), n, via, _ptr(count), _ptr(first), _stream_ptr(stream)))
    return count, first


def _opts(stream=None, pa_t=None, via=None, shifts_out=None, seg_len=None) -> SeedOpts:
    o = SeedOpts()
    load().god_seed_opts_init(C.byref(o))
    o.stream = _stream_ptr(stream)
    if seg_len is not None:
        o.seg_len = seg_len
    if pa_t is not None:
        o.pa_t = pa_t
    if via is not None:
        o.via = via
    o.shifts_out = _ptr(shifts_out)
    return o


def _owned_anchors(ptr: C.c_void_p, m: int) -> np.ndarray:
    """Anchor array over a library-allocated host buffer (no copy); the buffer
    goes back through god_free when the last numpy view of it is released."""
    L = load()
    if not m:
        L.god_free(ptr)
        return np.zeros(0, np.uint32).view(ANCHOR_DTYPE)
    buf = (C.c_uint32 * (4 * m)).from_address(ptr.value)
    weakref.finalize(buf, L.god_free, C.c_void_p(ptr.value))
    return np.frombuffer(buf, dtype=np.uint32).view(ANCHOR_DTYPE)


def god_seed(index: GodIndex, reads, offsets):
    """Sorted anchors of a read batch (host numpy arrays in, structured array out)."""
    reads = _u8(reads)
    offs = np.ascontiguousarray(offsets, dtype=np.uint64) if isinstance(offsets, np.ndarray) else offsets
    n = (offs.size if isinstance(offs, np.ndarray) else offs.numel()) - 1
    ptr = C.c_void_p()
    cnt = C.c_uint64()
    L = load()
    check(L.god_seed(index.h, _ptr(reads), _ptr(offs), n, C.byref(ptr), C.byref(cnt)))
    return _owned_anchors(ptr, cnt.value)


def god_seed_into(index: GodIndex, reads, offsets, out, stream=None, pa_t=None, via=None, shifts_out=None,
                  seg_len=None) -> int:
    """Anchors written into `out` (host numpy or device tensor of 16-byte rows); returns the count.
    Raises GodError(rc=GOD_ERANGE) with the needed count when `out` is too small."""
    reads = _u8(reads)
    n = (offsets.size if isinstance(offsets, np.ndarray) else offsets.numel()) - 1
    cap = (out.nbytes if isinstance(out, np.ndarray) else out.numel() * out.element_size()) // 16
    cnt = C.c_uint64()
    o = _opts(stream, pa_t, via, shifts_out, seg_len)
    rc = load().god_seed_into(index.h, _ptr(reads), _ptr(offsets), n, _ptr(out), cap, C.byref(cnt), C.byref(o))
    if rc == -5:
        err = GodError(rc, f"output holds {cap} anchors, {cnt.value} needed")
        err.needed = cnt.value
        raise err
    check(rc)
    return cnt.value


def god_seed_device(index: GodIndex, d_reads, d_offsets, stream=None, pa_t=None, via=None, shifts_out=None,
                    seg_len=None):
    """Device inputs (torch CUDA tensors) -> (device pointer, count); free with god_free."""
    n = d_offsets.numel() - 1
    ptr = C.c_void_p()
    cnt = C.c_uint64()
    o = _opts(stream, pa_t, via, shifts_out, seg_len)
    check(load().god_seed_device(index.h, _ptr(d_reads), _ptr(d_offsets), n, C.byref(ptr), C.byref(cnt),
                                 C.byref(o)))
    return ptr.value, cnt.value


def god_sketch(seq, pattern: str, shift: int, k: int, w: int, stream=None):
    """(keys, original positions, z) of the minimizers of one sequence."""
    seq = _u8(seq)
    n = seq.size if isinstance(seq, np.ndarray) else seq.numel()
    cnt = C.c_uint64()
    L = load()
    rc = L.god_sketch(_ptr(seq), n, pattern.encode(), shift, k, w, None, None, None, 0, C.byref(cnt),
                      _stream_ptr(stream))
    if rc not in (0, -5):
        check(rc)
    m = cnt.value
    keys = np.zeros(max(m, 1), np.uint64)
    pos = np.zeros(max(m, 1), np.uint32)
    z = np.zeros(max(m, 1), np.uint8)
    check(L.god_sketch(_ptr(seq), n, pattern.encode(), shift, k, w, _ptr(keys), _ptr(pos), _ptr(z), m,
                       C.byref(cnt), _stream_ptr(stream)))
    return keys[:m], pos[:m], z[:m]


def _numel(x):
    return x.size if isinstance(x, np.ndarray) else x.numel()


def god_vote(anchors, offsets, D: int, V: int, max_out: int, out=None, counts=None, stream=None):
    """Location voting (god_vote) over an anchor list grouped by read id.

    Host inputs without `out`: returns (records of every read in read order as
    VOTE_DTYPE, per-read counts). With `out` (n_reads * max_out records: a
    numpy VOTE_DTYPE array or a device tensor of 40-byte rows) and `counts`,
    fills them in place and returns None. `n_anchors` comes from `anchors`
    (structured numpy array, (m, 4) array or tensor); a (ptr, m) pair of a
    device anchor list is accepted too."""
    if isinstance(anchors, tuple):
        a_ptr, m = anchors
    else:
        a_ptr = _ptr(anchors)
        m = _numel(anchors) if (isinstance(anchors, np.ndarray) and anchors.dtype.names) else _numel(anchors) // 4
    n = _numel(offsets) - 1
    prm = VoteParams(D, V, max_out)
    L = load()
    if out is not None:
        check(L.god_vote(a_ptr, m, _ptr(offsets), n, C.byref(prm), _ptr(out), _ptr(counts), _stream_ptr(stream)))
        return None
    rec = np.zeros(max(n * max_out, 1), VOTE_DTYPE)
    cnt = np.zeros(max(n, 1), np.uint32)
    check(L.god_vote(a_ptr, m, _ptr(offsets), n, C.byref(prm), _ptr(rec), _ptr(cnt), _stream_ptr(stream)))
    cnt = cnt[:n]
    keep = (np.arange(max_out)[None, :] < cnt[:, None]).reshape(-1)
    return rec[: n * max_out][keep], cnt


def god_contain(db, contig_offsets, contig_genome, n_genomes: int, reads, read_offsets, pattern: str = "10",
                k: int = 28, w: int = 40, max_occ: int = 1000, pa_t: int = 32, D: int = 100, V: int = 3,
                batch_bases: int = (1 << 32) - 1, index_kind: int = GOD_INDEX_HASH, stream=None):
    """Containment search (god_contain): (read genome (-1 = unmapped), read
    votes, genome mapped reads, genome mapped read bases)."""
    L = load()
    prm = ContainParams()
    L.god_contain_params_init(C.byref(prm))
    pat = pattern.encode()
    prm.pattern, prm.k, prm.w, prm.max_occ, prm.pa_t = pat, k, w, max_occ, pa_t
    prm.D, prm.V, prm.batch_bases, prm.index_kind = D, V, batch_bases, index_kind
    db = _u8(db)
    co = np.ascontiguousarray(contig_offsets, dtype=np.uint64)
    cg = np.ascontiguousarray(contig_genome, dtype=np.uint32)
    reads = _u8(reads)
    nr = _numel(read_offsets) - 1
    rg = np.zeros(max(nr, 1), np.int32)
    rv = np.zeros(max(nr, 1), np.uint32)
    gr = np.zeros(max(n_genomes, 1), np.uint64)
    gb = np.zeros(max(n_genomes, 1), np.uint64)
    check(L.god_contain(_ptr(db), _ptr(co), co.size - 1, _ptr(cg), n_genomes, _ptr(reads), _ptr(read_offsets), nr,
                        C.byref(prm), _ptr(rg), _ptr(rv), _ptr(gr), _ptr(gb), _stream_ptr(stream)))
    return rg[:nr], rv[:nr], gr[:n_genomes], gb[:n_genomes]


def god_seed_match(seqs, offsets, pattern: str, spaced: str, k: int, w: int, stream=None):
    """Seed matching evaluation (god_seed_match) of host pairs: (Levenshtein
    distance [n], matched [n, 4], total [n, 4]); columns All Seeds,
    Minimizers, Spaced, Genome-on-Diet."""
    seqs = _u8(seqs)
    offs = np.ascontiguousarray(offsets, dtype=np.uint64)
    n = (offs.size - 1) // 2
    ed = np.zeros(max(n, 1), np.uint32)
    mt = np.zeros((max(n, 1), 4), np.uint32)
    tt = np.zeros((max(n, 1), 4), np.uint32)
    check(load().god_seed_match(_ptr(seqs), _ptr(offs), n, pattern.encode(), spaced.encode(), k, w, _ptr(ed),
                                _ptr(mt), _ptr(tt), _stream_ptr(stream)))
    return ed[:n], mt[:n], tt[:n]


def god_rmi_root_grad(theta, H: int, x, y):
    th = np.ascontiguousarray(theta, np.float32)
    xs = np.ascontiguousarray(x, np.float32)
    ys = np.ascontiguousarray(y, np.float32)
    g = np.zeros(3 * H + 1, np.float32)
    loss = np.zeros(1, np.float32)
    check(load().god_rmi_root_grad(_ptr(th), H, _ptr(xs), _ptr(ys), xs.size, _ptr(g), _ptr(loss)))
    return float(loss[0]), g


def god_free(ptr):
    load().god_free(C.c_void_p(ptr) if isinstance(ptr, int) else ptr)


def god_launch_count() -> int:
    return int(load().god_launch_count())


def god_prof_enable(on: bool = True):
    load().god_prof_enable(1 if on else 0)


def god_set_graphs(on: bool = True):
    load().god_set_graphs(1 if on else 0)


def god_autotune_report() -> list:
    """Launch shapes chosen by the sketch autotuner so far."""
    import json
    L = load()
    need = L.god_autotune_report(None, 0)
    buf = C.create_string_buffer(max(need, 2) + 64)
    if L.god_autotune_report(buf, len(buf)) != 0:
        raise RuntimeError("autotune report buffer too small")
    return json.loads(buf.value.decode())


def god_prof_reset():
    load().god_prof_reset()


def god_prof_report() -> dict:
    """{kernel name: (launches, total ms, algorithmic bytes, units)} timed with CUDA events."""
    import json
    L = load()
    need = L.god_prof_report(None, 0)
    buf = C.create_string_buffer(max(need, 2) + 64)
    rc = L.god_prof_report(buf, len(buf))
    if rc != 0:
        raise RuntimeError("profile report buffer too small")
    return {k: (int(v[0]), float(v[1]), float(v[2]), float(v[3])) for k, v in json.loads(buf.value.decode()).items()}


def god_prof_timeline() -> list:
    """Timed launches as [(kernel, stream number, start ms, end ms)]."""
    import json
    L = load()
    need = L.god_prof_timeline(None, 0)
    buf = C.create_string_buffer(max(need, 2) + 64)
    rc = L.god_prof_timeline(buf, len(buf))
    if rc != 0:
        raise RuntimeError("profile timeline buffer too small")
    return [(k, int(s), float(a), float(b)) for k, s, a, b in json.loads(buf.value.decode())]


# ---------------------------------------------------------------- serving
class GodServer:
    def __init__(self, index: GodIndex, slots: int = 4, mem_budget: int = 0, max_batch_bases: int = 0):
        L = load()
        cfg = ServerConfig()
        L.god_server_config_init(C.byref(cfg))
        cfg.slots = slots
        if mem_budget:
            cfg.mem_budget = mem_budget
        if max_batch_bases:
            cfg.max_batch_bases = max_batch_bases
        h = C.c_void_p()
        check(L.god_server_create(index.h, C.byref(cfg), C.byref(h)))
        self.h = h
        self.index = index
        self._held = {}   # request id -> the arrays the server reads from until its wait returns

    def submit(self, reads, offsets) -> int:
        reads = _u8(reads)
        offs = np.ascontiguousarray(offsets, dtype=np.uint64)
        rid = C.c_uint64()
        check(load().god_server_submit(self.h, _ptr(reads), _ptr(offs), offs.size - 1, C.byref(rid)))
        self._held[rid.value] = (reads, offs)
        return rid.value

    def wait(self, request_id: int, timeout_ms: int = -1, with_latency: bool = False):
        ptr = C.c_void_p()
        cnt = C.c_uint64()
        lat = C.c_double()
        L = load()
        rc = L.god_server_wait(self.h, request_id, timeout_ms, C.byref(ptr), C.byref(cnt), C.byref(lat))
        if rc == -6:
            return None
        self._held.pop(request_id, None)
        check(rc)
        arr = _owned_anchors(ptr, cnt.value)
        if with_latency:
            return arr, lat.value
        return arr

    def stats(self) -> dict:
        s = ServerStats()
        check(load().god_server_get_stats(self.h, C.byref(s)))
        return {name: getattr(s, name) for name, _ in ServerStats._fields_}

    def close(self):
        if self.h and self.h.value:
            check(load().god_server_destroy(self.h))
            self.h = C.c_void_p(0)
        self._held.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
