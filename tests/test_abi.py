"""The C-ABI library loads and exports every symbol include/god.h declares
(no GPU compute), and argument checks fail cleanly before touching a device."""
import ctypes as C
import os
import re

import numpy as np

from paper_2211_08157_gb300 import _lib

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "god.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(god_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["god_build_index", "god_seed", "god_free", "god_strerror", "god_seed_device", "god_seed_into"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    L = _lib.load()
    names = declared_functions()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert set(names) == set(_lib.SIGNATURES), set(names) ^ set(_lib.SIGNATURES)


def test_strerror_and_defaults():
    L = _lib.load()
    assert L.god_strerror(0) == b"ok"
    assert L.god_strerror(-1) == b"invalid argument"
    p = _lib.Params()
    L.god_params_init(C.byref(p))
    assert p.pa_t == 32 and p.index_kind == 0 and p.rmi_eps_max == 64 and p.rmi_train_steps == 64
    o = _lib.SeedOpts()
    L.god_seed_opts_init(C.byref(o))
    assert o.pa_t == 0xFFFFFFFF and o.via == -1


def test_invalid_arguments_rejected_before_device_work():
    L = _lib.load()
    ref = np.frombuffer(b"ACGT" * 100, dtype=np.uint8)
    out = C.c_void_p()
    for pattern, k, w, occ in [(b"", 15, 10, 10), (b"102", 15, 10, 10), (b"000", 15, 10, 10),
                               (b"1" * 65, 15, 10, 10), (b"10", 0, 10, 10), (b"10", 29, 10, 10),
                               (b"10", 15, 0, 10), (b"10", 15, 256, 10), (b"10", 15, 10, 0)]:
        rc = L.god_build_index(ref.ctypes.data, ref.size, pattern, k, w, occ, C.byref(out))
        assert rc == -1, (pattern, k, w, occ)
        assert out.value is None
        assert L.god_last_error() != b""
    rc = L.god_build_index(ref.ctypes.data, 1 << 32, b"10", 15, 10, 10, C.byref(out))
    assert rc == -1
    cnt = C.c_uint64()
    assert L.god_sketch(ref.ctypes.data, ref.size, b"1x", 0, 15, 10, None, None, None, 0, C.byref(cnt), None) == -1
    L.god_free(None)  # ignored


def test_seeding_entry_points_reject_null_arguments():
    """Null index, output or input pointers are argument errors, returned before
    any device work (include/god.h: the library never aborts)."""
    L = _lib.load()
    reads = np.frombuffer(b"ACGT" * 40, dtype=np.uint8)
    offs = np.array([0, 80, 160], dtype=np.uint64)
    anchors = C.c_void_p()
    n = C.c_uint64()
    assert L.god_seed(None, reads.ctypes.data, offs.ctypes.data, 2, C.byref(anchors), C.byref(n)) == -1
    assert anchors.value is None
    assert L.god_seed(None, reads.ctypes.data, offs.ctypes.data, 2, None, C.byref(n)) == -1
    out = np.zeros((16, 4), np.uint32)
    assert L.god_seed_into(None, reads.ctypes.data, offs.ctypes.data, 2, out.ctypes.data, 16, C.byref(n), None) == -1
    assert L.god_seed_device(None, reads.ctypes.data, offs.ctypes.data, 2, None, C.byref(n), None) == -1
    server = C.c_void_p()
    assert L.god_server_create(None, None, C.byref(server)) == -1
    keys = np.zeros(4, np.uint64)
    cnt = np.zeros(4, np.uint32)
    first = np.zeros(4, np.uint64)
    assert L.god_index_lookup(None, keys.ctypes.data, 4, 0, cnt.ctypes.data, first.ctypes.data, None) == -1


def test_profile_reports_empty_without_timing():
    """The profile report and the launch timeline are host-side queries: with
    nothing timed they are an empty object and an empty list, and the
    size-query convention (return the needed size when cap is too small)
    holds."""
    import pytest
    import paper_2211_08157_gb300 as god
    L = _lib.load()
    if god.god_prof_report() or god.god_prof_timeline():
        pytest.skip("launches were timed earlier in this process")
    need = L.god_prof_timeline(None, 0)
    assert need == 3   # "[]" and its terminator
    buf = C.create_string_buffer(need)
    assert L.god_prof_timeline(buf, need) == 0 and buf.value == b"[]"
