"""The allocation-free sketch entry point (god_sketch_noalloc) against god_sketch.

god_sketch_noalloc serves callers that may not allocate device memory during a
call; it keeps the sketch kernel's scratch in a device array shared by all
calls. Two calls in a row with different sequences and parameters must each
return exactly what god_sketch returns (integer results: bit-exact), which
also shows that a call does not see the previous call's scratch contents.
This file is collected last so that a failure here stops a run only after
every other test has run.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2211_08157_gb300 import synth

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "god.h")
MAX_PATTERNED = int(re.search(r"#define GOD_NOALLOC_MAX_PATTERNED (\d+)ULL", open(HEADER).read()).group(1))


@pytest.fixture(scope="module")
def lib():
    import paper_2211_08157_gb300 as god
    return god.load()


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2211_08157_gb300 as god
    return god, god.load(), torch


def _noalloc(L, torch, seq, pattern, shift, k, w, cap):
    d_seq = torch.from_numpy(seq).cuda()
    d_out = torch.zeros((max(cap, 1), 4), dtype=torch.int32, device="cuda")
    n = C.c_uint64()
    rc = L.god_sketch_noalloc(d_seq.data_ptr(), seq.size, pattern.encode(), shift, k, w, d_out.data_ptr(), cap,
                              C.byref(n), None)
    rec = d_out.cpu().numpy().view(np.uint32).reshape(-1, 4)[: min(n.value, cap)]
    keys = rec[:, 0].astype(np.uint64) | (rec[:, 1].astype(np.uint64) << np.uint64(32))
    return rc, n.value, keys, rec[:, 2], rec[:, 3]


@pytest.mark.gpu
def test_noalloc_matches_sketch_two_calls(env):
    god, L, torch = env
    rng = np.random.default_rng(77)
    cases = [
        (synth.ACGT[rng.integers(0, 4, 300_001)], "10", 1, 21, 11),
        (synth.ACGT[rng.integers(0, 4, 50_000)], "110", 0, 15, 10),
    ]
    cases[1][0][rng.integers(0, 50_000, 40)] = ord("N")
    for seq, pattern, shift, k, w in cases:
        want_k, want_p, want_z = god.god_sketch(seq, pattern, shift, k, w)
        rc, n, keys, pos, z = _noalloc(L, torch, seq, pattern, shift, k, w, want_k.size + 10)
        assert rc == 0, L.god_last_error()
        assert n == want_k.size
        assert np.array_equal(keys, want_k)
        assert np.array_equal(pos, want_p)
        assert np.array_equal(z, want_z.astype(np.uint32))


@pytest.mark.gpu
def test_noalloc_reports_size_and_limits(env):
    god, L, torch = env
    rng = np.random.default_rng(78)
    seq = synth.ACGT[rng.integers(0, 4, 20_000)]
    want_k, _, _ = god.god_sketch(seq, "1", 0, 15, 10)
    rc, n, keys, _, _ = _noalloc(L, torch, seq, "1", 0, 15, 10, 100)
    assert rc == -5 and n == want_k.size            # too small: count reported, first 100 written
    assert np.array_equal(keys, want_k[:100])
    # beyond the scratch array's limit: rejected on the host, nothing launched
    d = torch.zeros(16, dtype=torch.uint8, device="cuda")
    o = torch.zeros((1, 4), dtype=torch.int32, device="cuda")
    cnt = C.c_uint64()
    too_long = 2 * MAX_PATTERNED + 10                 # pattern 10 keeps half of it
    assert L.god_sketch_noalloc(d.data_ptr(), too_long, b"10", 0, 15, 10, o.data_ptr(), 1, C.byref(cnt), None) == -1
    assert b"GOD_NOALLOC_MAX_PATTERNED" in L.god_last_error()
    # host memory is refused (it would need a device copy)
    assert L.god_sketch_noalloc(seq.ctypes.data, seq.size, b"1", 0, 15, 10, o.data_ptr(), 1, C.byref(cnt), None) == -1
    # an output address that is 8- but not 16-byte aligned is refused before any launch
    assert L.god_sketch_noalloc(d.data_ptr(), 16, b"1", 0, 15, 10, o.data_ptr() + 8, 1, C.byref(cnt), None) == -1
    assert b"16-byte aligned" in L.god_last_error()


def test_noalloc_limit_is_exact_on_host(lib):
    """The largest promised patterned length is accepted in the tightest case
    (k = 28, w = 255, the smallest sub-tile) and one more base is refused.
    Fake, non-device pointers are used: a length that fits reaches the device
    pointer check and is refused there, so nothing is launched."""
    L = lib
    cnt = C.c_uint64(7)
    fake_seq, fake_out = 4096, 8192
    rc = L.god_sketch_noalloc(fake_seq, MAX_PATTERNED, b"1", 0, 28, 255, fake_out, 1, C.byref(cnt), None)
    assert rc == -1 and b"device memory" in L.god_last_error() and cnt.value == 0
    rc = L.god_sketch_noalloc(fake_seq, MAX_PATTERNED + 1, b"1", 0, 28, 255, fake_out, 1, C.byref(cnt), None)
    assert rc == -1 and b"GOD_NOALLOC_MAX_PATTERNED" in L.god_last_error()
    rc = L.god_sketch_noalloc(fake_seq, 100, b"1", 0, 28, 255, fake_out + 8, 1, C.byref(cnt), None)
    assert rc == -1 and b"16-byte aligned" in L.god_last_error()
