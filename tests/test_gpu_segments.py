"""Segmented seeding on the GPU (god_seed_opts.seg_len) against the oracle.

Reads longer than the segment length are cut into segments of seg_len bases
(Sec. 2.2.2 splits ultra-long reads at 30,000 bases), each pattern-aligned on
its own (Sec. 3.2) and seeded; anchors keep the read's id and whole-read
positions, sorted per read. Anchors and the per-segment alignment indices must
equal the oracle's exactly, for host and device buffers, for segment lengths
from 30,000 down to a few hundred bases, and with reads shorter than,
equal to and just past a segment.
"""
import numpy as np
import pytest

import oracle
from paper_2211_08157_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2211_08157_gb300 as god
    god.load()
    ref = synth.reference(4_000_000, 61, synth.RepeatModel(40, 300, 4000, True, 0.05, 0.15, 0.3))
    reads, offs, _ = synth.reads(ref, 400, synth.ONT, synth.ONT_ERR, 0, rng=np.random.default_rng(62))
    # reads of exactly one segment, one base more, and very short ones
    extra = [ref[1000:1000 + 2500], ref[9000:9000 + 2501], ref[20:30], ref[50_000:50_000 + 777 * 3 + 1]]
    reads = np.concatenate([reads] + extra)
    offs = np.concatenate([offs, offs[-1] + np.cumsum([e.size for e in extra]).astype(np.uint64)])
    idx = god.god_build_index(ref, "10", 15, 10, 1000)
    o = oracle.Index(ref, "10", 15, 10, 1000)
    return god, torch, ref, reads, offs, idx, o


@pytest.mark.parametrize("seg_len", [30_000, 2500, 777])
def test_segmented_seeding_matches_oracle(env, seg_len):
    god, torch, ref, reads, offs, idx, o = env
    want, wshift = o.seed(reads, offs, 32, threads=8, seg_len=seg_len)
    if seg_len < 30_000:
        assert wshift.size > offs.size - 1
    # host buffers
    out = np.zeros((want.size + 16, 4), np.uint32)
    shifts = np.zeros(wshift.size, np.uint32)
    m = god.god_seed_into(idx, reads, offs, out, shifts_out=shifts, seg_len=seg_len)
    assert m == want.size
    assert np.array_equal(out[:m].reshape(-1), want.view(np.uint32))
    assert np.array_equal(shifts, wshift)
    # device buffers
    d_reads = torch.from_numpy(reads).cuda()
    d_offs = torch.from_numpy(offs.view(np.int64)).cuda()
    d_sh = torch.zeros(wshift.size, dtype=torch.int32, device="cuda")
    ptr, m2 = god.god_seed_device(idx, d_reads, d_offs, shifts_out=d_sh, seg_len=seg_len)
    assert m2 == want.size

    class V:
        __cuda_array_interface__ = {"shape": (m2, 4), "typestr": "<i4", "data": (ptr, False), "version": 2}
    got = torch.as_tensor(V(), device="cuda").cpu().numpy().view(np.uint32)
    god.god_free(ptr)
    assert np.array_equal(got.reshape(-1), want.view(np.uint32))
    assert np.array_equal(d_sh.cpu().numpy().view(np.uint32), wshift)


def test_segmented_output_too_small_reports_count(env):
    god, torch, ref, reads, offs, idx, o = env
    want, _ = o.seed(reads, offs, 32, threads=8, seg_len=2500)
    out = np.zeros((10, 4), np.uint32)
    with pytest.raises(god.GodError) as e:
        god.god_seed_into(idx, reads, offs, out, seg_len=2500)
    assert e.value.rc == -5 and e.value.needed == want.size
