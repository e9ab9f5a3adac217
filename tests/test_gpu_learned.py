"""Learned index (root MLP + linear leaves): training kernels and exactness.

* The GPU forward/backward kernels' gradient of the root's MSE equals the
  oracle's FP32 gradient (fixed reduction orders differ: rel. 1e-4).
* Lookups through the learned index return exactly what the hash table and
  the oracle return, for every indexed key, for absent keys and for keys
  outside the indexed range; seeding through it gives the same anchors.
* Ablation: the trained network routes keys far better than the same network
  untrained (smaller error bounds, fewer hash fallbacks), and about as well
  as a plain linear root on these near-uniform hash keys.
"""
import numpy as np
import pytest

import oracle
from paper_2211_08157_gb300 import synth

pytestmark = pytest.mark.gpu
H = 32


@pytest.fixture(scope="module")
def god():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2211_08157_gb300 as g
    g.load()
    return g


@pytest.mark.parametrize("seed,n", [(1, 1000), (2, 65536), (3, 7)])
def test_root_gradient_matches_oracle(god, seed, n):
    rng = np.random.default_rng(seed)
    th = np.concatenate([rng.normal(0, 1.5, H), rng.normal(0, 0.7, H), rng.normal(0, 0.3, H), [0.05]]).astype(np.float32)
    x = rng.random(n).astype(np.float32)
    y = np.sort(rng.random(n)).astype(np.float32)
    gl, gg = god.god_rmi_root_grad(th, H, x, y)
    ol, og = oracle.root_loss_grad_f32(th, H, x, y)
    ol64, og64 = oracle.root_loss_grad_f64(th.astype(np.float64), H, x.astype(np.float64), y.astype(np.float64))
    assert abs(gl - ol) <= 1e-4 * abs(ol) + 1e-7
    scale = np.max(np.abs(og64))
    assert np.max(np.abs(gg - og)) <= 1e-4 * scale
    assert np.max(np.abs(gg - og64)) <= 1e-4 * scale


def _ref(n=2_000_000, cfg=31):
    return synth.reference(n, cfg, synth.RepeatModel(40, 500, 3000, False, 0.0, 0.02, 0.05))


@pytest.mark.parametrize("bits", [16, 18])
def test_learned_lookup_exact(god, bits):
    ref = _ref()
    params = god.god_params_init(index_kind=god.GOD_INDEX_LEARNED, rmi_leaf_bits=bits)
    idx = god.god_build_index(ref, "10", 21, 11, 3, params=params)
    info = idx.info
    assert info["has_learned"] == 1 and info["rmi_leaves"] == 1 << bits
    keys, start, ent = god.god_index_export(idx)
    rng = np.random.default_rng(bits)
    absent = rng.integers(0, 4 ** 21, 200_000, dtype=np.uint64)
    edge = np.array([0, 1, keys[0] - 1 if keys[0] else 0, keys[0], keys[-1], keys[-1] + 1, 4 ** 21 - 1], np.uint64)
    q = np.concatenate([keys, absent, edge])
    c0, f0 = god.god_index_lookup(idx, q, via=0)
    c1, f1 = god.god_index_lookup(idx, q, via=1)
    assert np.array_equal(c0, c1)
    hit = c0 > 0
    assert np.array_equal(f0[hit], f1[hit])
    o = oracle.Index(ref, "10", 21, 11, 3)
    assert np.array_equal(c1.astype(np.uint64), o.count(q))
    assert (c1[: keys.size] > 0).all()


def test_learned_seed_equals_hash_and_oracle(god):
    ref = _ref(1_000_000, 32)
    reads, offs, _ = synth.reads(ref, 5000, synth.SHORT, synth.ILLUMINA_INDEL, 32)
    params = god.god_params_init(index_kind=god.GOD_INDEX_LEARNED)
    idx = god.god_build_index(ref, "10", 21, 11, 500, params=params)
    out = np.zeros((200_000, 4), np.uint32)
    m_l = god.god_seed_into(idx, reads, offs, out, via=1)
    got_l = out[:m_l].copy()
    m_h = god.god_seed_into(idx, reads, offs, out, via=0)
    got_h = out[:m_h].copy()
    want, _ = oracle.Index(ref, "10", 21, 11, 500).seed(reads, offs, 32)
    assert m_l == m_h == want.size
    assert np.array_equal(got_l, got_h)
    assert np.array_equal(got_l.view(np.uint32).reshape(-1), want.view(np.uint32))


def test_trained_root_ablation(god, capsys):
    """What the trained network gains: vs the same network untrained, vs its
    least-squares output layer alone (no Adam steps), and vs no network at
    all (linear root)."""
    ref = _ref(8_000_000, 33)
    res = {}
    for name, kind, steps in [("trained", god.GOD_ROOT_MLP, 64), ("readout", god.GOD_ROOT_MLP, 0),
                              ("untrained", god.GOD_ROOT_UNTRAINED, 64), ("linear", god.GOD_ROOT_LINEAR, 64)]:
        params = god.god_params_init(index_kind=god.GOD_INDEX_LEARNED, rmi_root=kind, rmi_leaf_bits=16,
                                     rmi_train_steps=steps)
        idx = god.god_build_index(ref, "10", 21, 11, 500, params=params)
        info = idx.info
        res[name] = info
        keys, _, _ = god.god_index_export(idx)
        c0, _ = god.god_index_lookup(idx, keys, via=0)
        c1, _ = god.god_index_lookup(idx, keys, via=1)
        assert np.array_equal(c0, c1)  # exact whatever the root
        idx.close()
    with capsys.disabled():
        for k, v in res.items():
            print(f"\n[ablation] {k:9s} loss={v['rmi_final_loss']:.3g} mean_eps={v['rmi_mean_eps']:.2f} "
                  f"max_eps={v['rmi_max_eps']} fallback_keys={v['rmi_fallback_key_frac']:.4f}")
    t, r, u, l = res["trained"], res["readout"], res["untrained"], res["linear"]
    assert t["rmi_final_loss"] <= r["rmi_final_loss"]      # Adam keeps the better of the two
    assert t["rmi_mean_eps"] < 0.25 * u["rmi_mean_eps"]
    assert t["rmi_fallback_key_frac"] <= u["rmi_fallback_key_frac"]
    assert t["rmi_fallback_key_frac"] < 0.01
    assert t["rmi_mean_eps"] < 2.0 * l["rmi_mean_eps"] + 1.0
