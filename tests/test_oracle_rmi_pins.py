"""Pins of the oracle's learned-index (RMI) reference.

The MLP root's analytic gradient is checked against central finite differences
of the loss; the FP32 sequential gradient against the double one; the leaf least
squares against numpy's lstsq-based polyfit; the per-leaf error bound against an
independent double-precision evaluation of the leaf predictions.
"""
import numpy as np
import pytest

import oracle

H = 32


def _theta(seed, H=H):
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, 2.0, H)
    b1 = rng.normal(0, 1.0, H)
    W2 = rng.normal(0, 0.3, H)
    b2 = rng.normal(0, 0.1)
    return np.concatenate([W1, b1, W2, [b2]])


def _loss_only(theta, x, y):
    W1, b1, W2, b2 = theta[:H], theta[H:2 * H], theta[2 * H:3 * H], theta[3 * H]
    a = np.maximum(np.outer(x, W1) + b1, 0.0)
    f = a @ W2 + b2
    return float(np.mean((f - y) ** 2))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_root_gradient_finite_differences(seed):
    rng = np.random.default_rng(50 + seed)
    x = np.sort(rng.random(400))
    y = x + 0.01 * rng.normal(size=x.size)
    th = _theta(seed)
    loss, g = oracle.root_loss_grad_f64(th, H, x, y)
    assert abs(loss - _loss_only(th, x, y)) <= 1e-12 * max(1.0, loss)
    h = 1e-6
    fd = np.zeros_like(th)
    for i in range(th.size):
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd[i] = (_loss_only(tp, x, y) - _loss_only(tm, x, y)) / (2 * h)
    scale = np.max(np.abs(g))
    assert np.max(np.abs(fd - g)) <= 1e-6 * scale + 1e-9


def test_root_gradient_f32_close_to_f64():
    rng = np.random.default_rng(60)
    x = rng.random(2000)
    y = np.sort(x)
    th = _theta(9)
    l64, g64 = oracle.root_loss_grad_f64(th, H, x, y)
    l32, g32 = oracle.root_loss_grad_f32(th.astype(np.float32), H, x.astype(np.float32), y.astype(np.float32))
    assert abs(l32 - l64) <= 1e-4 * max(l64, 1e-6)
    assert np.max(np.abs(g32 - g64)) <= 1e-4 * np.max(np.abs(g64))


def _keys(n, bits, seed):
    rng = np.random.default_rng(seed)
    k = np.unique(rng.integers(0, 1 << bits, int(n * 1.05), dtype=np.uint64))
    return k[:n]


def test_leaf_least_squares_and_error_bounds():
    keys = _keys(20000, 42, 70)
    kmin = int(keys[0])
    span = float(int(keys[-1]) - kmin)
    inv_span = np.float32(1.0 / span)
    n_leaves = 1024
    # a near-identity root: one active hidden unit passes x through
    th = np.zeros(3 * H + 1, np.float32)
    th[0] = 1.0
    th[2 * H] = 1.0
    slope, icept, base, eps = oracle.rmi_fit_leaves(th, H, keys, kmin, float(inv_span), n_leaves)
    x, leaf = oracle.root_route(th, H, keys, kmin, float(inv_span), n_leaves)
    assert leaf.max() < n_leaves
    rank = np.arange(keys.size, dtype=np.float64)
    for l in range(n_leaves):
        sel = np.nonzero(leaf == l)[0]
        if sel.size == 0:
            assert eps[l] == 0 and slope[l] == 0 and icept[l] == 0
            continue
        assert base[l] == keys[sel].min()
        dx = (keys[sel] - base[l]).astype(np.float64)
        if sel.size >= 2:
            b, a = np.polyfit(dx, rank[sel], 1)
            assert abs(float(slope[l]) - b) <= 1e-5 * abs(b) + 1e-12
            assert abs(float(icept[l]) - a) <= 1e-5 * max(abs(a), 1.0)
        else:
            assert slope[l] == 0 and float(icept[l]) == rank[sel][0]
        d32 = dx.astype(np.float32).astype(np.float64)
        pred = np.floor(np.float64(slope[l]) * d32 + np.float64(icept[l]))
        err = np.abs(rank[sel] - pred)
        assert err.max() <= eps[l] + 1
        assert err.max() >= eps[l] - 1
    # the bound is small for a well-routed uniform key set
    assert eps.max() < 64


def test_root_routing_covers_leaves_in_order():
    keys = _keys(5000, 38, 71)
    kmin = int(keys[0])
    inv_span = float(np.float32(1.0 / float(int(keys[-1]) - kmin)))
    th = np.zeros(3 * H + 1, np.float32)
    th[0] = 1.0
    th[2 * H] = 1.0
    x, leaf = oracle.root_route(th, H, keys, kmin, inv_span, 256)
    assert np.all(np.diff(x) >= 0) and x[0] == 0.0 and abs(x[-1] - 1.0) < 1e-6
    assert np.all(np.diff(leaf.astype(np.int64)) >= 0)
    assert leaf[0] == 0 and leaf[-1] == 255
