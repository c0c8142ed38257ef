"""Pins of the learned-threshold oracle (oracle/learned.py) against facts that do not
come from the oracle itself: a published hash value, hand-worked sketches, closed-form
losses, finite differences, a hand-built network, and planted mistakes."""
import numpy as np
import pytest

from oracle import learned as L
from paper_1011_2807_gb300 import synth


def test_fmix32_published_values():
    # MurmurHash3's finaliser: fmix32(0) = 0 and fmix32(1) = 0x514E28B7 (reference value)
    assert int(L.fmix32(0)) == 0
    assert int(L.fmix32(1)) == 0x514E28B7


def one_row(d, w, dim=100):
    return synth.CSR(np.array([0, len(d)], np.int64), np.array(d, np.int32), np.array(w, np.uint8), dim)


def test_sketch_single_feature_by_hand():
    seed = 5
    x = L.sketch(one_row([7], [3]), seed)[0]
    h = int(L.fmix32((7 * L.GOLDEN + (5 ^ L.SEED_MIX)) & 0xFFFFFFFF))
    expect = np.zeros(L.IN_PAD)
    expect[h & 511] = -1.0 if h >> 31 else 1.0        # w / ||r|| = 1
    expect[512:516] = np.log1p([1, 3, 3, 3])
    np.testing.assert_allclose(x, expect, rtol=0, atol=1e-15)


def test_sketch_bucket_energy_and_stats():
    R = synth.spectrum_u8(20, 77, role="R")
    X = L.sketch(R, 3)
    for i in range(R.n_rows):
        d, w = R.row(i)
        w = w.astype(np.float64)
        # with signs, the squared bucket sums equal sum (w/||w||)^2 = 1 plus cross terms
        # of colliding features; without collisions it is exactly 1
        h = L.fmix32((d.astype(np.uint64) * L.GOLDEN + L.hash_seed(3)) & 0xFFFFFFFF) & 511
        if len(np.unique(h)) == len(h):
            assert abs((X[i, :512] ** 2).sum() - 1.0) < 1e-12
        np.testing.assert_allclose(X[i, 512:516], np.log1p([len(d), w.sum(), np.sqrt((w * w).sum()), w.max()]))
        assert (X[i, 516:] == 0).all()


def test_pinball_closed_form():
    loss, g = L.pinball([1.0, 3.0], [2.0, 2.0], 0.25)
    # e = t - y = [1, -1]: q*1 and (q-1)*(-1) -> mean of 0.25 and 0.75
    assert loss == pytest.approx(0.5)
    np.testing.assert_allclose(g, [-0.25 / 2, 0.75 / 2])


def test_bf16_rounding_values():
    # 7 stored fraction bits: halfway cases round to the even neighbour
    np.testing.assert_array_equal(L.bf16_round([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 1.0 + 2 ** -7]),
                                  [1.0, 1.0, 1.0 + 2 ** -6, -2.5, 1.0 + 2 ** -7])


def test_backward_matches_central_differences():
    rng = np.random.default_rng(0)
    p = rng.normal(0, 0.05, size=L.N_PARAMS)
    x = rng.normal(0, 1, size=(6, L.IN_PAD))
    x[:, L.IN:] = 0
    t = rng.normal(0, 1, size=6)
    _, g, _ = L.mlp_forward_backward(p, x, t, 0.3, round_bf16=False)
    for idx in [5, L.IN_PAD * 3 + 7, L.OFF_B1 + 9, L.OFF_W2 + 1000, L.OFF_B2 + 3, L.OFF_W3 + 11, L.OFF_B3]:
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[idx] += h
        pm[idx] -= h
        fd = (L.mlp_forward_backward(pp, x, t, 0.3, False)[2] - L.mlp_forward_backward(pm, x, t, 0.3, False)[2]) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 + 1e-4 * abs(g[idx]), (idx, fd, g[idx])


def test_hand_built_network():
    # unit 0 of layer 1 copies input 0, unit 0 of layer 2 copies it, the output doubles
    # it and adds 1: y = 2 * relu(relu(x0)) + 1
    p = np.zeros(L.N_PARAMS)
    p[L.OFF_W1 + 0] = 1.0
    p[L.OFF_W2 + 0] = 1.0
    p[L.OFF_W3 + 0] = 2.0
    p[L.OFF_B3] = 1.0
    x = np.zeros((3, L.IN_PAD))
    x[:, 0] = [-1.0, 0.5, 2.0]
    y, g, loss = L.mlp_forward_backward(p, x, np.array([0.0, 0.0, 10.0]), 0.5, round_bf16=False)
    np.testing.assert_allclose(y, [1.0, 2.0, 5.0])
    # dL/dy = [0.5, 0.5, -0.5] / 3; db3 is their sum, dw3[0] = sum g * H2[:, 0]
    assert g[L.OFF_B3] == pytest.approx(0.5 / 3)
    assert g[L.OFF_W3] == pytest.approx((0.5 * 0 + 0.5 * 0.5 - 0.5 * 2.0) / 3)


def test_calibrated_scale_quantile_rule():
    kth = np.array([10, 20, 30, 40, 0], np.float32)
    pred = np.array([10, 10, 10, 10, 10], np.float32)   # ratios 1, 2, 3, 4, inf
    assert L.calibrated_scale(kth, pred, 0.0) == pytest.approx(1.0, rel=2e-6)
    assert L.calibrated_scale(kth, pred, 0.2) == pytest.approx(2.0, rel=2e-6)    # rank 1
    assert L.calibrated_scale(kth, pred, 0.5) == pytest.approx(3.0, rel=2e-6)    # rank 2
    s = L.calibrated_scale(kth, pred, 0.5)
    # rows with a k-th score that start above it: ranks 0 and 1 (floor(0.5 * 5) = 2)
    assert ((pred * s > kth) & (kth > 0)).sum() == 2


def test_planted_mistakes_fail_the_pins():
    """A mutant that drops the ReLU mask of layer 2 in the backward pass, or flips the
    pinball slope, must fail the finite-difference or closed-form pins."""
    rng = np.random.default_rng(1)
    p = rng.normal(0, 0.05, size=L.N_PARAMS)
    x = rng.normal(0, 1, size=(5, L.IN_PAD))
    x[:, L.IN:] = 0
    t = rng.normal(0, 1, size=5)

    def mutant(p, x, t, q):
        W1 = p[L.OFF_W1:L.OFF_B1].reshape(L.HID, L.IN_PAD)
        b1 = p[L.OFF_B1:L.OFF_W2]
        W2 = p[L.OFF_W2:L.OFF_B2].reshape(L.HID, L.HID)
        b2 = p[L.OFF_B2:L.OFF_W3]
        w3 = p[L.OFF_W3:L.OFF_B3]
        H1 = np.maximum(x @ W1.T + b1, 0)
        H2 = np.maximum(H1 @ W2.T + b2, 0)
        y = H2 @ w3 + p[L.OFF_B3]
        loss, g = L.pinball(y, t, q)
        dH2 = np.outer(g, w3)                      # mistake: no (H2 > 0) mask
        return dH2.sum(0), loss

    db2_bad, _ = mutant(p, x, t, 0.3)
    _, g_ok, _ = L.mlp_forward_backward(p, x, t, 0.3, round_bf16=False)
    assert not np.allclose(db2_bad, g_ok[L.OFF_B2:L.OFF_W3])
    # a flipped slope gives q - 1 where q belongs
    loss_ok, _ = L.pinball([1.0, 3.0], [2.0, 2.0], 0.25)
    e = np.array([1.0, -1.0])
    loss_bad = np.where(e > 0, (0.25 - 1) * e, 0.25 * e).mean()
    assert loss_bad != pytest.approx(loss_ok)
