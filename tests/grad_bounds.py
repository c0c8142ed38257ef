"""Per-element error allowance for the GPU's MLP gradients against the fp64 oracle.

The GPU computes the learned threshold's forward and backward pass with bf16 weights,
bf16 activations and bf16 activation gradients (H1, H2, dH2, dH1), fp32 accumulation
in every sum, and fp32 gradients.  ``oracle.learned.mlp_forward_backward`` rounds to
bf16 at the same points but computes everything else in fp64.  The two therefore
differ by (a) fp32 summation error, at most n * 2^-24 of the sum of the absolute
terms for n terms in any order, (b) a bf16 rounding step, only where the interval
the other side's pre-rounding value can lie in crosses a rounding boundary, and (c) a ReLU mask or a
pinball-loss sign that flips where the pre-activation (or the residual t - y) lies
within the error already accumulated.  ``error_bounds`` carries an absolute error
allowance through the network with these three rules -- |d(AB)| <= |dA||B| + |A||dB|
for products -- and returns it per gradient element, next to the oracle's gradient.

Nothing here is the oracle: it only states how far two correct computations in
different precisions can drift apart.  ``tests/test_grad_bounds_cpu.py`` checks on
the CPU that an fp32 simulation of the GPU's arithmetic stays inside the allowance
and that planted mistakes fall outside it.
"""
import numpy as np

from oracle import learned as L

U32 = 2.0 ** -24      # fp32 unit roundoff
FP32_FACTOR = 2.0     # the tensor cores' fp32 accumulation: allow twice the textbook bound


def _split(p):
    W1 = p[L.OFF_W1:L.OFF_B1].reshape(L.HID, L.IN_PAD)
    b1 = p[L.OFF_B1:L.OFF_W2]
    W2 = p[L.OFF_W2:L.OFF_B2].reshape(L.HID, L.HID)
    b2 = p[L.OFF_B2:L.OFF_W3]
    w3 = p[L.OFF_W3:L.OFF_B3]
    b3 = float(p[L.OFF_B3])
    return W1, b1, W2, b2, w3, b3


def _rounded(v, e):
    """bf16 value stored from an exact pre-rounding value v when the other side's
    pre-rounding value lies within e of it: rounding is monotone, so both store the
    same value unless [v - e, v + e] crosses a rounding boundary; the difference is
    then at most the distance from bf16(v) to the rounded interval ends.  e is widened
    by 2^-22 |v| for the float32 step inside the rounding."""
    e = e + 2.0 ** -22 * np.abs(v)
    r = L.bf16_round(v)
    lo = L.bf16_round(v - e)
    hi = L.bf16_round(v + e)
    return r, np.maximum(np.abs(hi - r), np.abs(r - lo))


def error_bounds(p, x, t, q):
    """(oracle gradients, per-element allowance), both flat in the parameter layout."""
    rb = L.bf16_round
    p = np.asarray(p, np.float64)
    x = np.asarray(x, np.float64)
    t = np.asarray(t, np.float64)
    W1, b1, W2, b2, w3, b3 = _split(p)
    W1, W2, w3 = rb(W1), rb(W2), rb(w3)
    B = x.shape[0]
    ax, aW1, aW2, aw3 = np.abs(x), np.abs(W1), np.abs(W2), np.abs(w3)
    acc = lambda n: FP32_FACTOR * n * U32
    # forward: H = bf16(relu(z)) -- relu then bf16 is monotone in z
    z1 = x @ W1.T + b1
    e_z1 = acc(L.IN_PAD + 1) * (ax @ aW1.T + np.abs(b1))
    H1, e_H1 = _rounded(np.maximum(z1, 0.0), 0.0 * z1)
    e_H1 = np.maximum(e_H1, np.abs(rb(np.maximum(z1 + e_z1, 0.0)) - H1))
    e_H1 = np.maximum(e_H1, np.abs(H1 - rb(np.maximum(z1 - e_z1, 0.0))))
    unc1 = np.abs(z1) <= e_z1                        # the ReLU mask may differ
    z2 = H1 @ W2.T + b2
    e_z2 = e_H1 @ aW2.T + acc(L.HID + 1) * ((np.abs(H1) + e_H1) @ aW2.T + np.abs(b2))
    H2 = rb(np.maximum(z2, 0.0))
    e_H2 = np.maximum(np.abs(rb(np.maximum(z2 + e_z2, 0.0)) - H2), np.abs(H2 - rb(np.maximum(z2 - e_z2, 0.0))))
    e_H2 = e_H2 + 2.0 ** -22 * np.abs(H2)
    unc2 = np.abs(z2) <= e_z2
    y = H2 @ w3 + b3
    e_y = e_H2 @ aw3 + acc(L.HID + 1) * ((np.abs(H2) + e_H2) @ aw3 + abs(b3))
    _, g = L.pinball(y, t, q)
    flip = np.abs(t - y) <= e_y + U32 * np.abs(t) * 4      # the loss slope may differ
    e_g = np.where(flip, 1.0 / B, 2 * U32 * np.abs(g))
    ag = np.abs(g) + e_g
    # backward, output layer
    dw3 = g @ H2
    e_dw3 = ag @ e_H2 + e_g @ np.abs(H2) + acc(B) * (ag @ (np.abs(H2) + e_H2))
    db3 = g.sum()
    e_db3 = e_g.sum() + acc(B) * ag.sum()
    # dH2 = bf16(g w3) where H2 > 0
    gw = np.outer(g, w3)
    mask2 = H2 > 0
    dH2, e_dH2 = _rounded(gw * mask2, 2 * U32 * np.abs(gw))
    big = np.outer(ag, aw3) * (1 + 2.0 ** -7)               # any value the entry can take
    e_dH2 = np.where(unc2 | flip[:, None], np.abs(dH2) + big * (mask2 | unc2), e_dH2)
    adH2 = np.abs(dH2) + e_dH2
    # hidden layer 2
    db2 = dH2.sum(0)
    e_db2 = e_dH2.sum(0) + acc(B) * adH2.sum(0)
    aH1 = np.abs(H1) + e_H1
    dW2 = dH2.T @ H1
    e_dW2 = e_dH2.T @ aH1 + np.abs(dH2).T @ e_H1 + acc(B) * (adH2.T @ aH1)
    # dH1 = bf16(dH2 W2) where H1 > 0
    pre = dH2 @ W2
    e_pre = e_dH2 @ aW2 + acc(L.HID) * (adH2 @ aW2)
    mask1 = H1 > 0
    dH1, e_dH1 = _rounded(pre * mask1, e_pre * mask1)
    e_dH1 = np.where(unc1, np.abs(dH1) + (np.abs(pre) + e_pre) * (1 + 2.0 ** -7), e_dH1)
    adH1 = np.abs(dH1) + e_dH1
    # hidden layer 1
    db1 = dH1.sum(0)
    e_db1 = e_dH1.sum(0) + acc(B) * adH1.sum(0)
    dW1 = dH1.T @ x
    e_dW1 = e_dH1.T @ ax + acc(B) * (adH1.T @ ax)
    grads = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dw3, [db3]])
    allow = np.concatenate([e_dW1.ravel(), e_db1, e_dW2.ravel(), e_db2, e_dw3, [e_db3]])
    # the pass above restates the oracle's to get its intermediates: it must agree
    _, g_oracle, _ = L.mlp_forward_backward(p, x, t, q, round_bf16=True)
    assert np.allclose(grads, g_oracle, rtol=1e-12, atol=1e-15), "restated pass differs from the oracle's"
    return g_oracle, allow


def check(g, grads, allow, slack=1.5, floor=1e-12):
    """Indices of elements outside the allowance (empty when the check passes)."""
    err = np.abs(np.asarray(g, np.float64) - grads)
    return np.nonzero(err > slack * allow + floor)[0]


def dyadic_case(seed, B=64):
    """Inputs on which every sum of the forward and backward pass is exact in fp32 (and
    in fp64), so that the GPU's gradients must equal the oracle's bit for bit: x in
    {0, +-1} with 16 nonzeros per row, weights and biases small multiples of 1/8 or
    1/16, B = 64 rows, quantile 0.25 (so every loss slope, -q/B or (1-q)/B, is a power
    of two times 1 or 3), and targets 5 away from the prediction.  Every partial sum is
    a multiple of a common power of two below 2^24 of it: for instance z1 is a multiple
    of 1/8 below 8.5 in magnitude, z2 of 1/128 below 272, y of 1/1024 below 8,704; the
    bf16 roundings (of H2 and dH1) then round identical values.  Returns (p, x, q) and a
    function mapping predictions to targets."""
    rng = np.random.default_rng(seed)
    p = np.zeros(L.N_PARAMS)
    p[L.OFF_W1:L.OFF_B1] = rng.integers(-4, 5, L.HID * L.IN_PAD) / 8.0
    p[L.OFF_B1:L.OFF_W2] = rng.integers(-4, 5, L.HID) / 8.0
    p[L.OFF_W2:L.OFF_B2] = rng.integers(-2, 3, L.HID * L.HID) / 16.0
    p[L.OFF_B2:L.OFF_W3] = rng.integers(-8, 9, L.HID) / 16.0
    p[L.OFF_W3:L.OFF_B3] = rng.integers(-1, 2, L.HID) / 8.0
    p[L.OFF_B3] = 3.0
    x = np.zeros((B, L.IN_PAD))
    for b in range(B):
        cols = rng.choice(L.IN, size=16, replace=False)
        x[b, cols] = rng.choice([-1.0, 1.0], size=16)
    signs = rng.choice([-5.0, 5.0], size=B)
    return p, x, 0.25, (lambda y: y + signs)
