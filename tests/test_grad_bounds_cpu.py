"""The per-element gradient allowance (tests/grad_bounds.py) on the CPU: an fp32
simulation of the GPU's arithmetic (bf16 storage at the same points, fp32 sums) stays
inside it, and planted mistakes -- one wrong element, a dropped ReLU mask, swapped
pinball slopes, transposed weights -- fall outside it."""
import numpy as np
import pytest

from oracle import learned as L
import grad_bounds

F = np.float32


def bf16(a):
    return L.bf16_round(np.asarray(a, F)).astype(F)


def gpu_like(p, x, t, q, plant=None):
    """The GPU's forward/backward restated in fp32 numpy (bf16 where it stores bf16)."""
    W1, b1, W2, b2, w3, b3 = [np.asarray(a, F) if np.ndim(a) else F(a) for a in grad_bounds._split(p)]
    W1, W2, w3 = bf16(W1), bf16(W2), bf16(w3)
    x = np.asarray(x, F)
    t = np.asarray(t, F)
    B = x.shape[0]
    if plant == "transposed_w2":
        W2 = W2.T.copy()
    H1 = bf16(np.maximum(x @ W1.T + b1, F(0)))
    H2 = bf16(np.maximum(H1 @ W2.T + b2, F(0)))
    y = H2 @ w3 + b3
    qq = (1 - q) if plant == "swapped_pinball" else q
    g = (np.where(t - y > 0, -F(qq), F(1 - qq)) / F(B)).astype(F)
    dw3 = g @ H2
    db3 = g.sum(dtype=F)
    dH2 = bf16((np.outer(g, w3) * (H2 > 0)).astype(F))
    db2 = dH2.sum(0, dtype=F)
    dW2 = dH2.T @ H1
    pre = dH2 @ W2
    dH1 = bf16(pre if plant == "no_relu_mask" else pre * (H1 > 0))
    db1 = dH1.sum(0, dtype=F)
    dW1 = dH1.T @ x
    out = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dw3, [db3]]).astype(np.float64)
    return out


@pytest.fixture(scope="module")
def case():
    rng = np.random.default_rng(11)
    B = 96
    p = np.zeros(L.N_PARAMS)
    p[L.OFF_W1:L.OFF_B1] = rng.normal(0, 1 / np.sqrt(L.IN), L.HID * L.IN_PAD)
    p[L.OFF_B1:L.OFF_W2] = rng.normal(0, 0.05, L.HID)
    p[L.OFF_W2:L.OFF_B2] = rng.normal(0, 1 / np.sqrt(L.HID), L.HID * L.HID)
    p[L.OFF_B2:L.OFF_W3] = rng.normal(0, 0.05, L.HID)
    p[L.OFF_W3:L.OFF_B3] = rng.normal(0, 1 / np.sqrt(L.HID), L.HID)
    p[L.OFF_B3] = 9.0
    p = p.astype(F).astype(np.float64)          # the GPU's fp32 master parameters
    x = np.zeros((B, L.IN_PAD))
    x[:, :L.IN] = rng.normal(0, 0.3, (B, L.IN))
    x = L.bf16_round(x)                          # the sketch is stored in bf16
    t = rng.normal(10.0, 0.5, B).astype(F).astype(np.float64)
    return p, x, t


@pytest.mark.parametrize("q", [0.1, 0.5])
def test_fp32_simulation_inside_the_allowance(case, q):
    p, x, t = case
    grads, allow = grad_bounds.error_bounds(p, x, t, q)
    bad = grad_bounds.check(gpu_like(p, x, t, q), grads, allow)
    assert bad.size == 0, (bad[:5], grads[bad[:5]], allow[bad[:5]])
    # past the first layer the allowance is a small fraction of the gradients (the
    # first layer's fp32 sums over 528 inputs carry the widest worst-case bound; the
    # exact-input case below covers it element by element)
    for a, b in ((L.OFF_W2, L.OFF_B2), (L.OFF_B2, L.OFF_W3), (L.OFF_W3, L.OFF_B3)):
        big = np.abs(grads[a:b]) > 1e-9
        assert np.median(allow[a:b][big] / np.abs(grads[a:b][big])) < 0.2


@pytest.mark.parametrize("plant", ["no_relu_mask", "swapped_pinball", "transposed_w2"])
def test_planted_mistakes_fall_outside(case, plant):
    p, x, t = case
    grads, allow = grad_bounds.error_bounds(p, x, t, 0.1)
    assert grad_bounds.check(gpu_like(p, x, t, 0.1, plant=plant), grads, allow).size > 0


def test_one_wrong_element_of_w2_is_seen(case):
    p, x, t = case
    grads, allow = grad_bounds.error_bounds(p, x, t, 0.1)
    g = gpu_like(p, x, t, 0.1)
    w2 = np.arange(L.OFF_W2, L.OFF_B2)
    i = w2[np.argmax(np.abs(grads[w2]))]
    g[i] *= 1.5                                  # 50 % off in one of 65,536 W2 entries
    assert list(grad_bounds.check(g, grads, allow)) == [i]


@pytest.mark.parametrize("seed", [1, 2])
def test_dyadic_inputs_are_exact_in_fp32(seed):
    """On the dyadic case every sum is exact, so fp32 arithmetic (with bf16 storage)
    gives the oracle's fp64 gradients bit for bit; one changed element is then seen
    with no tolerance at all."""
    p, x, q, target = grad_bounds.dyadic_case(seed)
    y, g_ref, _ = L.mlp_forward_backward(p, x, np.zeros(x.shape[0]), q)
    t = target(y)
    _, g_ref, _ = L.mlp_forward_backward(p, x, t, q)
    g = gpu_like(p, x, t, q)
    np.testing.assert_array_equal(g, g_ref)
    assert np.count_nonzero(g_ref[L.OFF_W1:L.OFF_B1]) > 1000   # the case exercises W1
    g[L.OFF_W1 + int(np.argmax(np.abs(g_ref[L.OFF_W1:L.OFF_B1])))] *= 1 + 2.0 ** -10
    assert np.count_nonzero(g != g_ref) == 1
