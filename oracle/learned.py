"""CPU oracle of the learned start threshold -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may import
this module; it shares no code with the CUDA library.  The learned threshold is not in
the paper: it generalises Section 4.4's MinPruneScore (a threshold derived from the
loops already run) to one predicted per query, and stays exact through
verify-and-fallback.  What the library computes, restated in plain numpy (fp64):

* :func:`sketch` -- the model input of one query r: 512 signed feature-hashing buckets
  (bucket and sign from the MurmurHash3 32-bit finaliser of d * 0x9E3779B1 + seed,
  value w / ||r||_2), then log1p of nnz(r), sum w, ||r||_2 and max w (516 values,
  padded with zeros to 528).
* :func:`mlp_forward_backward` -- 528 -> 256 -> 256 -> 1 with ReLU; the mean pinball
  loss at quantile q of the prediction y against the target t (log of the k-th best
  score), and every parameter's gradient by the chain rule.  With ``round_bf16`` the
  weights and activations are rounded to bfloat16 where the GPU stores them in it.
* :func:`calibrated_scale` -- the multiplier of the predictions for a target fallback
  rate: rank floor(miss_rate * n) of kth / prediction, less a relative 1e-6.

Parity status: pinned by ``tests/test_oracle_learned_pins.py`` (the published
finaliser value fmix32(1) = 0x514E28B7, hand-worked sketches, closed-form pinball
values, central finite differences of the loss, a hand-built network, the quantile
rule on small arrays).
"""
from __future__ import annotations

import numpy as np

BUCKETS = 512
IN = BUCKETS + 4      # 516
IN_PAD = 528
HID = 256
OFF_W1 = 0
OFF_B1 = HID * IN_PAD
OFF_W2 = OFF_B1 + HID
OFF_B2 = OFF_W2 + HID * HID
OFF_W3 = OFF_B2 + HID
OFF_B3 = OFF_W3 + HID
N_PARAMS = OFF_B3 + 1
GOLDEN = 0x9E3779B1   # multiplier of the feature id before hashing
SEED_MIX = 0x5BD1E995  # a model's hash seed is its creation seed xor this


def fmix32(x):
    """MurmurHash3's 32-bit finaliser (xor-shift / multiply rounds), elementwise."""
    x = np.asarray(x, dtype=np.uint64) & 0xFFFFFFFF
    x ^= x >> 16
    x = (x * 0x85EBCA6B) & 0xFFFFFFFF
    x ^= x >> 13
    x = (x * 0xC2B2AE35) & 0xFFFFFFFF
    x ^= x >> 16
    return x


def hash_seed(model_seed: int) -> int:
    return (int(model_seed) ^ SEED_MIX) & 0xFFFFFFFF


def sketch(R, model_seed: int) -> np.ndarray:
    """[n_rows][528] fp64 model inputs of the rows of R (a CSR with .row(i))."""
    seed = hash_seed(model_seed)
    out = np.zeros((R.n_rows, IN_PAD))
    for i in range(R.n_rows):
        d, w = R.row(i)
        if len(d) == 0:
            continue
        w = np.asarray(w, dtype=np.float64)
        norm = np.sqrt((w * w).sum())
        h = fmix32((np.asarray(d, dtype=np.uint64) * GOLDEN + seed) & 0xFFFFFFFF)
        sign = np.where(h >> 31, -1.0, 1.0)
        np.add.at(out[i], (h & (BUCKETS - 1)).astype(np.int64), sign * w / norm)
        out[i, BUCKETS:IN] = np.log1p([len(d), w.sum(), norm, w.max()])
    return out


def bf16_round(a) -> np.ndarray:
    """Round-to-nearest-even to bfloat16 (8 significant bits), returned as fp64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def pinball(y, t, q):
    """Mean pinball loss at quantile q and its gradient with respect to y."""
    y = np.asarray(y, np.float64)
    e = np.asarray(t, np.float64) - y
    loss = np.where(e > 0, q * e, (q - 1) * e).mean()
    g = np.where(e > 0, -q, 1 - q) / len(y)
    return loss, g


def mlp_forward_backward(p, x, t, q, round_bf16: bool = True):
    """Predictions, gradients of the mean pinball loss (flat, in the parameter layout
    W1 [256][528] | b1 | W2 [256][256] | b2 | w3 | b3) and the loss."""
    rb = bf16_round if round_bf16 else (lambda a: np.asarray(a, np.float64))
    p = np.asarray(p, np.float64)
    x = np.asarray(x, np.float64)
    W1 = rb(p[OFF_W1:OFF_B1].reshape(HID, IN_PAD))
    b1 = p[OFF_B1:OFF_W2]
    W2 = rb(p[OFF_W2:OFF_B2].reshape(HID, HID))
    b2 = p[OFF_B2:OFF_W3]
    w3 = rb(p[OFF_W3:OFF_B3])
    b3 = float(p[OFF_B3])
    H1 = rb(np.maximum(x @ W1.T + b1, 0.0))
    H2 = rb(np.maximum(H1 @ W2.T + b2, 0.0))
    y = H2 @ w3 + b3
    loss, g = pinball(y, t, q)
    dw3 = g @ H2
    db3 = g.sum()
    dH2 = rb(np.outer(g, w3) * (H2 > 0))
    db2 = dH2.sum(0)
    dW2 = dH2.T @ H1
    dH1 = rb((dH2 @ W2) * (H1 > 0))
    db1 = dH1.sum(0)
    dW1 = dH1.T @ x
    grads = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dw3, [db3]])
    return y, grads, loss


def calibrated_scale(kth, pred, miss_rate: float) -> float:
    """Largest multiplier leaving at most floor(miss_rate * n) rows with
    scale * pred > kth (rows without a k-th score, kth <= 0, count as misses)."""
    kth = np.asarray(kth, np.float32)
    pred = np.asarray(pred, np.float32)
    ratio = np.full(len(kth), np.inf, dtype=np.float32)
    ok = (kth > 0) & (pred > 0)
    ratio[ok] = kth[ok] / pred[ok]
    v = np.sort(ratio)[min(len(ratio) - 1, int(np.floor(miss_rate * len(ratio))))]
    return float(np.float32(np.float64(v) * (1.0 - 1e-6)))
