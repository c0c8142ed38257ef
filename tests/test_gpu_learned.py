"""The learned start threshold: tensor-core GEMM, sketch, MLP forward/backward against
fp64 references, training, and the learned join's exactness (verify-and-fallback)."""
import numpy as np
import pytest

from oracle import learned as L
from paper_1011_2807_gb300 import synth
import compare
import grad_bounds

pytestmark = pytest.mark.gpu

W1_SHAPE = (L.HID, L.IN_PAD)
OFF_B1, OFF_W2, OFF_B2, OFF_W3, OFF_B3 = L.OFF_B1, L.OFF_W2, L.OFF_B2, L.OFF_W3, L.OFF_B3


@pytest.fixture(scope="module")
def knn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1011_2807_gb300 as knn
    knn.lib()
    return knn


# ----------------------------------------------------------------------------------
# GEMM on tensor cores
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("M,N,K", [(64, 64, 32), (100, 70, 53), (3, 300, 528), (256, 256, 1000), (1, 1, 1)])
@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True)])
def test_gemm_bf16(knn, M, N, K, ta, tb):
    import torch
    from paper_1011_2807_gb300.binding import knn_gemm_bf16
    g = torch.Generator().manual_seed(M * 7 + N + K)
    A = torch.randn((K, M) if ta else (M, K), generator=g).to(torch.bfloat16).cuda()
    B = torch.randn((N, K) if tb else (K, N), generator=g).to(torch.bfloat16).cuda()
    sa = (1, M) if ta else (K, 1)
    sb = (1, K) if tb else (N, 1)
    C = torch.full((M, N), 3.0, device="cuda")
    knn_gemm_bf16(A, sa, B, sb, C, (N, 1), M, N, K)
    torch.cuda.synchronize()
    Ad = A.double().cpu().numpy()
    Bd = B.double().cpu().numpy()
    ref = (Ad.T if ta else Ad) @ (Bd.T if tb else Bd)
    np.testing.assert_allclose(C.cpu().numpy(), ref, rtol=1e-4, atol=1e-4 * np.sqrt(K))
    knn_gemm_bf16(A, sa, B, sb, C, (N, 1), M, N, K, accumulate=True)
    torch.cuda.synchronize()
    np.testing.assert_allclose(C.cpu().numpy(), 2 * ref, rtol=1e-4, atol=2e-4 * np.sqrt(K))


# ----------------------------------------------------------------------------------
# sketch
# ----------------------------------------------------------------------------------

def test_sketch(knn):
    R = synth.spectrum_u8(64, 301, role="R")
    m = knn.ThresholdModel(seed=17)
    X = m.sketch(knn.DeviceCSR.from_host(R)).float().cpu().numpy()
    ref = L.sketch(R, 17)
    np.testing.assert_allclose(X, L.bf16_round(ref), rtol=1e-2, atol=2e-3)
    assert (X[:, 516:] == 0).all()
    m.close()


# ----------------------------------------------------------------------------------
# forward / backward against an fp64 restatement (itself pinned by finite differences)
# ----------------------------------------------------------------------------------

def mlp_ref(p, x, t, q, round_like_gpu=True):
    return L.mlp_forward_backward(p, x, t, q, round_bf16=round_like_gpu)


@pytest.mark.parametrize("q", [0.1, 0.5])
def test_forward_backward_vs_fp64(knn, q):
    import torch
    m = knn.ThresholdModel(seed=5)
    R = synth.spectrum_u8(96, 311, role="R")
    x = m.sketch(knn.DeviceCSR.from_host(R))
    rng = np.random.default_rng(1)
    t = torch.from_numpy(rng.normal(10.0, 0.5, size=R.n_rows).astype(np.float32)).cuda()
    pred, grads = m.forward_backward(x, t, q)
    torch.cuda.synchronize()
    p = m.params().cpu().numpy()
    y_ref, g_ref, _ = mlp_ref(p, x.float().cpu().numpy().astype(np.float64), t.cpu().numpy().astype(np.float64), q)
    np.testing.assert_allclose(pred.cpu().numpy(), y_ref, rtol=1e-3, atol=1e-3)
    # every gradient element within the allowance derived from fp32 sums, bf16 storage
    # points and possible ReLU / loss-slope flips (tests/grad_bounds.py)
    g = grads.cpu().numpy().astype(np.float64)
    xs = x.float().cpu().numpy().astype(np.float64)
    ts = t.cpu().numpy().astype(np.float64)
    g_ref2, allow = grad_bounds.error_bounds(p.astype(np.float64), xs, ts, q)
    np.testing.assert_array_equal(g_ref2, g_ref)
    bad = grad_bounds.check(g, g_ref, allow)
    assert bad.size == 0, (bad.size, bad[:5].tolist(), g[bad[:5]].tolist(), g_ref[bad[:5]].tolist(),
                           allow[bad[:5]].tolist())
    m.close()


@pytest.mark.parametrize("seed", [1, 2])
def test_forward_backward_exact_on_dyadic_inputs(knn, seed):
    """Weights, inputs and targets chosen so that every sum of the pass is exact in
    fp32 (tests/grad_bounds.py: dyadic_case): the GPU's prediction and every one of
    the 201,473 gradient elements must equal the fp64 oracle's exactly."""
    import torch
    p, x, q, target = grad_bounds.dyadic_case(seed)
    m = knn.ThresholdModel(seed=5)
    blob = bytearray(m.get_params())
    off = 8 + 8                                   # header, step
    blob[off:off + 4 * L.N_PARAMS] = p.astype(np.float32).tobytes()
    m.set_params(bytes(blob))
    y_ref, _, _ = L.mlp_forward_backward(p, x, np.zeros(x.shape[0]), q)
    t = target(y_ref)
    xb = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).cuda()
    tt = torch.from_numpy(t.astype(np.float32)).cuda()
    pred, grads = m.forward_backward(xb, tt, q)
    torch.cuda.synchronize()
    _, g_ref, _ = L.mlp_forward_backward(p, x, t, q)
    np.testing.assert_array_equal(pred.cpu().numpy().astype(np.float64), y_ref)
    g = grads.cpu().numpy().astype(np.float64)
    bad = np.nonzero(g != g_ref)[0]
    assert bad.size == 0, (bad.size, bad[:5].tolist(), g[bad[:5]].tolist(), g_ref[bad[:5]].tolist())
    assert np.count_nonzero(g_ref[L.OFF_W1:L.OFF_B1]) > 1000
    m.close()


# ----------------------------------------------------------------------------------
# training and the learned join
# ----------------------------------------------------------------------------------

@pytest.fixture(scope="module")
def trained(knn):
    import torch
    S = synth.spectrum_u8(30000, 321, role="S")
    T = synth.spectrum_u8(6000, 322, role="R")
    idx = knn.knn_join_build_index(S, block_size=4096)
    _, sc = knn.knn_join(idx, knn.DeviceCSR.from_host(T), 5)
    kth = sc[:, 4].float()
    m = knn.ThresholdModel(seed=3)
    loss0 = m.train(T, kth, epochs=1, batch=256, quantile=0.1, seed=1)
    loss1 = m.train(T, kth, epochs=25, batch=256, quantile=0.1, seed=2)
    torch.cuda.synchronize()
    yield dict(S=S, T=T, idx=idx, kth=kth, model=m, loss0=loss0, loss1=loss1)
    m.close()
    idx.close()


def test_training_reduces_loss(trained):
    assert trained["loss1"] < 0.7 * trained["loss0"], (trained["loss0"], trained["loss1"])


def test_prediction_quantile(knn, trained):
    tau = trained["model"].predict(trained["T"]).cpu().numpy()
    kth = trained["kth"].cpu().numpy()
    below = (tau <= kth).mean()
    assert below > 0.6, below     # trained at q = 0.1: mostly below the true k-th score


def test_save_load_roundtrip(knn, trained):
    blob = trained["model"].get_params()
    m2 = knn.ThresholdModel(seed=99)
    m2.set_params(blob)
    R = synth.spectrum_u8(50, 331, role="R")
    a = trained["model"].predict(R).cpu().numpy()
    b = m2.predict(R).cpu().numpy()
    np.testing.assert_array_equal(a, b)
    m2.close()


def test_learned_join_is_exact(knn, trained, oracle_mod):
    import torch
    E = synth.spectrum_u8(400, 341, role="R")
    idx = trained["idx"]
    Ed = knn.DeviceCSR.from_host(E)
    pids, psc = knn.knn_join(idx, Ed, 5)
    lids, lsc, st = knn.knn_join_learned(idx, trained["model"], Ed, 5)
    torch.cuda.synchronize()
    assert torch.equal(pids, lids) and torch.equal(psc, lsc)
    assert st["rows"] == E.n_rows and 0 <= st["fallback_rows"] < E.n_rows
    eids, esc, _ = oracle_mod.iib_join(E, trained["S"], 5, threads=8)
    compare.assert_exact(lids.cpu().numpy(), lsc.cpu().numpy(), eids, esc, "learned")


def test_over_predicting_thresholds_fall_back_everywhere(knn, trained):
    import torch
    E = synth.spectrum_u8(200, 351, role="R")
    Ed = knn.DeviceCSR.from_host(E)
    idx = trained["idx"]
    pids, psc = knn.knn_join(idx, Ed, 5)
    inf = torch.full((E.n_rows,), float("inf"), device="cuda")
    lids, lsc, st = knn.knn_join_learned(idx, None, Ed, 5, tau=inf)
    assert st["fallback_rows"] == E.n_rows
    assert torch.equal(pids, lids) and torch.equal(psc, lsc)
    zero = torch.zeros(E.n_rows, device="cuda")
    lids, lsc, st = knn.knn_join_learned(idx, None, Ed, 5, tau=zero)
    assert st["fallback_rows"] == 0
    assert torch.equal(pids, lids) and torch.equal(psc, lsc)


def test_good_thresholds_scan_fewer_postings(knn, trained):
    import torch
    E = synth.spectrum_u8(300, 361, role="R")
    Ed = knn.DeviceCSR.from_host(E)
    idx = trained["idx"]
    c_plain = torch.zeros(1, dtype=torch.int64, device="cuda")
    pids, psc = knn.knn_join(idx, Ed, 5, s_groups=1, postings_scanned=c_plain)
    tau = (psc[:, 4].float() * 0.9).contiguous()
    c_l = torch.zeros(1, dtype=torch.int64, device="cuda")
    lids, lsc, st = knn.knn_join_learned(idx, None, Ed, 5, tau=tau, s_groups=1, postings_scanned=c_l)
    torch.cuda.synchronize()
    assert st["fallback_rows"] == 0
    assert torch.equal(pids, lids) and torch.equal(psc, lsc)
    assert int(c_l.item()) < int(c_plain.item())


def test_calibrate_picks_the_ratio_quantile(knn, trained):
    m = knn.ThresholdModel(seed=7)
    m.set_params(trained["model"].get_params())
    V = synth.spectrum_u8(800, 371, role="R")
    _, vsc = knn.knn_join(trained["idx"], knn.DeviceCSR.from_host(V), 5)
    kth = vsc[:, 4].float().contiguous()
    scale = m.calibrate(V, kth, 0.05)
    pred = m.predict(V).cpu().numpy()
    kk = kth.cpu().numpy()
    expect = L.calibrated_scale(kk, pred, 0.05)
    assert abs(scale - expect) <= 1e-5 * expect, (scale, expect)
    assert (pred * scale > kk).mean() <= 0.05 + 1e-9
    # the multiplier travels with the parameters and is the learned join's default
    m2 = knn.ThresholdModel(seed=8)
    m2.set_params(m.get_params())
    W = synth.spectrum_u8(300, 372, role="R")
    Wd = knn.DeviceCSR.from_host(W)
    a = knn.knn_join_learned(trained["idx"], m2, Wd, 5)
    b = knn.knn_join_learned(trained["idx"], m, Wd, 5, tau_scale=scale)
    assert a[2]["fallback_rows"] == b[2]["fallback_rows"]
    pids, psc = knn.knn_join(trained["idx"], Wd, 5)
    import torch
    assert torch.equal(a[0], pids) and torch.equal(a[1], psc)
    m.close()
    m2.close()


def test_calibrated_fallback_rate_on_fresh_queries(knn, trained):
    m = knn.ThresholdModel(seed=9)
    m.set_params(trained["model"].get_params())
    V = synth.spectrum_u8(1500, 381, role="R")
    _, vsc = knn.knn_join(trained["idx"], knn.DeviceCSR.from_host(V), 5)
    m.calibrate(V, vsc[:, 4].float().contiguous(), 0.02)
    E = synth.spectrum_u8(1500, 382, role="R")
    _, _, st = knn.knn_join_learned(trained["idx"], m, knn.DeviceCSR.from_host(E), 5)
    # a 2 % target on 1,500 fresh rows: far from the 100 % an uncalibrated over-prediction gives
    assert st["fallback_rows"] <= 0.08 * E.n_rows, st
    m.close()


def test_trained_model_gains_over_the_plain_join(knn, trained):
    """What the trained network gains: with its own calibrated predictions as start
    thresholds, the learned join returns exactly the plain join's result on fresh
    queries, falls back on about the calibrated share of rows, and scans fewer
    postings than the plain join, whose running threshold starts at 0."""
    import torch
    idx = trained["idx"]
    m = knn.ThresholdModel(seed=13)
    m.set_params(trained["model"].get_params())
    V = synth.spectrum_u8(1500, 391, role="R")           # held-out calibration queries
    _, vsc = knn.knn_join(idx, knn.DeviceCSR.from_host(V), 5)
    scale = m.calibrate(V, vsc[:, 4].float().contiguous(), 0.02)
    assert 0.0 < scale < 2.0
    E = synth.spectrum_u8(1000, 392, role="R")           # fresh queries
    Ed = knn.DeviceCSR.from_host(E)
    c_plain = torch.zeros(1, dtype=torch.int64, device="cuda")
    pids, psc = knn.knn_join(idx, Ed, 5, s_groups=1, postings_scanned=c_plain)
    c_learned = torch.zeros(1, dtype=torch.int64, device="cuda")
    lids, lsc, st = knn.knn_join_learned(idx, m, Ed, 5, s_groups=1, postings_scanned=c_learned)
    torch.cuda.synchronize()
    assert torch.equal(pids, lids) and torch.equal(psc, lsc)
    # a 2 % target: the 1,000 fresh rows' fallback count stays within binomial noise of it
    assert st["fallback_rows"] <= 0.05 * E.n_rows, st
    plain, learned = int(c_plain.item()), int(c_learned.item())   # fallback reruns included
    assert learned < plain, (learned, plain)
    m.close()
