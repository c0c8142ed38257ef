"""The batched, learned-threshold and float workloads at their full sizes, in the launch
configuration the benchmark uses, checked against the CPU oracle on sampled rows.

* 64 uneven joins (|R| log-U[100, 50k], |S| log-U[1e4, 1e6], k in {1,5,10,20,50}) in one
  persistent launch from a CUDA graph: every job equals its separate knn_join, and two
  sampled rows per job equal the oracle bit for bit.
* The learned threshold at |S| = 5,000,000 with 1,000,000 evaluation queries, k = 10:
  the learned form equals the plain join on every row, and 48 sampled rows of both
  equal the oracle bit for bit.
* The float workload at |S| = 10,000,000 (d = 50,000, Zipf ids, L2-normalised, k = 20):
  the first 65,536 of its 1,000,000 query rows (one generator chunk, identical to the
  full set's first rows) through the plain IIIB and IIB joins, the learned form and a
  batched launch of 8 uneven jobs; 24 sampled rows of each within the float tolerance
  of the fp64 oracle.

Inputs are drawn by processes of their own (spawned) so that the whole file runs in a
few minutes."""
import os

import numpy as np
import pytest

from paper_1011_2807_gb300 import synth
import compare

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

PROCS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def knn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1011_2807_gb300 as knn
    knn.lib()
    return knn


def test_config3_full_size_batched(knn, oracle_mod):
    import torch
    spec = synth.config3_jobs()
    data = synth.generate([("config3_job_data", (js,)) for js in spec], processes=PROCS)
    jobs = []
    for (R, S, k) in data:
        idx = knn.knn_join_build_index(S, block_size=16384)
        jobs.append((idx, knn.DeviceCSR.from_host(R), k))
    b = knn.Batch(jobs, use_graph=True, threads=512)
    b.launch()
    torch.cuda.synchronize()
    rng = np.random.default_rng(33)
    for j, ((R, S, k), (idx, Rd, _), (bids, bsc)) in enumerate(zip(data, jobs, b.outputs)):
        ids, sc = knn.knn_join(idx, Rd, k)
        assert torch.equal(ids, bids) and torch.equal(sc, bsc), f"job {j}: batched != separate"
        rows = np.sort(rng.choice(R.n_rows, size=min(2, R.n_rows), replace=False))
        eids, esc, _ = oracle_mod.bf_join(R.take_rows(rows), S, k, threads=0)
        compare.assert_exact(bids.cpu().numpy()[rows], bsc.cpu().numpy()[rows], eids, esc,
                             f"config3 job {j} (|R|={R.n_rows}, |S|={S.n_rows}, k={k})")
    b.close()
    for idx, _, _ in jobs:
        idx.close()


def test_config4_full_size_learned(knn, oracle_mod):
    import torch
    T, E, S = synth.generate([
        ("spectrum_u8", (200000, synth.config_seed(4, "train")), {"role": "R"}),
        ("spectrum_u8", (1000000, synth.config_seed(4, "eval")), {"role": "R"}),
        ("spectrum_u8", (5000000, synth.config_seed(4, "S")), {"role": "S"}),
    ], processes=3)
    k = 10
    assert (T.n_rows, E.n_rows, S.n_rows) == (200000, 1000000, 5000000)
    idx = knn.knn_join_build_index(S)
    Td, Ed = knn.DeviceCSR.from_host(T), knn.DeviceCSR.from_host(E)
    _, tsc = knn.knn_join(idx, Td, k)
    lab = tsc[:, k - 1].float()
    n_fit = T.n_rows - 10000
    model = knn.ThresholdModel(seed=1)
    model.train(T.slice_rows(0, n_fit), lab[:n_fit].contiguous(), epochs=15, batch=512, quantile=0.1, seed=1)
    model.calibrate(T.slice_rows(n_fit, T.n_rows), lab[n_fit:].contiguous(), 0.002)
    pids, psc = knn.knn_join(idx, Ed, k)
    lids, lsc, st = knn.knn_join_learned(idx, model, Ed, k)
    torch.cuda.synchronize()
    assert torch.equal(pids, lids) and torch.equal(psc, lsc)
    assert st["fallback_rows"] < E.n_rows // 20
    rows = np.sort(np.random.default_rng(44).choice(E.n_rows, size=48, replace=False))
    eids, esc, _ = oracle_mod.bf_join(E.take_rows(rows), S, k, threads=0)
    compare.assert_exact(pids.cpu().numpy()[rows], psc.cpu().numpy()[rows], eids, esc, "config4 plain")
    compare.assert_exact(lids.cpu().numpy()[rows], lsc.cpu().numpy()[rows], eids, esc, "config4 learned")
    model.close()
    idx.close()


def test_config5_full_size_forms(knn, oracle_mod):
    import torch
    k = 20
    S = synth.zipf_f32(10000000, synth.config_seed(5, "S"), processes=PROCS)
    R = synth.zipf_f32(synth.ZIPF_CHUNK, synth.config_seed(5, "R"))
    A = synth.zipf_f32(12000, synth.config_seed(5, "train"))
    assert S.n_rows == 10000000 and R.n_rows == 65536
    rows = np.sort(np.random.default_rng(55).choice(R.n_rows, size=24, replace=False))
    eids, esc, _ = oracle_mod.bf_join(R.take_rows(rows), S, k, threads=0)
    idx = knn.knn_join_build_index(S)
    Rd = knn.DeviceCSR.from_host(R)

    def check(ids, sc, what):
        compare.assert_close(R, S, rows, ids.cpu().numpy()[rows], sc.cpu().numpy()[rows], eids, esc,
                             what=f"config5 {what}")

    for mode in ("iiib", "iib"):
        ids, sc = knn.knn_join(idx, Rd, k, mode=mode)
        check(ids, sc, mode)
    Ad = knn.DeviceCSR.from_host(A)
    _, asc = knn.knn_join(idx, Ad, k)
    kth = asc[:, k - 1].float()
    model = knn.ThresholdModel(seed=5)
    model.train(A.slice_rows(0, 9000), kth[:9000].contiguous(), epochs=15, batch=512, quantile=0.1, seed=5)
    model.calibrate(A.slice_rows(9000, A.n_rows), kth[9000:].contiguous(), 0.002)
    lids, lsc, _ = knn.knn_join_learned(idx, model, Rd, k)
    check(lids, lsc, "learned")
    model.close()
    cuts = [0] + sorted(int(R.n_rows * f) for f in (0.02, 0.05, 0.1, 0.2, 0.35, 0.55, 0.75)) + [R.n_rows]
    parts = [knn.DeviceCSR.from_host(R.slice_rows(a, b)) for a, b in zip(cuts[:-1], cuts[1:])]
    b = knn.Batch([(idx, P, k) for P in parts], use_graph=True)
    b.launch()
    torch.cuda.synchronize()
    check(torch.cat([o[0] for o in b.outputs]), torch.cat([o[1] for o in b.outputs]), "batched")
    b.close()
    idx.close()
