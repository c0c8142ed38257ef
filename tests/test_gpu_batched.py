"""The batched form: many joins in one persistent launch (optionally a CUDA graph)
return exactly what separate knn_join calls return."""
import numpy as np
import pytest

from paper_1011_2807_gb300 import synth
import compare
from cases import long_row_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def knn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1011_2807_gb300 as knn
    knn.lib()
    return knn


@pytest.fixture(scope="module")
def jobs(knn):
    rng = np.random.default_rng(44)
    out = []
    for j in range(9):
        n_s = int(rng.choice([3000, 9000, 20000, 45000]))
        n_r = int(rng.choice([0, 1, 40, 300, 2500])) if j else 0
        k = int(rng.choice([1, 5, 10, 20, 50]))
        S = synth.spectrum_u8(n_s, 500 + j, role="S")
        R = synth.spectrum_u8(n_r, 600 + j, role="R")
        idx = knn.knn_join_build_index(S, block_size=int(rng.choice([2048, 4096, 16384])))
        out.append(dict(S=S, R=R, k=k, idx=idx, Rd=knn.DeviceCSR.from_host(R)))
    yield out
    for j in out:
        j["idx"].close()


def reference(knn, jobs):
    import torch
    res = []
    for j in jobs:
        ids, sc = knn.knn_join(j["idx"], j["Rd"], j["k"])
        res.append((ids.cpu(), sc.cpu()))
    torch.cuda.synchronize()
    return res


@pytest.mark.parametrize("bpg", [0, 1, 3, 100])
def test_batched_equals_separate_joins(knn, jobs, bpg):
    ref = reference(knn, jobs)
    outs = knn.knn_join_batched([(j["idx"], j["Rd"], j["k"]) for j in jobs], blocks_per_group=bpg)
    for (ids, sc), (rid, rsc) in zip(outs, ref):
        assert np.array_equal(ids.cpu().numpy(), rid.numpy())
        assert np.array_equal(sc.cpu().numpy(), rsc.numpy())


def test_batched_against_oracle(knn, jobs, oracle_mod):
    outs = knn.knn_join_batched([(j["idx"], j["Rd"], j["k"]) for j in jobs])
    for j, (ids, sc) in zip(jobs[:5], outs[:5]):
        eids, esc, _ = oracle_mod.iib_join(j["R"], j["S"], j["k"], threads=8)
        compare.assert_exact(ids.cpu().numpy(), sc.cpu().numpy(), eids, esc, "batched")


def test_graph_replay(knn, jobs):
    import torch
    ref = reference(knn, jobs)
    b = knn.Batch([(j["idx"], j["Rd"], j["k"]) for j in jobs], use_graph=True)
    info = b.info()
    assert info["graph"] == 1 and info["work_items"] > 0
    for _ in range(3):
        for ids, sc in b.outputs:
            ids.fill_(-5)
        outs = b.launch()
        torch.cuda.synchronize()
        for (ids, sc), (rid, rsc) in zip(outs, ref):
            assert np.array_equal(ids.cpu().numpy(), rid.numpy())
            assert np.array_equal(sc.cpu().numpy(), rsc.numpy())
    # new query contents of the same shape: a replay joins the new contents
    j = jobs[3]
    R2 = synth.spectrum_u8(j["R"].n_rows, 777, role="R", nnz=np.diff(j["R"].indptr))
    j["Rd"].indices.copy_(knn.DeviceCSR.from_host(R2).indices)
    j["Rd"].values.copy_(knn.DeviceCSR.from_host(R2).values)
    outs = b.launch()
    torch.cuda.synchronize()
    rid, rsc = knn.knn_join(j["idx"], j["Rd"], j["k"])
    assert np.array_equal(outs[3][0].cpu().numpy(), rid.cpu().numpy())
    b.close()


def test_batched_float_jobs(knn, oracle_mod):
    js = []
    for j in range(3):
        S = synth.uniform_f32(4000 + 1000 * j, 800, 5, 40, 900 + j)
        R = synth.uniform_f32(50, 800, 5, 40, 950 + j)
        js.append((S, R, 10, knn.knn_join_build_index(S, block_size=2048)))
    outs = knn.knn_join_batched([(idx, knn.DeviceCSR.from_host(R), k) for S, R, k, idx in js])
    for (S, R, k, idx), (ids, sc) in zip(js, outs):
        eids, esc, _ = oracle_mod.iib_join(R, S, k, threads=8)
        compare.assert_close(R, S, list(range(R.n_rows)), ids.cpu().numpy(), sc.cpu().numpy(), eids, esc,
                             what="batched f32")
        idx.close()


def test_batched_errors(knn, jobs):
    from paper_1011_2807_gb300.binding import KNN_EINVAL, KNN_EUNSUPPORTED, KnnError
    S = synth.uniform_f32(3000, 10000, 5, 40, 991)
    fidx = knn.knn_join_build_index(S)
    R = synth.uniform_f32(10, 10000, 5, 40, 992)
    with pytest.raises(KnnError) as e:      # mixed dtypes
        knn.knn_join_batched([(jobs[0]["idx"], jobs[0]["Rd"], 5), (fidx, knn.DeviceCSR.from_host(R), 5)])
    assert e.value.status == KNN_EINVAL
    with pytest.raises(KnnError) as e:      # a 256-vector S block cannot feed 512 threads
        tiny = knn.knn_join_build_index(synth.spectrum_u8(200, 993, role="S"), block_size=256)
        knn.knn_join_batched([(tiny, jobs[1]["Rd"], 5)])
    assert e.value.status == KNN_EUNSUPPORTED
    fidx.close()


def test_autotune_picks_a_valid_config(knn, tmp_path, monkeypatch):
    from paper_1011_2807_gb300 import autotune
    monkeypatch.setenv("KNN_TUNE_CACHE", str(tmp_path / "tune.json"))
    S = synth.spectrum_u8(30000, 1201, role="S")
    R = synth.spectrum_u8(100, 1202, role="R")
    best = autotune.tune(S, R, 5, threads=512, reps=1, max_trials=6)
    assert 4 * best["threads"] <= best["block_size"] <= 64 * best["threads"] and best["ms"] > 0
    got = autotune.lookup(S.n_rows, R.n_rows, R.nnz / R.n_rows, 5, "u8")
    assert got["block_size"] == best["block_size"]
    # the default margin stays unless one of the alternatives times faster
    assert got["level_margin"] in (autotune.DEFAULT["level_margin"],) + autotune.MARGINS


def test_bounded_wait_reports_timeout(knn, jobs):
    """A work item that waits for a flag nothing sets gives up after its bounded spin and
    the host reads KNN_ETIMEOUT; the GPU context stays usable afterwards."""
    import torch
    from paper_1011_2807_gb300.binding import KNN_ETIMEOUT, KnnError
    multi = [j for j in jobs if j["idx"].info()["n_blocks"] > 1 and j["R"].n_rows > 0]
    assert multi
    j = multi[0]
    b = knn.Batch([(j["idx"], j["Rd"], j["k"])], use_graph=False, blocks_per_group=1, wait_spins=200,
                  test_never_publish=True)
    b.launch()
    with pytest.raises(KnnError) as e:
        b.check()
    assert e.value.status == KNN_ETIMEOUT
    b.close()
    # the context still works: a normal batch afterwards is exact
    ids, sc = knn.knn_join(j["idx"], j["Rd"], j["k"])
    (bids, bsc), = knn.knn_join_batched([(j["idx"], j["Rd"], j["k"])], blocks_per_group=1)
    torch.cuda.synchronize()
    assert torch.equal(ids, bids) and torch.equal(sc, bsc)


@pytest.mark.parametrize("dtype", ["u8", "f32"])
@pytest.mark.parametrize("bpg", [0, 1])
def test_batched_long_rows_split(knn, oracle_mod, dtype, bpg):
    """Jobs whose longest rows need a layout above 110 KB run as two sub-jobs: the rows
    that fit a layout within 110 KB in a persistent launch at two CTAs per SM (with the
    jobs that fit it whole), the long rows in a launch of their own.  Results against the
    oracle (uint8 bit-exact), with one S-block group per row and with one group per S
    block (rows then wait for their previous group within either launch)."""
    import torch
    S, R, Rshort = long_row_case(dtype, 1301)
    idx = knn.knn_join_build_index(S, block_size=16384)
    jobs = [(idx, knn.DeviceCSR.from_host(R), 9), (idx, knn.DeviceCSR.from_host(Rshort), 5),
            (idx, knn.DeviceCSR.from_host(R), 20)]
    hosts = [R, Rshort, R]
    b = knn.Batch(jobs, use_graph=True, blocks_per_group=bpg)
    passes = 2 if dtype == "f32" else 1
    assert b.info()["kernels_per_launch"] == 2 * passes   # the small-layout launch and the full-layout one
    outs = b.launch()
    b.check()
    torch.cuda.synchronize()
    for (ix, Rd, k), Rh, (ids, sc) in zip(jobs, hosts, outs):
        eids, esc, _ = oracle_mod.bf_join(Rh, S, k, threads=8)
        if dtype == "u8":
            compare.assert_exact(ids.cpu().numpy(), sc.cpu().numpy(), eids, esc, f"batched long rows k={k}")
        else:
            compare.assert_close(Rh, S, list(range(Rh.n_rows)), ids.cpu().numpy(), sc.cpu().numpy(), eids, esc,
                                 what=f"batched long rows k={k}")
    b.close()
    idx.close()


def test_batched_row_grown_since_creation(knn):
    """A batch's layouts are sized for R's row lengths when it is made.  A row that has
    grown past its layout since is not joined -- the kernel compares the row's length
    with the layout before it reads a feature of it -- and knn_batch_check reports
    KNN_EINVAL; with the lengths restored the batch returns the same results again."""
    import torch
    from paper_1011_2807_gb300.binding import KNN_EINVAL, KnnError
    S, R, _ = long_row_case("u8", 1311)
    idx = knn.knn_join_build_index(S, block_size=16384)
    Rd = knn.DeviceCSR.from_host(R)
    b = knn.Batch([(idx, Rd, 5)], use_graph=False, blocks_per_group=1)
    b.launch()
    b.check()
    ref = [t.clone() for t in b.outputs[0]]
    # rows 30-32 are the long ones, row 33 a short one: moving row 33's start back to row
    # 32's start empties row 32 and gives row 33 its 2,500 features too
    assert int(R.indptr[33] - R.indptr[32]) == 2500 and int(R.indptr[34] - R.indptr[33]) < 200
    Rd.indptr[33] = int(R.indptr[32])
    b.launch()
    with pytest.raises(KnnError) as e:
        b.check()
    assert e.value.status == KNN_EINVAL
    Rd.indptr[33] = int(R.indptr[33])
    b.launch()
    b.check()
    torch.cuda.synchronize()
    assert torch.equal(b.outputs[0][0], ref[0]) and torch.equal(b.outputs[0][1], ref[1])
    b.close()
    idx.close()
