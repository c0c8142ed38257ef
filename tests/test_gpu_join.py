"""Parity of the CUDA join (through the C ABI) with the CPU oracle."""
import numpy as np
import pytest

from paper_1011_2807_gb300 import synth
import compare
from cases import long_row_case, random_u8
import goldens
import refdefs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def knn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1011_2807_gb300 as knn
    knn.lib()
    return knn


def run(knn, S, R, k, device_r=True, **kw):
    import torch
    bopts = {x: kw.pop(x) for x in ("block_size", "n_levels") if x in kw}
    idx = knn.knn_join_build_index(S, **bopts)
    Rin = knn.DeviceCSR.from_host(R) if device_r else R
    ids, sc = knn.knn_join(idx, Rin, k, **kw)
    torch.cuda.synchronize()
    out = (ids.cpu().numpy(), sc.cpu().numpy())
    idx.close()
    return out


# ----------------------------------------------------------------------------------
# hand-worked examples
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("mode", ["iib", "iiib"])
def test_h1(knn, oracle_mod, mode):
    g = goldens.load("h1_topk.txt")
    for k, exp in g["cases"]:
        ids, sc = run(knn, g["S"], g["R"], k, mode=mode)
        eids, esc = goldens.expected_arrays(exp, g["R"].n_rows, k)
        np.testing.assert_array_equal(ids, eids)
        np.testing.assert_array_equal(sc, esc)


def test_h2(knn, oracle_mod):
    g = goldens.load("h2_iiib_trace.txt")
    (k, exp), = g["cases"]
    ids, sc = run(knn, g["S"], g["R"], k, block_size=256)
    eids, esc = goldens.expected_arrays(exp, g["R"].n_rows, k)
    np.testing.assert_array_equal(ids, eids)
    np.testing.assert_array_equal(sc, esc)


# ----------------------------------------------------------------------------------
# uint8: bit-exact against the oracle
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("mode", ["iib", "iiib"])
@pytest.mark.parametrize("bs,nl", [(256, 1), (256, 16), (1024, 4), (2048, 32)])
@pytest.mark.parametrize("k", [1, 5, 64])
def test_spectrum_u8_exact(knn, oracle_mod, mode, bs, nl, k):
    S = synth.spectrum_u8(5000, 31, role="S")          # 20 blocks of 256: a ragged tail
    R = synth.spectrum_u8(120, 32, role="R")
    eids, esc, _ = oracle_mod.iib_join(R, S, k, threads=8)
    ids, sc = run(knn, S, R, k, mode=mode, block_size=bs, n_levels=nl)
    compare.assert_exact(ids, sc, eids, esc, f"mode={mode} bs={bs} nl={nl} k={k}")


@pytest.mark.parametrize("groups", [1, 2, 7, 0])
def test_s_groups(knn, oracle_mod, groups):
    S = synth.spectrum_u8(9000, 41, role="S")
    R = synth.spectrum_u8(60, 42, role="R")
    eids, esc, _ = oracle_mod.iib_join(R, S, 10, threads=8)
    ids, sc = run(knn, S, R, 10, block_size=512, s_groups=groups)
    compare.assert_exact(ids, sc, eids, esc, f"groups={groups}")


@pytest.mark.parametrize("bpl", [1, 3, 7, 100])
@pytest.mark.parametrize("mode", ["iib", "iiib"])
def test_block_synchronous_launches(knn, oracle_mod, bpl, mode):
    # one group per row: rows carry their top-k across launches of bpl S blocks
    S = synth.spectrum_u8(5000, 131, role="S")      # 20 blocks of 256
    R = synth.spectrum_u8(90, 132, role="R")
    eids, esc, _ = oracle_mod.iib_join(R, S, 7, threads=8)
    ids, sc = run(knn, S, R, 7, mode=mode, block_size=256, s_groups=1, blocks_per_launch=bpl)
    compare.assert_exact(ids, sc, eids, esc, f"bpl={bpl} {mode}")


@pytest.mark.parametrize("threads", [128, 256, 512, 1024])
def test_threads(knn, oracle_mod, threads):
    S = synth.spectrum_u8(6000, 51, role="S")
    R = synth.spectrum_u8(50, 52, role="R")
    eids, esc, _ = oracle_mod.iib_join(R, S, 5, threads=8)
    ids, sc = run(knn, S, R, 5, block_size=4096, threads=threads)
    compare.assert_exact(ids, sc, eids, esc, f"threads={threads}")


@pytest.mark.parametrize("mode", ["iib", "iiib"])
def test_largest_s_block(knn, oracle_mod, mode):
    """S blocks of KNN_MAX_BLOCK = 32,768 vectors (a 128 KB accumulator, 1,024 threads,
    one CTA per SM), three blocks with a ragged last one, bit-exact."""
    S = synth.spectrum_u8(70000, 151, role="S")
    R = synth.spectrum_u8(120, 152, role="R")
    eids, esc, _ = oracle_mod.iib_join(R, S, 7, threads=8)
    ids, sc = run(knn, S, R, 7, mode=mode, block_size=32768)
    compare.assert_exact(ids, sc, eids, esc, f"block 32768 {mode}")


@pytest.mark.parametrize("dtype", ["u8", "f32"])
def test_long_rows_run_in_a_launch_of_their_own(knn, oracle_mod, dtype):
    """A few query rows too long for a two-CTA-per-SM shared-memory layout among short
    ones: each S-block launch runs the short rows with the small layout and the long rows
    with the full one.  Results against the oracle (uint8 bit-exact), for S-block-
    synchronous launches, IIB, one launch over all S blocks and the fp32 path; the extra
    launches show that the split ran."""
    import torch
    from paper_1011_2807_gb300.binding import KNN_STATS
    S, R, Rshort = long_row_case(dtype, 961)
    k = 9
    eids, esc, _ = oracle_mod.bf_join(R, S, k, threads=8)
    idx = knn.knn_join_build_index(S, block_size=16384)
    assert idx.info()["n_blocks"] == 3
    Rd, Rsd = knn.DeviceCSR.from_host(R), knn.DeviceCSR.from_host(Rshort)
    for kw in (dict(blocks_per_launch=2), dict(blocks_per_launch=2, mode="iib"), dict(blocks_per_launch=100),
               dict(blocks_per_launch=1, fixed_point=False)):
        st = torch.zeros(len(KNN_STATS), dtype=torch.int64, device="cuda")
        ids, sc = knn.knn_join(idx, Rd, k, s_groups=1, stats=st, **kw)
        ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
        if dtype == "u8":
            compare.assert_exact(ids, sc, eids, esc, f"long rows {kw}")
        else:
            compare.assert_close(R, S, list(range(R.n_rows)), ids, sc, eids, esc, what=f"long rows {kw}")
        w = dict(zip(KNN_STATS, st.cpu().tolist()))
        assert w["block_steps"] >= R.n_rows * 3   # every row, every block
    if dtype == "u8":
        # one launch step: the split adds k_split_rows and the long rows' launch
        n0 = knn.knn_kernel_launch_count()
        knn.knn_join(idx, Rsd, k, s_groups=1, blocks_per_launch=100)
        n1 = knn.knn_kernel_launch_count()
        knn.knn_join(idx, Rd, k, s_groups=1, blocks_per_launch=100)
        n2 = knn.knn_kernel_launch_count()
        assert (n2 - n1) - (n1 - n0) == 2, (n0, n1, n2)
    idx.close()


@pytest.mark.parametrize("seed", range(4))
def test_random_small_dims_many_ties(knn, oracle_mod, seed):
    # few dimensions and weights in {1,2}: scores tie everywhere
    S = random_u8(700, 12, 6, 60 + seed, wmax=2)
    R = random_u8(40, 12, 6, 70 + seed, wmax=2)
    for k in (1, 3, 20, 64):
        eids, esc, _ = oracle_mod.bf_join(R, S, k, threads=8)
        ids, sc = run(knn, S, R, k, block_size=256)
        compare.assert_exact(ids, sc, eids, esc, f"ties k={k}")


def test_max_weights_and_long_rows(knn, oracle_mod):
    # weight 255 everywhere, R rows of up to 2,000 features, S rows of up to 300
    rng = np.random.default_rng(5)
    S = random_u8(1500, 4000, 300, 81, wmax=255, nnz_lo=200)
    R = random_u8(20, 4000, 2000, 82, wmax=255, nnz_lo=1500)
    S.values[:] = 255
    eids, esc, _ = oracle_mod.iib_join(R, S, 8, threads=8)
    ids, sc = run(knn, S, R, 8, block_size=512)
    compare.assert_exact(ids, sc, eids, esc, "max weights")


def test_config2_scaled(knn, oracle_mod):
    R, S, k = synth.config2(n_r=400, n_s=100000)
    eids, esc, _ = oracle_mod.iib_join(R, S, k, threads=8)
    for mode in ("iib", "iiib"):
        ids, sc = run(knn, S, R, k, mode=mode)
        compare.assert_exact(ids, sc, eids, esc, f"config2 scaled {mode}")


# ----------------------------------------------------------------------------------
# float32: 1e-5 relative, boundary ties allowed
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("mode", ["iib", "iiib"])
def test_config1_scaled_f32(knn, oracle_mod, mode):
    R, S, k = synth.config1(scale=0.2)
    eids, esc, _ = oracle_mod.iib_join(R, S, k, threads=8)
    ids, sc = run(knn, S, R, k, mode=mode, block_size=512)
    compare.assert_close(R, S, list(range(R.n_rows)), ids, sc, eids, esc, what=f"config1 {mode}")


def test_config1_full_f32(knn, oracle_mod):
    R, S, k = synth.config1()
    eids, esc, _ = oracle_mod.iib_join(R, S, k, threads=8)
    ids, sc = run(knn, S, R, k)
    compare.assert_close(R, S, list(range(R.n_rows)), ids, sc, eids, esc, what="config1 full")


def test_zipf_normalised_f32(knn, oracle_mod):
    S = synth.zipf_f32(3000, 91, dim=2000, nnz_hi=200)
    R = synth.zipf_f32(40, 92, dim=2000, nnz_hi=200)
    eids, esc, _ = oracle_mod.iib_join(R, S, 20, threads=8)
    for mode in ("iib", "iiib"):
        ids, sc = run(knn, S, R, 20, mode=mode, block_size=512)
        compare.assert_close(R, S, list(range(R.n_rows)), ids, sc, eids, esc, what=f"zipf {mode}")


def near_cut_f32(seed, k=20, dim=6000, base_nnz=1200, n_other=4000):
    """S made of scaled copies of one long vector V (base_nnz features) and partial
    copies, so that for ANY query r, score(r, c V) = c (r . V) orders the copies by c:
      * k copies with c in [1, 1 + 1e-6]: the true top-k, all within 1e-6 of the cut;
      * 30 copies with c in [1 - 2e-5, 1 - 1.2e-5]: the nearest non-neighbours, just
        outside the 1e-5 tolerance (returning one instead of a true neighbour fails);
      * n_other vectors holding 10-60 % of V's features at c in [0.3, 0.9] plus random
        other features (scores below 0.9 of the cut).
    The query rows overlap V heavily (800-1200 of its features plus others)."""
    rng = np.random.default_rng(seed)
    vd = np.sort(rng.choice(dim, base_nnz, replace=False))
    vw = rng.lognormal(0.0, 1.0, base_nnz)
    rows, tags = [], []
    for c in 1.0 + rng.uniform(0.0, 1e-6, k):
        rows.append(list(zip(vd.tolist(), (c * vw).tolist())))
        tags.append("top")
    for c in 1.0 - rng.uniform(1.2e-5, 2e-5, 30):
        rows.append(list(zip(vd.tolist(), (c * vw).tolist())))
        tags.append("near")
    others = np.setdiff1d(np.arange(dim), vd)
    for _ in range(n_other):
        keep = rng.random(base_nnz) < rng.uniform(0.1, 0.6)
        ex = rng.choice(others, size=int(rng.integers(0, 300)), replace=False)
        c = rng.uniform(0.3, 0.9)
        f = dict(zip(vd[keep].tolist(), (c * vw[keep]).tolist()))
        f.update(zip(ex.tolist(), rng.lognormal(0.0, 1.0, ex.size).tolist()))
        rows.append(sorted(f.items()))
        tags.append("other")
    order = rng.permutation(len(rows))
    S = synth.from_rows([rows[i] for i in order], dim, np.float32)
    tags = np.asarray(tags)[order]
    qs = []
    for _ in range(8):
        keep = rng.random(base_nnz) < rng.uniform(0.65, 1.0)
        ex = rng.choice(others, size=int(rng.integers(0, 200)), replace=False)
        f = dict(zip(vd[keep].tolist(), rng.lognormal(0.0, 1.0, int(keep.sum())).tolist()))
        f.update(zip(ex.tolist(), rng.lognormal(0.0, 1.0, ex.size).tolist()))
        qs.append(sorted(f.items()))
    return synth.from_rows(qs, dim, np.float32), S, tags


def test_float_weights_across_binades(knn, oracle_mod):
    """Float weights from 1e-12 to 1e12, a fifth of them just below a power of two (the
    scan's rounded-up 17-bit weights then carry into the exponent), against the fp64
    oracle in every form of the join."""
    rng = np.random.default_rng(777)
    dim = 3000

    def draw(n, seed):
        r = np.random.default_rng(seed)
        rows = []
        for _ in range(n):
            m = int(r.integers(5, 120))
            d = np.sort(r.choice(dim, m, replace=False))
            w = 10.0 ** r.uniform(-12, 12, m)
            edge = r.random(m) < 0.2
            w[edge] = (2.0 - 2.0 ** -20) * 2.0 ** np.round(np.log2(w[edge]))
            rows.append(list(zip(d.tolist(), w.astype(np.float32).tolist())))
        return synth.from_rows(rows, dim, np.float32)

    S, R = draw(5000, 778), draw(60, 779)
    k = 12
    eids, esc, _ = oracle_mod.bf_join(R, S, k, threads=8)
    idx = knn.knn_join_build_index(S, block_size=1024)
    Rd = knn.DeviceCSR.from_host(R)
    for kw in (dict(mode="iib"), dict(mode="iiib"), dict(mode="iiib", level_margin=1.0, s_groups=1),
               dict(mode="iiib", s_groups=3), dict(mode="bf")):
        ids, sc = knn.knn_join(idx, Rd, k, **kw)
        compare.assert_close(R, S, list(range(R.n_rows)), ids.cpu().numpy(), sc.cpu().numpy(), eids, esc,
                             what=f"binades {kw}")
    idx.close()


@pytest.mark.parametrize("seed", [501, 502])
def test_float_long_rows_neighbours_at_the_cut(knn, oracle_mod, seed):
    """Long, heavily overlapping float rows (n = 800-1,200 shared features, so the fp32
    sums carry up to ~1e-4 of worst-case rounding) with the true neighbours within 1e-6
    of the k-th score and the nearest non-neighbours 1.2e-5 to 2e-5 below it: every
    form of the join, including the Section 4.4 cut at its most aggressive margin,
    must return exactly the k true neighbours."""
    R, S, tags = near_cut_f32(seed)
    k = 20
    eids, esc, _ = oracle_mod.bf_join(R, S, k, threads=8)
    assert all(set(tags[eids[i]]) == {"top"} for i in range(R.n_rows))   # the construction holds
    idx = knn.knn_join_build_index(S, block_size=256, n_levels=32)
    Rd = knn.DeviceCSR.from_host(R)
    for kw in (dict(mode="iib"), dict(mode="iiib"), dict(mode="iiib", level_margin=1.0),
               dict(mode="iiib", level_margin=1.0, s_groups=1), dict(mode="iiib", s_groups=4),
               dict(mode="bf")):
        ids, sc = knn.knn_join(idx, Rd, k, **kw)
        ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
        compare.assert_close(R, S, list(range(R.n_rows)), ids, sc, eids, esc, what=f"near cut {kw}")
        for i in range(R.n_rows):
            assert set(ids[i].tolist()) == set(eids[i].tolist()), (kw, i)
    idx.close()


@pytest.mark.parametrize("mode", ["iib", "iiib"])
def test_float_fixed_point_scan(knn, oracle_mod, mode):
    """Float joins sum their scans in fixed point, and rows whose fixed-point error is
    not small enough against their own scores are joined again in fp32.  Both sums (and
    the batched form) agree with the fp64 oracle within the float tolerance, and the
    fixed-point path ran for most (row, launch) pairs."""
    import torch
    from paper_1011_2807_gb300.binding import KNN_STATS
    S = synth.zipf_f32(12000, 931, dim=3000, nnz_hi=400)
    R = synth.zipf_f32(150, 932, dim=3000, nnz_hi=400)
    k = 15
    eids, esc, _ = oracle_mod.bf_join(R, S, k, threads=8)
    idx = knn.knn_join_build_index(S, block_size=512)          # 24 S blocks
    Rd = knn.DeviceCSR.from_host(R)
    n_blocks = idx.info()["n_blocks"]
    n_launch = -(-n_blocks // 3)
    nonempty = int((np.diff(R.indptr) > 0).sum())
    for fixed in (True, False):
        st = torch.zeros(len(KNN_STATS), dtype=torch.int64, device="cuda")
        ids, sc = knn.knn_join(idx, Rd, k, mode=mode, s_groups=1, blocks_per_launch=3, fixed_point=fixed,
                               stats=st)
        compare.assert_close(R, S, list(range(R.n_rows)), ids.cpu().numpy(), sc.cpu().numpy(), eids, esc,
                             what=f"fixed_point={fixed} {mode}")
        w = dict(zip(KNN_STATS, st.cpu().tolist()))
        assert w["block_steps"] >= nonempty * n_blocks           # re-joined rows add theirs
        if fixed:
            assert w["fixed_point_rows"] > 0.9 * nonempty * n_launch, w
        else:
            assert w["fixed_point_rows"] == 0 and w["block_steps"] == nonempty * n_blocks
    b = knn.Batch([(idx, knn.DeviceCSR.from_host(R.slice_rows(0, 60)), k),
                   (idx, knn.DeviceCSR.from_host(R.slice_rows(60, 150)), k)], mode=mode, blocks_per_group=5,
                  threads=128, use_graph=True)
    b.launch()
    torch.cuda.synchronize()
    ids = torch.cat([o[0] for o in b.outputs]).cpu().numpy()
    sc = torch.cat([o[1] for o in b.outputs]).cpu().numpy()
    compare.assert_close(R, S, list(range(R.n_rows)), ids, sc, eids, esc, what=f"batched fixed point {mode}")
    b.close()
    idx.close()


def test_float_fixed_point_rejoins_imprecise_rows(knn, oracle_mod):
    """Rows whose L2 norm comes mostly from a dimension no S vector has: the fixed-point
    scale (set by |r| max|s|) is then too coarse for their small scores, so every such
    row must be flagged and joined again in fp32 -- with results within the float
    tolerance of the oracle, for the plain and the batched form."""
    import torch
    from paper_1011_2807_gb300.binding import KNN_STATS
    dim = 3001
    S = synth.zipf_f32(6000, 941, dim=3000, nnz_hi=200)
    S = synth.CSR(S.indptr, S.indices, S.values, dim)          # dimension 3000 stays empty in S
    rng = np.random.default_rng(942)
    rows = []
    for i in range(40):
        d = np.sort(rng.choice(3000, 30, replace=False))
        w = rng.lognormal(0.0, 1.0, 30) * 1e-4
        f = list(zip(d.tolist(), w.tolist())) + [(3000, 1e4)]   # |r| ~ 1e4, scores ~ 1e-5
        rows.append(f)
    R = synth.from_rows(rows, dim, np.float32)
    k = 10
    eids, esc, _ = oracle_mod.bf_join(R, S, k, threads=8)
    idx = knn.knn_join_build_index(S, block_size=1024)
    Rd = knn.DeviceCSR.from_host(R)
    st = torch.zeros(len(KNN_STATS), dtype=torch.int64, device="cuda")
    ids, sc = knn.knn_join(idx, Rd, k, s_groups=1, blocks_per_launch=2, stats=st)
    compare.assert_close(R, S, list(range(R.n_rows)), ids.cpu().numpy(), sc.cpu().numpy(), eids, esc,
                         what="re-joined rows")
    w = dict(zip(KNN_STATS, st.cpu().tolist()))
    assert w["block_steps"] == 2 * R.n_rows * idx.info()["n_blocks"], w   # every row joined twice
    b = knn.Batch([(idx, Rd, k)], blocks_per_group=2, threads=256, use_graph=False)
    b.launch()
    torch.cuda.synchronize()
    compare.assert_close(R, S, list(range(R.n_rows)), b.outputs[0][0].cpu().numpy(),
                         b.outputs[0][1].cpu().numpy(), eids, esc, what="batched re-joined rows")
    b.close()
    idx.close()


def test_batched_fp32_pass_takes_only_flagged_rows(knn, oracle_mod):
    """Rows too imprecise for fixed point (a large weight in a dimension S never uses)
    interleaved with ordinary rows, in two jobs with one S-block group per block: the
    batched fp32 pass claims its items in runs of 32 and joins only the flagged rows,
    every group of them; results within the float tolerance of the oracle, and the work
    counters show the flagged rows joined twice, as many as the plain join re-joins."""
    import torch
    from paper_1011_2807_gb300.binding import KNN_STATS
    dim = 3001
    S = synth.zipf_f32(6000, 943, dim=3000, nnz_hi=200)
    S = synth.CSR(S.indptr, S.indices, S.values, dim)          # dimension 3000 stays empty in S
    rng = np.random.default_rng(944)
    rows, flagged = [], []
    for i in range(150):
        d = np.sort(rng.choice(3000, 30, replace=False))
        if rng.random() < 0.2:
            w = rng.lognormal(0.0, 1.0, 30) * 1e-4
            rows.append(list(zip(d.tolist(), w.tolist())) + [(3000, 1e4)])   # scores ~1e-5 of |r|
            flagged.append(i)
        else:
            rows.append(list(zip(d.tolist(), rng.lognormal(0.0, 1.0, 30).tolist())))
    R = synth.from_rows(rows, dim, np.float32)
    k = 10
    eids, esc, _ = oracle_mod.bf_join(R, S, k, threads=8)
    idx = knn.knn_join_build_index(S, block_size=1024)
    nb = idx.info()["n_blocks"]
    parts = [(0, 70), (70, 150)]
    jobs = [(idx, knn.DeviceCSR.from_host(R.slice_rows(a, b)), k) for a, b in parts]
    st = torch.zeros(len(KNN_STATS), dtype=torch.int64, device="cuda")
    b = knn.Batch(jobs, blocks_per_group=1, threads=256, use_graph=False, stats=st)
    b.launch()
    b.check()
    ids = np.concatenate([o[0].cpu().numpy() for o in b.outputs])
    sc = np.concatenate([o[1].cpu().numpy() for o in b.outputs])
    compare.assert_close(R, S, list(range(R.n_rows)), ids, sc, eids, esc, what="batched, some rows re-joined")
    w = dict(zip(KNN_STATS, st.cpu().tolist()))
    assert w["fixed_point_rows"] == R.n_rows * nb, w       # the fixed-point pass: every item
    n_again = w["block_steps"] // nb - R.n_rows            # rows the fp32 pass joined
    assert w["block_steps"] % nb == 0 and len(flagged) <= n_again < R.n_rows, (w, len(flagged))
    sp = torch.zeros(len(KNN_STATS), dtype=torch.int64, device="cuda")
    knn.knn_join(idx, knn.DeviceCSR.from_host(R), k, s_groups=1, blocks_per_launch=2, stats=sp)
    assert sp[0].item() == w["block_steps"], (sp.tolist(), w)   # the same rows re-joined
    b.close()
    idx.close()


@pytest.mark.slow
def test_config5_shaped_f32_sampled_rows(knn, oracle_mod):
    """The float scale-up's generator (Zipf ids over d = 50,000, power-law nnz up to
    2,000, L2-normalised log-normal weights, k = 20) at |S| = 150,000 (10 S blocks), on
    24 query rows, against the fp64 oracle."""
    S = synth.zipf_f32(150000, synth.config_seed(5, "S"))
    R = synth.zipf_f32(24, synth.config_seed(5, "R"))
    eids, esc, _ = oracle_mod.iib_join(R, S, 20, threads=8)
    idx = knn.knn_join_build_index(S)
    Rd = knn.DeviceCSR.from_host(R)
    for mode, margin in (("iib", 0.0), ("iiib", 0.25), ("iiib", 0.6)):
        ids, sc = knn.knn_join(idx, Rd, 20, mode=mode, level_margin=margin)
        compare.assert_close(R, S, list(range(R.n_rows)), ids.cpu().numpy(), sc.cpu().numpy(), eids, esc,
                             what=f"config5-shaped {mode} {margin}")
    idx.close()


# ----------------------------------------------------------------------------------
# degenerate inputs
# ----------------------------------------------------------------------------------

def test_degenerate(knn, oracle_mod):
    import torch
    S = synth.from_rows([[(1, 2), (3, 1)], [], [(3, 2)], [(2, 4)], [(1, 1), (3, 1)]], 6)
    # R with an empty row and a row without overlap
    R = synth.from_rows([[], [(0, 9)], [(1, 1), (3, 1)]], 6)
    ids, sc = run(knn, S, R, 7)
    eids, esc, _ = oracle_mod.bf_join(R, S, 7)
    compare.assert_exact(ids, sc, eids, esc, "degenerate")
    # empty R
    idx = knn.knn_join_build_index(S)
    e = synth.from_rows([], 6)
    ids, sc = knn.knn_join(idx, e, 3)
    assert ids.shape == (0, 3)
    # all S rows identical: every score ties, ids ascending
    same = synth.from_rows([[(2, 3), (5, 1)]] * 1000, 8)
    ids, sc = run(knn, same, same.slice_rows(0, 2), 6, block_size=256, s_groups=3)
    assert ids.tolist() == [[0, 1, 2, 3, 4, 5]] * 2 and sc.tolist() == [[10] * 6] * 2
    # empty S
    empty_s = synth.from_rows([[]] * 3, 6)
    ids, sc = run(knn, empty_s, R, 2)
    assert (ids == -1).all() and (sc == 0).all()
    idx.close()


def test_host_inputs_and_host_outputs(knn, oracle_mod):
    S = synth.spectrum_u8(4000, 61, role="S")
    R = synth.spectrum_u8(30, 62, role="R")
    eids, esc, _ = oracle_mod.iib_join(R, S, 5, threads=8)
    idx = knn.knn_join_build_index(S)
    ids, sc = knn.knn_join(idx, R, 5, outputs_on_host=True)
    compare.assert_exact(ids.numpy(), sc.numpy(), eids, esc, "host in/out")
    idx.close()


# ----------------------------------------------------------------------------------
# input validation (host-side error codes, no fault)
# ----------------------------------------------------------------------------------

def test_validation_errors(knn):
    from paper_1011_2807_gb300.binding import KNN_EINVAL, KNN_EUNSUPPORTED, KnnError
    good = synth.from_rows([[(1, 2), (3, 1)], [(0, 1)]], 6)
    idx = knn.knn_join_build_index(good)
    bad_cases = []
    b = synth.from_rows([[(1, 2), (3, 1)]], 6); b.indices[:] = [3, 1]; bad_cases.append(("unsorted", b))
    b = synth.from_rows([[(1, 2), (3, 1)]], 6); b.indices[:] = [1, 1]; bad_cases.append(("duplicate", b))
    b = synth.from_rows([[(1, 2), (3, 1)]], 6); b.indices[1] = 6; bad_cases.append(("d >= dim", b))
    b = synth.from_rows([[(1, 2), (3, 1)]], 6); b.indices[0] = -1; bad_cases.append(("d < 0", b))
    b = synth.from_rows([[(1, 2), (3, 1)]], 6); b.values[0] = 0; bad_cases.append(("w = 0", b))
    b = synth.from_rows([[(1, 2), (3, 1)], [(2, 1)]], 6); b.indptr[1] = 5; bad_cases.append(("indptr", b))
    f = synth.from_rows([[(1, 0.5), (3, 1.0)]], 6, np.float32); f.values[0] = np.nan
    for name, bcsr in bad_cases:
        for dev in (False, True):
            with pytest.raises(KnnError) as e:
                knn.knn_join(idx, knn.DeviceCSR.from_host(bcsr) if dev else bcsr, 2)
            assert e.value.status == KNN_EINVAL, name
            with pytest.raises(KnnError):
                knn.knn_join_build_index(bcsr)
    with pytest.raises(KnnError) as e:
        knn.knn_join_build_index(f)
    assert e.value.status == KNN_EINVAL
    with pytest.raises(KnnError) as e:
        knn.knn_join(idx, good, 65)
    assert e.value.status == KNN_EUNSUPPORTED
    with pytest.raises(KnnError) as e:
        knn.knn_join(idx, good, 0)
    assert e.value.status == KNN_EINVAL
    with pytest.raises(KnnError) as e:      # dim mismatch
        knn.knn_join(idx, synth.from_rows([[(1, 2)]], 7), 2)
    assert e.value.status == KNN_EINVAL
    with pytest.raises(KnnError) as e:      # dtype mismatch
        knn.knn_join(idx, synth.from_rows([[(1, 0.5)]], 6, np.float32), 2)
    assert e.value.status == KNN_EINVAL
    idx.close()


# ----------------------------------------------------------------------------------
# a learned start threshold: rows keep only scores >= tau, n_found counts them
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("mode", ["iib", "iiib"])
def test_init_threshold(knn, oracle_mod, mode):
    import torch
    S = synth.spectrum_u8(8000, 71, role="S")
    R = synth.spectrum_u8(80, 72, role="R")
    k = 10
    eids, esc, _ = oracle_mod.iib_join(R, S, 64, threads=8)
    rng = np.random.default_rng(3)
    # thresholds around each row's k-th score: some rows over-predicted, some under
    tau = (esc[:, k - 1] * rng.uniform(0.5, 1.5, size=R.n_rows)).astype(np.float32)
    tau[0] = 0.0
    tau[1] = np.float32(esc[1, k - 1])          # exactly the k-th score (inclusive)
    tau[2] = np.float32(1e9)                    # nothing passes
    t_tau = torch.from_numpy(tau).cuda()
    found = torch.zeros(R.n_rows, dtype=torch.int32, device="cuda")
    idx = knn.knn_join_build_index(S, block_size=1024)
    ids, sc = knn.knn_join(idx, knn.DeviceCSR.from_host(R), k, mode=mode, init_threshold=t_tau, n_found=found)
    torch.cuda.synchronize()
    ids, sc, found = ids.cpu().numpy(), sc.cpu().numpy(), found.cpu().numpy()
    for i in range(R.n_rows):
        keep = esc[i] >= max(tau[i], 1e-30)
        want = min(k, int(keep.sum()))
        assert found[i] == want, (i, found[i], want)
        np.testing.assert_array_equal(ids[i, :want], eids[i, :want])
        np.testing.assert_array_equal(sc[i, :want], esc[i, :want])
        assert (ids[i, want:] == -1).all()
    idx.close()


# ----------------------------------------------------------------------------------
# posting counters: IIB scans exactly the eq. 4 count; IIIB scans no more
# ----------------------------------------------------------------------------------

def test_posting_counter_eq4(knn):
    import torch
    S = synth.spectrum_u8(20000, 111, role="S")
    R = synth.spectrum_u8(100, 112, role="R")
    want = refdefs.postings_touched_iib(R, S)
    idx = knn.knn_join_build_index(S, block_size=2048)
    counts = {}
    for mode in ("iib", "iiib"):
        c = torch.zeros(1, dtype=torch.int64, device="cuda")
        # one group per row: every S block after the first carries the row's threshold
        knn.knn_join(idx, knn.DeviceCSR.from_host(R), 5, mode=mode, postings_scanned=c, s_groups=1)
        torch.cuda.synchronize()
        counts[mode] = int(c.item())
    assert counts["iib"] == want
    assert counts["iiib"] < counts["iib"]
    idx.close()


# ----------------------------------------------------------------------------------
# brute force (Algorithm 2) on the GPU: the baseline mode gives the same results
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("bs,groups", [(256, 0), (1024, 1), (2048, 3)])
@pytest.mark.parametrize("k", [1, 5, 64])
def test_bf_mode_u8_exact(knn, oracle_mod, bs, groups, k):
    S = synth.spectrum_u8(5000, 131, role="S")          # ragged last block
    R = synth.spectrum_u8(90, 132, role="R")
    eids, esc, _ = oracle_mod.bf_join(R, S, k, threads=8)
    ids, sc = run(knn, S, R, k, mode="bf", block_size=bs, s_groups=groups)
    compare.assert_exact(ids, sc, eids, esc, f"bf bs={bs} groups={groups} k={k}")


def test_bf_mode_f32_and_degenerate(knn, oracle_mod):
    S = synth.zipf_f32(3000, 141, dim=2000, nnz_hi=200)
    R = synth.zipf_f32(40, 142, dim=2000, nnz_hi=200)
    eids, esc, _ = oracle_mod.bf_join(R, S, 20, threads=8)
    ids, sc = run(knn, S, R, 20, mode="bf", block_size=512)
    compare.assert_close(R, S, list(range(R.n_rows)), ids, sc, eids, esc, what="bf f32")
    S2 = synth.from_rows([[(1, 2), (3, 1)], [], [(3, 2)], [(2, 4)], [(1, 1), (3, 1)]], 6)
    R2 = synth.from_rows([[], [(0, 9)], [(1, 1), (3, 1)]], 6)
    ids, sc = run(knn, S2, R2, 7, mode="bf")
    eids, esc, _ = oracle_mod.bf_join(R2, S2, 7)
    compare.assert_exact(ids, sc, eids, esc, "bf degenerate")


def test_bf_mode_reads_every_feature_of_s(knn):
    """The brute-force work counter is nnz(S) per non-empty query row (every S vector is
    scored in full, eq. 3's S-side term), whatever the block size."""
    import torch
    S = synth.spectrum_u8(6000, 151, role="S")
    R = synth.spectrum_u8(50, 152, role="R")
    idx = knn.knn_join_build_index(S, block_size=1024)
    c = torch.zeros(1, dtype=torch.int64, device="cuda")
    knn.knn_join(idx, knn.DeviceCSR.from_host(R), 5, mode="bf", postings_scanned=c)
    torch.cuda.synchronize()
    nonempty = int((np.diff(R.indptr) > 0).sum())
    assert int(c.item()) == nonempty * S.nnz
    idx.close()


# ----------------------------------------------------------------------------------
# the index in pinned host memory (out-of-core form): the same results
# ----------------------------------------------------------------------------------

def test_host_resident_index(knn, oracle_mod):
    import torch
    S = synth.spectrum_u8(20000, 161, role="S")
    R = synth.spectrum_u8(150, 162, role="R")
    Rd = knn.DeviceCSR.from_host(R)
    idx = knn.knn_join_build_index(S, block_size=2048)
    ref = {}
    for mode, groups in (("iiib", 0), ("iiib", 3), ("iib", 1), ("bf", 1)):
        ref[mode, groups] = knn.knn_join(idx, Rd, 7, mode=mode, s_groups=groups)
    bref = knn.knn_join_batched([(idx, Rd, 7)])
    before = idx.info()
    assert before["device_bytes"] > 0 and before["host_bytes"] == 0
    idx.to_host()
    after = idx.info()
    assert after["device_bytes"] == 0 and after["host_bytes"] >= before["device_bytes"] // 2
    for (mode, groups), (ids, sc) in ref.items():
        hids, hsc = knn.knn_join(idx, Rd, 7, mode=mode, s_groups=groups)
        assert torch.equal(ids, hids) and torch.equal(sc, hsc), (mode, groups)
    hb = knn.knn_join_batched([(idx, Rd, 7)])
    assert torch.equal(bref[0][0], hb[0][0]) and torch.equal(bref[0][1], hb[0][1])
    eids, esc, _ = oracle_mod.iib_join(R, S, 7, threads=8)
    hids, hsc = knn.knn_join(idx, Rd, 7)
    compare.assert_exact(hids.cpu().numpy(), hsc.cpu().numpy(), eids, esc, "host-resident index")
    idx.to_host()   # a second move is a no-op
    idx.close()


# ----------------------------------------------------------------------------------
# S in ranges (shards, or an S joined range by range) merged with knn_merge_topk
# ----------------------------------------------------------------------------------

def test_merge_topk_of_s_ranges(knn, oracle_mod):
    import torch
    from paper_1011_2807_gb300.binding import knn_merge_topk
    S = synth.spectrum_u8(7000, 171, role="S")
    R = synth.spectrum_u8(60, 172, role="R")
    Rd = knn.DeviceCSR.from_host(R)
    full = knn.knn_join_build_index(S, block_size=1024)
    fids, fsc = knn.knn_join(full, Rd, 9)
    cuts = [0, 2500, 2501, 7000]                 # a one-vector range in the middle
    parts, idxs = [], []
    for i, (a, b) in enumerate(zip(cuts[:-1], cuts[1:])):
        idx = knn.knn_join_build_index(S.slice_rows(a, b), block_size=1024)
        if i == 2:
            idx.to_host()                          # one range joined from host memory
        parts.append(knn.knn_join(idx, Rd, 9))
        idxs.append(idx)
    mids, msc = knn_merge_topk(parts, cuts[:-1], 9)
    assert torch.equal(mids, fids) and torch.equal(msc, fsc)
    eids, esc, _ = oracle_mod.iib_join(R, S, 9, threads=8)
    compare.assert_exact(mids.cpu().numpy(), msc.cpu().numpy(), eids, esc, "merged ranges")
    # float ranges
    Sf = synth.zipf_f32(3000, 181, dim=2000, nnz_hi=200)
    Rf = synth.zipf_f32(30, 182, dim=2000, nnz_hi=200)
    Rfd = knn.DeviceCSR.from_host(Rf)
    fparts = []
    for a, b in ((0, 1700), (1700, 3000)):
        idx = knn.knn_join_build_index(Sf.slice_rows(a, b), block_size=512)
        fparts.append(knn.knn_join(idx, Rfd, 12))
        idxs.append(idx)
    fi, fs = knn_merge_topk(fparts, [0, 1700], 12)
    eids, esc, _ = oracle_mod.iib_join(Rf, Sf, 12, threads=8)
    compare.assert_close(Rf, Sf, list(range(Rf.n_rows)), fi.cpu().numpy(), fs.cpu().numpy(), eids, esc,
                         what="merged float ranges")
    with pytest.raises(ValueError):
        knn_merge_topk(parts, [0, 1], 9)
    for idx in idxs + [full]:
        idx.close()


# ----------------------------------------------------------------------------------
# the benchmark's configuration at full size, on sampled rows
# ----------------------------------------------------------------------------------

@pytest.mark.slow
def test_config2_full_size_sampled_rows(knn, oracle_mod):
    import torch
    R, S, k = synth.config2()
    idx = knn.knn_join_build_index(S)
    ids, sc = knn.knn_join(idx, knn.DeviceCSR.from_host(R), k)
    torch.cuda.synchronize()
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    # 2,000 rows spread over all of R (a stratified draw: one per 50-row stretch), bit-exact
    rng = np.random.default_rng(7)
    rows = np.arange(0, R.n_rows, R.n_rows // 2000)[:2000] + rng.integers(0, R.n_rows // 2000, size=2000)
    assert rows.size == 2000 and rows.max() < R.n_rows
    Rs = R.take_rows(rows)
    eids, esc, _ = oracle_mod.iib_join(Rs, S, k, threads=0)
    compare.assert_exact(ids[rows], sc[rows], eids, esc, "config2 full size")
    idx.close()
