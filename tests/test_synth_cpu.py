"""The seeded input generators: rows are sets of distinct ascending ids with positive
values, drawn from the stated distributions; checked against brute force and closed
forms on the CPU."""
import numpy as np
import pytest

from paper_1011_2807_gb300 import synth


def check_rows(X, lo, hi):
    lens = np.diff(X.indptr)
    assert X.indptr[0] == 0 and X.indptr[-1] == len(X.indices) == len(X.values)
    assert lens.min(initial=lo) >= lo and lens.max(initial=hi) <= hi
    d = np.diff(X.indices.astype(np.int64))
    inner = np.ones(len(d), bool)
    inner[X.indptr[1:-1][X.indptr[1:-1] > 0] - 1] = False    # steps across a row boundary
    assert (d[inner] > 0).all()
    assert X.indices.min(initial=0) >= 0 and X.indices.max(initial=0) < X.dim
    assert (X.values > 0).all()


def test_first_distinct_matches_brute_force():
    """Each row holds the first need[i] distinct ids of its own draw sequence (the first
    batch's row, then its rows of later batches), sorted; long quotas force several
    continuation batches."""
    calls = []

    def draw(rng, shape):
        x = rng.integers(0, 12, size=shape)
        calls.append(x)
        return x

    need = np.array([1, 3, 5, 8, 10, 12, 12, 0, 7])
    rng = np.random.default_rng(3)
    indptr, idx = synth._first_distinct(rng, need, draw, width=6)
    assert len(calls) > 1
    seqs = [list(r) for r in calls[0]]
    short = [i for i in range(len(need))]
    for batch in calls[1:]:
        # rows still short after the previous batches, in row order
        short = [i for i in short if len(dict.fromkeys(seqs[i])) < need[i]]
        assert len(short) == batch.shape[0]
        for i, r in zip(short, batch):
            seqs[i] += list(r)
    for i, n in enumerate(need):
        first = list(dict.fromkeys(int(v) for v in seqs[i]))[:n]
        assert list(idx[indptr[i]:indptr[i + 1]]) == sorted(first), i


def test_alias_sampler_frequencies():
    """Walker's alias table reproduces p(rank) ~ rank^-1.1: chi-square over the first
    30 ranks and the tail mass, 2M draws (critical value at p = 1e-6)."""
    dim, alpha = 5000, 1.1
    prob, alias, draws = synth._zipf_tables(dim, alpha)
    d = synth._zipf_alias_draw(np.arange(dim), prob, alias)(np.random.default_rng(1), (2_000_000,))
    p = np.arange(1, dim + 1, dtype=np.float64) ** -alpha
    p /= p.sum()
    cnt = np.bincount(d, minlength=dim)
    obs = np.append(cnt[:30], cnt[30:].sum())
    exp = np.append(p[:30], p[30:].sum()) * d.size
    chi2 = ((obs - exp) ** 2 / exp).sum()
    assert chi2 < 90.0, chi2           # 31 cells: 30 degrees of freedom
    # the draw table: n distinct ranks need at least n draws, more for a skewed law
    assert draws[1] == 1 and (np.diff(draws[1:]) >= 0).all() and (draws[1:] >= np.arange(1, dim + 1)).all()
    assert draws[200] > 1.5 * 200


def test_zipf_rows_and_chunk_prefix():
    X = synth.zipf_f32(70000, 11)
    check_rows(X, 5, 2000)
    norms = np.bincount(np.repeat(np.arange(X.n_rows), np.diff(X.indptr)),
                        weights=X.values.astype(np.float64) ** 2)
    np.testing.assert_allclose(norms, 1.0, rtol=1e-6)
    assert 50 < np.diff(X.indptr).mean() < 70          # power law on [5, 2000]: mean ~60
    Y = synth.zipf_f32(synth.ZIPF_CHUNK, 11)
    assert np.array_equal(X.indptr[:Y.n_rows + 1], Y.indptr)
    assert np.array_equal(X.indices[:Y.nnz], Y.indices) and np.array_equal(X.values[:Y.nnz], Y.values)


def test_zipf_parallel_equals_serial():
    n = 2 * synth.ZIPF_CHUNK + 17
    a = synth.zipf_f32(n, 5, dim=3000, nnz_hi=300)
    b = synth.zipf_f32(n, 5, dim=3000, nnz_hi=300, processes=2)
    assert np.array_equal(a.indptr, b.indptr) and np.array_equal(a.indices, b.indices)
    assert np.array_equal(a.values, b.values)


def test_zipf_small_dim_needs_long_continuations():
    # rows of up to 200 of 220 ids: most draws repeat the head, so rows continue often
    X = synth.zipf_f32(3000, 2, dim=220, nnz_hi=200)
    check_rows(X, 5, 200)


@pytest.mark.parametrize("role,lo,hi", [("S", 20, 60), ("R", 20, 600)])
def test_spectrum_rows(role, lo, hi):
    X = synth.spectrum_u8(20000, 77, role=role)
    check_rows(X, lo, hi)
    assert X.values.min() >= 1 and X.values.max() <= 100
    if role == "R":
        assert 135 < np.diff(X.indptr).mean() < 165     # log-normal, mean ~150
