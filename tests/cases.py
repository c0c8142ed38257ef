"""Seeded query/S cases shared by the GPU tests (inputs only: no arithmetic of the join)."""
import numpy as np

from paper_1011_2807_gb300 import synth


def random_u8(n, dim, nnz_hi, seed, wmax=100, nnz_lo=0):
    rng = np.random.default_rng(seed)
    rows = []
    for _ in range(n):
        m = int(rng.integers(nnz_lo, min(nnz_hi, dim) + 1))
        d = rng.choice(dim, size=m, replace=False)
        w = rng.integers(1, wmax + 1, size=m)
        rows.append(list(zip(d.tolist(), w.tolist())))
    return synth.from_rows(rows, dim, np.uint8)


def long_row_case(dtype, seed, n_s=40000, dim=6000):
    """S, and R with rows of 1,000-2,500 features (too long for a two-CTA-per-SM layout
    with 16,384-vector S blocks: the split starts above ~920) among short rows (5-200
    features, and one of 900)."""
    rng = np.random.default_rng(seed)
    if dtype == "u8":
        S = random_u8(n_s, dim, 80, seed + 1, nnz_lo=10)
        draw = lambda n: rng.integers(1, 101, n).tolist()
    else:
        S = synth.zipf_f32(n_s, seed + 1, dim=dim, nnz_hi=300)
        draw = lambda n: rng.lognormal(0.0, 1.0, n).tolist()
    row = lambda n: list(zip(np.sort(rng.choice(dim, n, replace=False)).tolist(), draw(n)))
    short = [row(int(rng.integers(5, 200))) for _ in range(60)] + [row(900)]
    rows = short[:30] + [row(n) for n in (1000, 1400, 2500)] + short[30:]
    return S, synth.from_rows(rows, dim, np.uint8 if dtype == "u8" else np.float32), \
        synth.from_rows(short, dim, np.uint8 if dtype == "u8" else np.float32)
