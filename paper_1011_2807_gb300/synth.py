"""Seeded synthetic sparse-vector workloads.

This module only draws random inputs: it holds none of the join's arithmetic, and it
is the one module that both the CUDA path's tests/bench and the CPU oracle's checks
take their inputs from.

A sparse vector is a set of features (d, w) with w > 0, kept in ascending d
(Section 3 of the paper).  A set of vectors is held as CSR:
``indptr`` int64[n+1], ``indices`` int32[nnz] (strictly ascending per row, 0-based),
``values`` uint8[nnz] or float32[nnz].

The paper describes its synthetic data only as random sparse vectors with 10,000
dimensions (Section 5) and its real data as MS/MS spectra whose m/z x 10 is the
dimension and whose peak intensity is the value (Section 5).  The workloads below stand
in for both; their parameters are this library's own choice:

* ``uniform_f32``: nnz ~ U{lo..hi}, ids uniform without replacement, w = 1 - U[0,1).
* ``spectrum_u8``: ids from an 8-component Gaussian mixture (centres U[3000,7000],
  sigma 200 bins, rounded and clipped), without replacement by rejection in draw
  order; w ~ U{1..100} as uint8.  Query rows draw nnz from a clipped log-normal
  (mean ~150, [20,600]); database rows from U{20..60}.
* ``zipf_f32``: ids Zipf(alpha) over ranks mapped through a seeded permutation (drawn
  with Walker's alias method), without replacement by rejection in draw order; nnz
  from a discrete power law p(n) ~ n^-1.67 on [5, 2000] (mean ~60), w log-normal(0,1),
  each row L2-normalised.  Rows come in independently seeded chunks of 65,536.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable

import numpy as np

SEED_BASE = 1011


def config_seed(config: int, role: str) -> int:
    """Seed of one input of one workload: base + 100*config + role offset."""
    return SEED_BASE + 100 * config + {"S": 0, "R": 1, "train": 2, "eval": 3, "mix": 99}[role]


@dataclasses.dataclass
class CSR:
    """A set of sparse vectors in CSR form (numpy arrays on the host)."""

    indptr: np.ndarray   # int64 [n+1]
    indices: np.ndarray  # int32 [nnz]
    values: np.ndarray   # uint8 or float32 [nnz]
    dim: int

    @property
    def n_rows(self) -> int:
        return int(self.indptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.indptr[-1])

    def row(self, i: int):
        a, b = int(self.indptr[i]), int(self.indptr[i + 1])
        return self.indices[a:b], self.values[a:b]

    def take_rows(self, rows) -> "CSR":
        rows = np.asarray(rows, dtype=np.int64)
        lens = self.indptr[rows + 1] - self.indptr[rows]
        indptr = np.zeros(len(rows) + 1, dtype=np.int64)
        np.cumsum(lens, out=indptr[1:])
        idx = np.concatenate([np.arange(self.indptr[r], self.indptr[r + 1]) for r in rows]) \
            if len(rows) else np.zeros(0, dtype=np.int64)
        return CSR(indptr, self.indices[idx].copy(), self.values[idx].copy(), self.dim)

    def slice_rows(self, a: int, b: int) -> "CSR":
        lo, hi = int(self.indptr[a]), int(self.indptr[b])
        return CSR(self.indptr[a:b + 1] - lo, self.indices[lo:hi].copy(),
                   self.values[lo:hi].copy(), self.dim)

    def to_dense(self, dtype=np.float64) -> np.ndarray:
        out = np.zeros((self.n_rows, self.dim), dtype=dtype)
        rows = np.repeat(np.arange(self.n_rows), np.diff(self.indptr))
        out[rows, self.indices] = self.values.astype(dtype)
        return out


def from_rows(rows, dim: int, dtype=np.uint8) -> CSR:
    """CSR from a list of rows, each a list of (d, w) pairs (any order)."""
    indptr = [0]
    idx, val = [], []
    for r in rows:
        r = sorted(r)
        idx.extend(d for d, _ in r)
        val.extend(w for _, w in r)
        indptr.append(len(idx))
    return CSR(np.asarray(indptr, np.int64), np.asarray(idx, np.int32),
               np.asarray(val, dtype), dim)


# ----------------------------------------------------------------------------------
# unique-id sampling: first `nnz[i]` distinct draws in draw order, then sorted
# ----------------------------------------------------------------------------------

def _unique_rows(rng, nnz, draw, dim, chunk=1 << 18, over=1.3, pos_bits=12):
    """Rejection sampling without replacement, vectorised over rows.

    For each row, ids are drawn one after another from ``draw``; a repeat of an id
    already drawn in that row is rejected, until the row holds nnz[i] ids.  Each row
    first gets an oversampled batch of draws; a row that is still short continues
    its own draw sequence in small batches.  Returns (indptr, indices), each row's
    ids sorted ascending.
    """
    if np.any(nnz > dim):
        raise ValueError("nnz larger than dim")
    n = int(nnz.shape[0])
    nnz = nnz.astype(np.int64)
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(nnz, out=indptr[1:])
    out = np.empty(int(indptr[-1]), dtype=np.int32)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        need = nnz[a:b]
        width = min((1 << pos_bits) - 1, max(8, int(int(need.max(initial=0)) * over) + 8))
        ids = draw(rng, (b - a, width)).astype(np.int64)
        key = ids * (1 << pos_bits) + np.arange(width)[None, :]
        key.sort(axis=1)
        val = key >> pos_bits
        pos = key & ((1 << pos_bits) - 1)
        first = np.ones_like(val, dtype=bool)
        first[:, 1:] = val[:, 1:] != val[:, :-1]
        keep = np.zeros_like(first)
        np.put_along_axis(keep, pos, first, axis=1)
        cum = np.cumsum(keep, axis=1)
        ok = cum[:, -1] >= need
        sel = keep & (cum <= need[:, None])
        # selected values, re-sorted per row: sort keys restricted to selected entries
        sval = np.where(sel, ids, np.int64(1) << 40)
        sval.sort(axis=1)
        rows_ok = np.nonzero(ok)[0]
        # gather the first need[i] entries of each ok row
        lens = need[rows_ok]
        if rows_ok.size:
            colmask = np.arange(width)[None, :] < lens[:, None]
            vals = sval[rows_ok][colmask]
            starts = indptr[a + rows_ok]
            dst = np.repeat(starts, lens) + (np.arange(lens.sum()) - np.repeat(np.cumsum(lens) - lens, lens))
            out[dst] = vals.astype(np.int32)
        for j in np.nonzero(~ok)[0]:
            # finish this row by continuing its own draw sequence in small batches
            have = list(ids[j][keep[j]])
            seen = set(have)
            while len(have) < need[j]:
                for x in draw(rng, (1, 64))[0]:
                    x = int(x)
                    if x not in seen and len(have) < need[j]:
                        seen.add(x)
                        have.append(x)
            r = a + j
            out[indptr[r]:indptr[r + 1]] = np.sort(np.asarray(have[:need[j]], dtype=np.int64))
    return indptr, out


def _first_distinct(rng, need, draw, width):
    """First ``need[i]`` distinct ids of row i's own draw sequence, sorted ascending.

    Every row gets ``width`` draws at once; rows that are still short extend their own
    sequence by further batches (all short rows at once) until each holds its quota, so
    each row is exactly the first distinct ids of one i.i.d. draw sequence.  Returns
    (indptr, indices) in row order."""
    m = int(need.shape[0])
    need = need.astype(np.int64)
    indptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(need, out=indptr[1:])
    out = np.empty(int(indptr[-1]), dtype=np.int32)
    rows = np.arange(m)
    ids = draw(rng, (m, width))
    while rows.size:
        w = ids.shape[1]
        pos_bits = max(1, int(w - 1).bit_length())
        key = ids * (1 << pos_bits) + np.arange(w)[None, :]
        key.sort(axis=1)
        val = key >> pos_bits
        first = np.ones(val.shape, dtype=bool)
        first[:, 1:] = val[:, 1:] != val[:, :-1]
        keep = np.zeros_like(first)
        np.put_along_axis(keep, key & ((1 << pos_bits) - 1), first, axis=1)
        cum = np.cumsum(keep, axis=1)
        nd = need[rows]
        ok = cum[:, -1] >= nd
        if ok.any():
            sel = keep[ok] & (cum[ok] <= nd[ok][:, None])
            sval = np.where(sel, ids[ok], np.int64(1) << 40)
            sval.sort(axis=1)
            lens = nd[ok]
            vals = sval[np.arange(w)[None, :] < lens[:, None]]
            dst = np.repeat(indptr[rows[ok]], lens) + (np.arange(int(lens.sum()))
                                                         - np.repeat(np.cumsum(lens) - lens, lens))
            out[dst] = vals.astype(np.int32)
        short = ~ok
        rows = rows[short]
        if rows.size:
            ids = np.concatenate([ids[short], draw(rng, (int(rows.size), max(16, w // 4)))], axis=1)
    return indptr, out


_ZIPF_TABLES: dict = {}


def _zipf_tables(dim: int, alpha: float):
    """Walker's alias table for p(rank) ~ rank^-alpha over ranks 1..dim (Vose's
    construction), and, for every n <= dim, the number of i.i.d. draws whose expected
    count of distinct ranks, sum_i 1 - (1 - p_i)^m, first reaches n."""
    key = (dim, float(alpha))
    if key in _ZIPF_TABLES:
        return _ZIPF_TABLES[key]
    p = np.arange(1, dim + 1, dtype=np.float64) ** (-alpha)
    p /= p.sum()
    scaled = p * dim
    prob = np.ones(dim, dtype=np.float64)
    alias = np.arange(dim, dtype=np.int64)
    small = [i for i in range(dim) if scaled[i] < 1.0]
    large = [i for i in range(dim) if scaled[i] >= 1.0]
    while small and large:
        s_, l_ = small.pop(), large.pop()
        prob[s_] = scaled[s_]
        alias[s_] = l_
        scaled[l_] -= 1.0 - scaled[s_]
        (small if scaled[l_] < 1.0 else large).append(l_)
    # draws needed for n distinct: evaluate the expected distinct count on a grid of m
    grid = np.unique(np.rint(np.geomspace(1, 64.0 * dim, 4096)).astype(np.int64))
    q = np.log1p(-p)
    expect = np.array([float((-np.expm1(m * q)).sum()) for m in grid])
    n_all = np.arange(dim + 1, dtype=np.float64)
    draws = grid[np.minimum(np.searchsorted(expect, n_all - 1e-6, side="left"), len(grid) - 1)]
    _ZIPF_TABLES[key] = (prob, alias, draws)
    return _ZIPF_TABLES[key]


def _zipf_alias_draw(perm: np.ndarray, prob: np.ndarray, alias: np.ndarray):
    dim = len(perm)

    def draw(rng, shape):
        x = rng.random(size=shape) * dim
        i = x.astype(np.int64)
        np.minimum(i, dim - 1, out=i)
        r = np.where(x - i < prob[i], i, alias[i])
        return perm[r]
    return draw


ZIPF_CHUNK = 1 << 16


# ----------------------------------------------------------------------------------
# id distributions
# ----------------------------------------------------------------------------------

def _uniform_draw(dim: int):
    def draw(rng, shape):
        return rng.integers(0, dim, size=shape, dtype=np.int64)
    return draw


def mixture_centres(seed: int, n_comp: int = 8, lo: float = 3000.0, hi: float = 7000.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=n_comp)


def _mixture_draw(centres: np.ndarray, sigma: float, dim: int):
    def draw(rng, shape):
        comp = rng.integers(0, len(centres), size=shape)
        x = centres[comp] + sigma * rng.standard_normal(size=shape)
        return np.clip(np.rint(x), 0, dim - 1).astype(np.int64)
    return draw


# ----------------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------------

def uniform_f32(n: int, dim: int, nnz_lo: int, nnz_hi: int, seed: int) -> CSR:
    """Uniform ids without replacement; w = 1 - U[0,1) in (0, 1] as float32."""
    rng = np.random.default_rng(seed)
    nnz = rng.integers(nnz_lo, nnz_hi + 1, size=n)
    indptr, idx = _unique_rows(rng, nnz, _uniform_draw(dim), dim)
    vals = (1.0 - rng.random(size=idx.shape[0])).astype(np.float32)
    vals = np.maximum(vals, np.float32(np.finfo(np.float32).tiny))
    return CSR(indptr, idx, vals, dim)


def spectrum_nnz_query(rng, n: int) -> np.ndarray:
    # mean of LogNormal(4.835, 0.6) is exp(4.835 + 0.18) ~ 150
    x = rng.lognormal(mean=4.835, sigma=0.6, size=n)
    return np.clip(np.rint(x), 20, 600).astype(np.int64)


def spectrum_u8(n: int, seed: int, *, role: str = "S", dim: int = 10000,
                mix_seed: int | None = None, nnz: np.ndarray | None = None,
                nnz_lo: int = 20, nnz_hi: int = 60) -> CSR:
    """Spectrum-shaped uint8 vectors (ids from a shared Gaussian mixture)."""
    rng = np.random.default_rng(seed)
    if nnz is None:
        if role == "R":
            nnz = spectrum_nnz_query(rng, n)
        else:
            nnz = rng.integers(nnz_lo, nnz_hi + 1, size=n)
    centres = mixture_centres(config_seed(2, "mix") if mix_seed is None else mix_seed)
    nnz = np.minimum(nnz, dim)
    indptr, idx = _unique_rows(rng, nnz, _mixture_draw(centres, 200.0, dim), dim)
    vals = rng.integers(1, 101, size=idx.shape[0], dtype=np.uint8)
    return CSR(indptr, idx, vals, dim)


def spectra_text(n: int, seed: int, *, fmt: str = "mgf", peaks_lo: int = 20, peaks_hi: int = 600,
                 mz_max: float = 999.9, noise: bool = True) -> str:
    """MS/MS peak lists as MGF or MS2 text: n spectra, peak counts log-normal (mean
    ~150, clipped to [peaks_lo, peaks_hi]), m/z around the spectrum-shaped workload's
    mixture centres (dimension / 10, 4 decimals), log-normal intensities.  With
    ``noise`` the text also carries what real files do: CRLF and tab-separated lines,
    comments, header records, a charge field after some MGF peaks, intensities in
    scientific notation, zero or negative intensities, and peaks closer than 0.1 in
    m/z (two peaks in one dimension)."""
    rng = np.random.default_rng(seed)
    centres = mixture_centres(config_seed(2, "mix")) / 10.0
    counts = np.clip(np.rint(rng.lognormal(4.835, 0.6, size=n)), peaks_lo, peaks_hi).astype(np.int64)
    out = []
    nl = "\n"
    if fmt == "ms2":
        out.append("H\tCreationDate\tsynthetic" + nl + "H\tExtractor\tsynth.spectra_text" + nl)
    for i in range(n):
        m = int(counts[i])
        mz = centres[rng.integers(0, len(centres), size=m)] + 20.0 * rng.standard_normal(size=m)
        mz = np.clip(mz, 0.0, mz_max)
        if noise and m > 2:   # a few peaks within 0.1 of another
            k = max(1, m // 20)
            src = rng.integers(0, m, size=k)
            mz[rng.integers(0, m, size=k)] = np.clip(mz[src] + rng.uniform(-0.04, 0.04, size=k), 0.0, mz_max)
        inten = rng.lognormal(6.0, 1.5, size=m)
        if noise:
            bad = rng.random(size=m) < 0.02
            inten[bad] = rng.choice([0.0, -1.0], size=int(bad.sum()))
        eol = "\r\n" if noise and rng.random() < 0.3 else nl
        if fmt == "mgf":
            out.append("BEGIN IONS" + eol + f"TITLE=synthetic spectrum {i}" + eol +
                       f"PEPMASS={rng.uniform(300, 1500):.4f}" + eol + f"CHARGE={int(rng.integers(1, 4))}+" + eol)
        else:
            out.append(f"S\t{i + 1:06d}\t{i + 1:06d}\t{rng.uniform(300, 1500):.4f}" + eol +
                       f"Z\t{int(rng.integers(1, 4))}\t{rng.uniform(600, 3000):.4f}" + eol)
        for j in range(m):
            style = int(rng.integers(0, 4)) if noise else 0
            w = f"{inten[j]:.2f}" if style != 1 else f"{inten[j]:.6e}"
            sep = "\t" if style == 2 else " "
            extra = " 1+" if (fmt == "mgf" and style == 3) else ""
            out.append(f"{mz[j]:.4f}{sep}{w}{extra}{eol}")
            if noise and rng.random() < 0.005:
                out.append("# a comment line" + eol)
        if fmt == "mgf":
            out.append("END IONS" + eol + (eol if noise and rng.random() < 0.5 else ""))
    return "".join(out)


def powerlaw_nnz(rng, n: int, lo: int = 5, hi: int = 2000, a: float = 1.67) -> np.ndarray:
    support = np.arange(lo, hi + 1, dtype=np.float64)
    p = support ** (-a)
    cdf = np.cumsum(p)
    cdf /= cdf[-1]
    return (lo + np.searchsorted(cdf, rng.random(size=n), side="right")).clip(lo, hi).astype(np.int64)


def _zipf_chunk(n: int, seed: int, chunk: int, dim: int, alpha: float, perm: np.ndarray,
                nnz_lo: int, nnz_hi: int, budget: int = 1 << 23):
    """Rows of chunk ``chunk`` of a Zipf workload, from their own generator
    (entropy [seed, chunk]): nnz, ids, log-normal w, L2-normalised.  Ids are drawn for
    rows in ascending nnz order, in sub-chunks of at most ``budget`` draws whose rows'
    draw widths lie within 1.25x of each other."""
    rng = np.random.default_rng([seed, chunk])
    nnz = np.minimum(powerlaw_nnz(rng, n, nnz_lo, nnz_hi), dim)
    prob, alias, draws = _zipf_tables(dim, alpha)
    draw = _zipf_alias_draw(perm, prob, alias)
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(nnz, out=indptr[1:])
    idx = np.empty(int(indptr[-1]), dtype=np.int32)
    order = np.argsort(nnz, kind="stable")
    width = (draws[nnz[order]] * 1.1).astype(np.int64) + 16      # ascending with the rows
    a = 0
    while a < n:
        # rows whose draw width is within 1.25x of the first one's, up to ``budget`` draws
        top = a + int(np.searchsorted(width[a:], int(width[a] * 1.25), side="right"))
        cost = (np.arange(1, top - a + 1, dtype=np.int64)) * width[a:top]
        b = a + max(1, int(np.searchsorted(cost, budget, side="right")))
        rows = order[a:b]
        lens = nnz[rows]
        cptr, cidx = _first_distinct(rng, lens, draw, int(width[b - 1]))
        dst = np.repeat(indptr[rows], lens) + (np.arange(int(lens.sum())) - np.repeat(cptr[:-1], lens))
        idx[dst] = cidx
        a = b
    w = rng.lognormal(0.0, 1.0, size=idx.shape[0])
    rid = np.repeat(np.arange(n), nnz)
    norm = np.sqrt(np.bincount(rid, weights=w * w, minlength=n))
    vals = (w / norm[rid]).astype(np.float32)
    vals = np.maximum(vals, np.float32(np.finfo(np.float32).tiny))
    return nnz, idx, vals


def zipf_f32(n: int, seed: int, *, dim: int = 50000, alpha: float = 1.1,
             perm_seed: int | None = None, nnz_lo: int = 5, nnz_hi: int = 2000,
             processes: int = 1) -> CSR:
    """Zipf ids over a seeded permutation, power-law nnz, L2-normalised log-normal w.

    Rows come in chunks of ``ZIPF_CHUNK`` rows, each drawn by its own generator, so the
    first rows of a longer set equal a shorter set whose size is a multiple of the
    chunk.  With ``processes`` > 1 the chunks are drawn by a pool of that many
    processes (spawned, so it is safe after CUDA has been initialised); the result does
    not depend on it."""
    n_chunks = (n + ZIPF_CHUNK - 1) // ZIPF_CHUNK
    args = [(n, seed, c, dim, alpha, perm_seed, nnz_lo, nnz_hi) for c in range(n_chunks)]
    if processes > 1 and n_chunks > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(min(processes, n_chunks)) as pool:
            chunks = pool.starmap(_zipf_chunk_args, args)
    else:
        chunks = [_zipf_chunk_args(*a) for a in args]
    nnz = np.concatenate([c[0] for c in chunks]) if chunks else np.zeros(0, np.int64)
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(nnz, out=indptr[1:])
    idx = np.concatenate([c[1] for c in chunks]) if chunks else np.zeros(0, np.int32)
    vals = np.concatenate([c[2] for c in chunks]) if chunks else np.zeros(0, np.float32)
    return CSR(indptr, idx, vals, dim)


def _zipf_chunk_args(n, seed, chunk, dim, alpha, perm_seed, nnz_lo, nnz_hi):
    """Chunk ``chunk`` of ``zipf_f32(n, seed, ...)``: (nnz, indices, values)."""
    perm = np.random.default_rng(config_seed(5, "mix") if perm_seed is None else perm_seed).permutation(dim)
    rows = min(ZIPF_CHUNK, n - chunk * ZIPF_CHUNK)
    return _zipf_chunk(rows, seed, chunk, dim, alpha, perm, nnz_lo, nnz_hi)


def _call(name, args, kwargs):
    return globals()[name](*args, **kwargs)


def generate(calls, processes: int = 1):
    """Run generator calls ``[(name, args, kwargs), ...]`` (names of this module's
    functions) and return their results in order; with ``processes`` > 1, in a pool of
    that many spawned processes.  Every generator is seeded by its arguments, so the
    results do not depend on ``processes``."""
    calls = [(c[0], tuple(c[1]), dict(c[2]) if len(c) > 2 else {}) for c in calls]
    if processes > 1 and len(calls) > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(min(processes, len(calls))) as pool:
            return pool.starmap(_call, calls)
    return [_call(*c) for c in calls]


# ----------------------------------------------------------------------------------
# the five workloads, with sizes scaled by `scale` for tests
# ----------------------------------------------------------------------------------

def config1(scale: float = 1.0):
    """Plain join, tiny: |R|=1,000, |S|=10,000, d=10,000, nnz U{20..100}, f32, k=10."""
    nr, ns = max(1, int(1000 * scale)), max(1, int(10000 * scale))
    S = uniform_f32(ns, 10000, 20, 100, config_seed(1, "S"))
    R = uniform_f32(nr, 10000, 20, 100, config_seed(1, "R"))
    return R, S, 10


def config2(scale: float = 1.0, n_r: int | None = None, n_s: int | None = None):
    """Spectrum-shaped: |R|=100,000, |S|=2,000,000, d=10,000, u8 1..100, k=5."""
    nr = n_r if n_r is not None else max(1, int(100000 * scale))
    ns = n_s if n_s is not None else max(1, int(2000000 * scale))
    S = spectrum_u8(ns, config_seed(2, "S"), role="S")
    R = spectrum_u8(nr, config_seed(2, "R"), role="R")
    return R, S, 5


def config3_jobs(n_jobs: int = 64, scale: float = 1.0):
    """64 uneven joins: |R| log-U[100, 50k], |S| log-U[1e4, 1e6], k in {1,5,10,20,50}."""
    rng = np.random.default_rng(config_seed(3, "mix"))
    jobs = []
    for j in range(n_jobs):
        nr = int(round(math.exp(rng.uniform(math.log(100), math.log(50000)))))
        ns = int(round(math.exp(rng.uniform(math.log(1e4), math.log(1e6)))))
        k = int(rng.choice([1, 5, 10, 20, 50]))
        jobs.append(dict(n_r=max(1, int(nr * scale)), n_s=max(1, int(ns * scale)), k=k,
                         seed=config_seed(3, "S") + 1000 * j))
    return jobs


def config3_job_data(job: dict):
    S = spectrum_u8(job["n_s"], job["seed"], role="S")
    R = spectrum_u8(job["n_r"], job["seed"] + 1, role="R")
    return R, S, job["k"]


def config4(scale: float = 1.0, n_train: int | None = None, n_eval: int | None = None,
            n_s: int | None = None):
    """Learned threshold: |S|=5,000,000, 200,000 training and 1,000,000 eval queries, k=10."""
    ns = n_s if n_s is not None else max(1, int(5000000 * scale))
    nt = n_train if n_train is not None else max(1, int(200000 * scale))
    ne = n_eval if n_eval is not None else max(1, int(1000000 * scale))
    S = spectrum_u8(ns, config_seed(4, "S"), role="S")
    T = spectrum_u8(nt, config_seed(4, "train"), role="R")
    E = spectrum_u8(ne, config_seed(4, "eval"), role="R")
    return T, E, S, 10


def config5(scale: float = 1.0, n_r: int | None = None, n_s: int | None = None, processes: int = 1):
    """Float scale-up: |R|=1M, |S|=10M, d=50,000, Zipf(1.1) ids, L2-normalised, k=20."""
    nr = n_r if n_r is not None else max(1, int(1000000 * scale))
    ns = n_s if n_s is not None else max(1, int(10000000 * scale))
    S = zipf_f32(ns, config_seed(5, "S"), processes=processes)
    R = zipf_f32(nr, config_seed(5, "R"), processes=processes)
    return R, S, 20
