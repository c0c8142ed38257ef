"""Independent statements of the KNN-join result used to pin the oracle.

Nothing here is the oracle: each function restates the result definition (Section 3,
eq. 1) through a different route -- a dense matmul from numpy, or Python dicts -- so
that a mistake in the oracle's merge, index or insertion code shows up as a mismatch.
"""
import numpy as np


def dense_topk(R, S, k, dtype=np.int64):
    """Dense R.S^T (numpy matmul), then a stable sort by (-score, id), positives only."""
    A = R.to_dense(dtype) @ S.to_dense(dtype).T if R.n_rows and S.n_rows else \
        np.zeros((R.n_rows, S.n_rows), dtype)
    ids = np.full((R.n_rows, k), -1, np.int64)
    sc = np.zeros((R.n_rows, k), dtype)
    for i in range(R.n_rows):
        row = A[i]
        order = np.argsort(-row, kind="stable")   # ties keep ascending id
        order = order[row[order] > 0][:k]
        ids[i, :len(order)] = order
        sc[i, :len(order)] = row[order]
    return ids, sc, A


def dict_topk(R, S, k):
    """Pure-Python brute force: dict lookups for dot(r, s), sorted() with a key."""
    srows = []
    for j in range(S.n_rows):
        d, w = S.row(j)
        srows.append({int(a): float(b) for a, b in zip(d, w)})
    out_ids, out_sc = [], []
    for i in range(R.n_rows):
        d, w = R.row(i)
        r = {int(a): float(b) for a, b in zip(d, w)}
        scores = []
        for j, s in enumerate(srows):
            v = sum(r[x] * s[x] for x in r.keys() & s.keys())
            if v > 0:
                scores.append((v, j))
        scores = sorted(scores, key=lambda t: (-t[0], t[1]))[:k]
        scores += [(0.0, -1)] * (k - len(scores))
        out_ids.append([j for _, j in scores])
        out_sc.append([v for v, _ in scores])
    return np.asarray(out_ids, np.int64).reshape(R.n_rows, k), \
        np.asarray(out_sc, np.float64).reshape(R.n_rows, k)


def postings_touched_iib(R, S):
    """Second term of eq. 4: sum over r, over d in r, of |I_d| (list length = df_S(d))."""
    df = np.bincount(S.indices, minlength=S.dim).astype(np.int64)
    return int(df[R.indices].sum())


def bf_cost_c2(R, S):
    """eq. 3: sum over (r_i, s_j) of |r_i| + |s_j|."""
    lr = np.diff(R.indptr).astype(np.int64)
    ls = np.diff(S.indptr).astype(np.int64)
    return int(lr.sum() * S.n_rows + ls.sum() * R.n_rows)
