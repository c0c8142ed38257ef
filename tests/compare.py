"""Result comparison between the CUDA path and the CPU oracle.

uint8 inputs: ids and int32 scores must be identical (bit-exact).
float32 inputs: each returned score within RTOL (relative) of the exact score of the
returned id, the score lists within RTOL position by position, and ids may differ
from the oracle's only where both ids' exact scores lie within RTOL of the row's
k-th score (boundary ties).  RTOL = 1e-5: the tolerance the workload fixes for
float scores.
"""
import numpy as np

RTOL = 1e-5


def exact_scores(R, S, rows, ids):
    """fp64 dot(r, s) for the given (row, id) pairs; -1 ids give 0."""
    out = np.zeros(ids.shape, np.float64)
    for a, r in enumerate(rows):
        d, w = R.row(int(r))
        rd = dict(zip(d.tolist(), w.astype(np.float64).tolist()))
        for b, s in enumerate(ids[a]):
            if s < 0:
                continue
            sd, sw = S.row(int(s))
            out[a, b] = sum(rd.get(x, 0.0) * float(y) for x, y in zip(sd.tolist(), sw.tolist()))
    return out


def assert_exact(gids, gsc, eids, esc, what=""):
    gids = np.asarray(gids)
    gsc = np.asarray(gsc)
    bad = np.nonzero((gids != eids).any(axis=1) | (gsc.astype(np.float64) != esc).any(axis=1))[0]
    if bad.size:
        i = int(bad[0])
        raise AssertionError(f"{what}: {bad.size} rows differ; first row {i}: "
                             f"gpu {gids[i].tolist()} {gsc[i].tolist()} vs oracle {eids[i].tolist()} {esc[i].tolist()}")


def assert_close(R, S, rows, gids, gsc, eids, esc, rtol=RTOL, what=""):
    gids = np.asarray(gids)
    gsc = np.asarray(gsc).astype(np.float64)
    # returned scores vs exact score of the returned id
    ex = exact_scores(R, S, rows, gids)
    valid = gids >= 0
    err = np.abs(gsc - ex)
    assert np.all(err[valid] <= rtol * ex[valid] + 1e-30), f"{what}: score of a returned id off by > rtol"
    assert np.all(gsc[~valid] == 0)
    # same number of entries per row
    assert np.array_equal((gids >= 0).sum(1), (eids >= 0).sum(1)), f"{what}: entry counts differ"
    # score lists agree position by position
    assert np.all(np.abs(gsc - esc) <= rtol * np.maximum(np.abs(esc), 1e-30) + 1e-30), f"{what}: score lists differ"
    # ids: differences only at the boundary
    for a in range(gids.shape[0]):
        G = set(gids[a][gids[a] >= 0].tolist())
        E = set(eids[a][eids[a] >= 0].tolist())
        if G == E:
            continue
        kth = esc[a][eids[a] >= 0].min()
        for s in G ^ E:
            v = exact_scores(R, S, [rows[a]], np.array([[s]]))[0, 0]
            assert abs(v - kth) <= rtol * kth, f"{what}: row {rows[a]} id {s} ({v}) not a boundary tie of {kth}"
