"""Reader for the hand-worked fixtures under tests/golden/ (plain text)."""
import os

import numpy as np

from paper_1011_2807_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _feat(tok):
    d, w = tok.split(":")
    return int(d), int(w)


def load(name):
    """Returns dict(S=CSR, R=CSR, cases=[(k, {row: [(id, score)]})], extra={key: int})."""
    dim = None
    S, R = [], []
    cases = []
    extra = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "dim":
                dim = int(tok[1])
            elif tok[0] == "S":
                S.append([_feat(t) for t in tok[1:]])
            elif tok[0] == "R":
                R.append([_feat(t) for t in tok[1:]])
            elif tok[0] == "k":
                cases.append((int(tok[1]), {}))
            elif tok[0] == "expect":
                cases[-1][1][int(tok[1])] = [_feat(t) for t in tok[2:]]
            else:
                extra[tok[0]] = int(tok[1])
    return dict(S=synth.from_rows(S, dim), R=synth.from_rows(R, dim), cases=cases, extra=extra)


def expected_arrays(exp, n_rows, k):
    ids = np.full((n_rows, k), -1, np.int64)
    sc = np.zeros((n_rows, k), np.int64)
    for r, lst in exp.items():
        for q, (i, s) in enumerate(lst):
            ids[r, q], sc[r, q] = i, s
    return ids, sc
