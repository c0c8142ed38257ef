"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

* H1 / H2: hand-worked examples (tests/golden/), Section 3 and Algorithms 1, 4.
* A dense numpy matmul with a stable sort (library special case of eq. 1).
* A pure-Python dict brute force on tiny inputs.
* Theorem 1: BF, IIB and IIIB return the same result for every R/S block split and k.
* eq. 4: IIB touches exactly sum_r sum_{d in r} |I_d| postings; eq. 3 bounds BF.
* Planted mistakes in a copy of the oracle source fail at least one of these pins.
"""
import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from paper_1011_2807_gb300 import synth
import goldens
import refdefs

ALGOS = ("bf_join", "iib_join", "iiib_join")


def _run(oracle_mod, name, R, S, k, **kw):
    fn = getattr(oracle_mod, name)
    if name == "bf_join":
        kw.pop("rblock", None)
        kw.pop("sblock", None)
    return fn(R, S, k, **kw)


def random_u8(n, dim, nnz_hi, seed, wmax=100):
    rng = np.random.default_rng(seed)
    rows = []
    for _ in range(n):
        m = int(rng.integers(0, min(nnz_hi, dim) + 1))
        d = rng.choice(dim, size=m, replace=False)
        w = rng.integers(1, wmax + 1, size=m)
        rows.append(list(zip(d.tolist(), w.tolist())))
    return synth.from_rows(rows, dim, np.uint8)


def random_f32(n, dim, nnz_hi, seed):
    rng = np.random.default_rng(seed)
    rows = []
    for _ in range(n):
        m = int(rng.integers(0, min(nnz_hi, dim) + 1))
        d = rng.choice(dim, size=m, replace=False)
        w = (1.0 - rng.random(m)).astype(np.float32)
        rows.append(list(zip(d.tolist(), w.tolist())))
    return synth.from_rows(rows, dim, np.float32)


# ----------------------------------------------------------------------------------
# hand-worked examples
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("algo", ALGOS)
def test_h1_hand_example(oracle_mod, algo):
    g = goldens.load("h1_topk.txt")
    for k, exp in g["cases"]:
        ids, sc, _ = _run(oracle_mod, algo, g["R"], g["S"], k)
        eids, esc = goldens.expected_arrays(exp, g["R"].n_rows, k)
        np.testing.assert_array_equal(ids, eids)
        np.testing.assert_array_equal(sc, esc)


def test_h2_iiib_trace(oracle_mod):
    g = goldens.load("h2_iiib_trace.txt")
    (k, exp), = g["cases"]
    sb = g["extra"]["sblock"]
    ids, sc, st = oracle_mod.iiib_join(g["R"], g["S"], k, sblock=sb)
    eids, esc = goldens.expected_arrays(exp, g["R"].n_rows, k)
    np.testing.assert_array_equal(ids, eids)
    np.testing.assert_array_equal(sc, esc)
    assert st["postings_touched"] == g["extra"]["touched_total"]
    assert st["postings_indexed"] == g["extra"]["indexed_total"]
    # block 1 alone: the same 6 touches, so block 2 touched none
    _, _, st1 = oracle_mod.iiib_join(g["R"], g["S"].slice_rows(0, sb), k)
    assert st1["postings_touched"] == g["extra"]["touched_block1"]
    # IIB on the same split scans block 2's lists (r0: 2, r1: 1)
    _, _, st_iib = oracle_mod.iib_join(g["R"], g["S"], k, sblock=sb)
    assert st_iib["postings_touched"] == g["extra"]["touched_total"] + 3


# ----------------------------------------------------------------------------------
# library special case and brute force
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("algo", ALGOS)
def test_dense_matmul_u8(oracle_mod, algo, seed):
    dim = [5, 12, 40, 200, 8, 30][seed]
    R = random_u8(13, dim, 9, 100 + seed, wmax=[3, 100, 255, 100, 2, 7][seed])
    S = random_u8(29, dim, 11, 200 + seed, wmax=[3, 100, 255, 100, 2, 7][seed])
    for k in (1, 3, 7, 40):
        ids, sc, _ = _run(oracle_mod, algo, R, S, k, rblock=4, sblock=7)
        eids, esc, _ = refdefs.dense_topk(R, S, k)
        np.testing.assert_array_equal(ids, eids)
        np.testing.assert_array_equal(sc, esc.astype(np.float64))


@pytest.mark.parametrize("algo", ALGOS)
def test_dense_matmul_f32(oracle_mod, algo):
    R = random_f32(11, 60, 15, 7)
    S = random_f32(37, 60, 15, 8)
    for k in (1, 5, 50):
        ids, sc, _ = _run(oracle_mod, algo, R, S, k, rblock=3, sblock=10)
        eids, esc, _ = refdefs.dense_topk(R, S, k, np.float64)
        np.testing.assert_array_equal(ids, eids)
        np.testing.assert_allclose(sc, esc, rtol=1e-12, atol=0)


@pytest.mark.parametrize("algo", ALGOS)
def test_dict_brute_force(oracle_mod, algo):
    R = random_u8(9, 15, 6, 11, wmax=4)
    S = random_u8(21, 15, 6, 12, wmax=4)
    for k in (1, 2, 5, 25):
        ids, sc, _ = _run(oracle_mod, algo, R, S, k, rblock=2, sblock=5)
        eids, esc = refdefs.dict_topk(R, S, k)
        np.testing.assert_array_equal(ids, eids)
        np.testing.assert_array_equal(sc, esc)


def test_config1_shape_against_dense(oracle_mod):
    R, S, k = synth.config1(scale=0.02)
    ids, sc, _ = oracle_mod.bf_join(R, S, k, threads=4)
    eids, esc, _ = refdefs.dense_topk(R, S, k, np.float64)
    np.testing.assert_array_equal(ids, eids)
    np.testing.assert_allclose(sc, esc, rtol=1e-12)


# ----------------------------------------------------------------------------------
# Theorem 1 (IIIB finds every s with dot > pruneScore), for every block split
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(4))
def test_theorem1_block_splits(oracle_mod, seed):
    R = random_u8(7, 10, 6, 300 + seed, wmax=3)
    S = random_u8(11, 10, 6, 400 + seed, wmax=3)
    ref_cache = {}
    for k in range(1, S.n_rows + 2):
        ref_cache[k] = oracle_mod.bf_join(R, S, k)[:2]
    for rb in (1, 2, 3, 0):
        for sb in (1, 2, 3, 5, 0):
            for k in (1, 2, 3, 5, S.n_rows + 1):
                eids, esc = ref_cache[k]
                for algo in ("iib_join", "iiib_join"):
                    ids, sc, _ = _run(oracle_mod, algo, R, S, k, rblock=rb, sblock=sb)
                    np.testing.assert_array_equal(ids, eids, err_msg=f"{algo} rb={rb} sb={sb} k={k}")
                    np.testing.assert_array_equal(sc, esc)


def test_theorem1_spectrum_shaped(oracle_mod):
    R = synth.spectrum_u8(40, 5, role="R")
    S = synth.spectrum_u8(600, 6, role="S")
    eids, esc, _ = oracle_mod.bf_join(R, S, 5, threads=4)
    for rb, sb in ((8, 100), (40, 64), (1, 600)):
        ids, sc, st3 = oracle_mod.iiib_join(R, S, 5, rblock=rb, sblock=sb)
        np.testing.assert_array_equal(ids, eids)
        np.testing.assert_array_equal(sc, esc)
        _, _, st2 = oracle_mod.iib_join(R, S, 5, rblock=rb, sblock=sb)
        # the refinement only removes work
        assert st3["postings_touched"] <= st2["postings_touched"]
        assert st3["postings_indexed"] <= st2["postings_indexed"]


# ----------------------------------------------------------------------------------
# cost counters: eq. 4 exactly, eq. 3 as a bound
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("sb", [0, 3, 17])
def test_eq4_posting_count(oracle_mod, sb):
    R = random_u8(15, 25, 9, 21)
    S = random_u8(40, 25, 9, 22)
    _, _, st = oracle_mod.iib_join(R, S, 3, rblock=4, sblock=sb)
    assert st["postings_touched"] == refdefs.postings_touched_iib(R, S)
    n_rblocks = -(-R.n_rows // 4)
    assert st["postings_indexed"] == S.nnz * n_rblocks   # first term of eq. 4 per R block


def test_eq3_merge_bound(oracle_mod):
    R = random_u8(10, 30, 12, 31)
    S = random_u8(20, 30, 12, 32)
    _, _, st = oracle_mod.bf_join(R, S, 2)
    assert 0 < st["merge_steps"] <= refdefs.bf_cost_c2(R, S)


# ----------------------------------------------------------------------------------
# degenerate cases
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("algo", ALGOS)
def test_degenerate(oracle_mod, algo):
    empty = synth.from_rows([], 8)
    some = synth.from_rows([[(1, 1)], [], [(1, 2), (7, 1)]], 8)
    ids, sc, _ = _run(oracle_mod, algo, empty, some, 3)
    assert ids.shape == (0, 3)
    ids, sc, _ = _run(oracle_mod, algo, some, empty, 2)
    assert (ids == -1).all() and (sc == 0).all()
    # identical vectors: all scores tie, ids must come out ascending
    same = synth.from_rows([[(2, 3), (5, 1)]] * 6, 8)
    ids, sc, _ = _run(oracle_mod, algo, same.slice_rows(0, 1), same, 4, sblock=2)
    assert ids.tolist() == [[0, 1, 2, 3]] and sc.tolist() == [[10.0] * 4]
    # no overlap at all
    a = synth.from_rows([[(0, 5)]], 8)
    b = synth.from_rows([[(1, 5)], [(2, 5)]], 8)
    ids, sc, _ = _run(oracle_mod, algo, a, b, 2)
    assert ids.tolist() == [[-1, -1]]


# ----------------------------------------------------------------------------------
# planted mistakes (in a copy of the oracle, on the CPU) are caught by the pins
# ----------------------------------------------------------------------------------

MUTANTS = [
    ("ret += wval(R, i) * wval(S, j);", "ret += wval(R, i) * wval(S, j) * (j % 2 ? 1.0 : 0.5);"),
    ("} else if (dr > ds) {", "} else if (dr < ds) {"),
    ("while (p < c->size && c->sc[p] >= v) p++;", "while (p < c->size && c->sc[p] > v) p++;"),
    ("cand_insert(&c, s, A[s - s0]);\n                            A[s - s0] = 0.0;",
     "cand_insert(&c, s, A[s - s0]);"),
    ("A[I.sid[p] - s0] += rw * I.w[p];\n                            touched++;\n                        }\n                    }\n                    for (int64_t s = s0; s < s1; s++) {\n                        if (A[s - s0] != 0.0) {\n                            if",
     "A[I.sid[p] - s0] += I.w[p];\n                            touched++;\n                        }\n                    }\n                    for (int64_t s = s0; s < s1; s++) {\n                        if (A[s - s0] != 0.0) {\n                            if"),
    ("if (t > mps) { removed[j - j0] = 1;", "if (t >= mps) { removed[j - j0] = 1;"),
    ("t += maxw[d] * wval(S, j);", "t += wval(S, j);"),
    ("if (x->id < y->id) return -1;\n    if (x->id > y->id) return 1;",
     "if (x->id < y->id) return 1;\n    if (x->id > y->id) return -1;"),
]


def _mutant_lib(src, old, new, tmp):
    assert old in src, old
    path = os.path.join(tmp, "m.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new, 1))
    so = os.path.join(tmp, f"m{abs(hash(new))}.so")
    subprocess.run(["gcc", "-O1", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-o", so, path],
                   check=True)
    return so


def _pins_pass(oracle_mod, lib_path):
    """Re-run a subset of the pins against another build of the oracle source."""
    saved = oracle_mod._lib
    try:
        lib = ctypes.CDLL(lib_path)
        P = ctypes.POINTER
        lib.oracle_bf_join.argtypes = [P(oracle_mod._CSR), P(oracle_mod._CSR), ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                       P(oracle_mod._Stats)]
        for name in ("oracle_iib_join", "oracle_iiib_join"):
            getattr(lib, name).argtypes = [P(oracle_mod._CSR), P(oracle_mod._CSR), ctypes.c_int32,
                                           ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                           ctypes.c_void_p, ctypes.c_void_p, P(oracle_mod._Stats)]
        oracle_mod._lib = lib
        checks = [
            lambda: [test_h1_hand_example(oracle_mod, a) for a in ALGOS],
            lambda: test_h2_iiib_trace(oracle_mod),
            lambda: [test_dense_matmul_u8(oracle_mod, a, s) for a in ALGOS for s in range(3)],
            lambda: test_theorem1_block_splits(oracle_mod, 0),
            lambda: [test_degenerate(oracle_mod, a) for a in ALGOS],
            lambda: test_eq4_posting_count(oracle_mod, 3),
        ]
        for c in checks:
            try:
                c()
            except AssertionError:
                return False
        return True
    finally:
        oracle_mod._lib = saved


def test_planted_mistakes_are_caught(oracle_mod):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    with open(oracle_mod._SRC) as f:
        src = f.read()
    tmp = tempfile.mkdtemp(prefix="oracle_mut_")
    try:
        # the unmodified source passes
        assert _pins_pass(oracle_mod, _mutant_lib(src, "#include <stdint.h>", "#include <stdint.h>", tmp))
        for old, new in MUTANTS:
            assert not _pins_pass(oracle_mod, _mutant_lib(src, old, new, tmp)), f"mutant survived: {new}"
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
